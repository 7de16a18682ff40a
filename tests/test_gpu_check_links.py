"""GPU tests of the link health check (sun_check_links): exact zeros on a cold
start, FP64 and FP32 rounding levels on Haar starts, drift that grows without
re-unitarization and vanishes with it, and non-finite or non-unitary links
counted and measured (the numbers checked against numpy on the same links)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sunlib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1112_4533_gb300 import build as b
    b.build()
    import paper_1112_4533_gb300 as p
    p.load_library()
    return p


def numpy_health(U):
    nc = U.shape[-1]
    m = U.reshape(-1, nc, nc)
    ok = np.isfinite(m.real).all(axis=(1, 2)) & np.isfinite(m.imag).all(axis=(1, 2))
    g = m[ok]
    dev = np.abs(g @ np.conj(np.swapaxes(g, 1, 2)) - np.eye(nc)).max()
    det = np.abs(np.linalg.det(g) - 1.0).max()
    return dev, det, int((~ok).sum())


@pytest.mark.parametrize("nc,st,prec", [(2, 4, 64), (3, 18, 64), (3, 12, 32), (4, 32, 32), (6, 72, 64)])
def test_health_of_starts(sunlib, nc, st, prec):
    with sunlib.Lattice(nc, (4, 4, 4, 4), 6.0, storage=st, precision=prec) as L:
        assert L.check_links() == (0.0, 0.0, 0)
    with sunlib.Lattice(nc, (4, 4, 4, 4), 6.0, hot_start=True, seed=2, storage=st, precision=prec) as L:
        dev, det, bad = L.check_links()
        want_dev, want_det, _ = numpy_health(L.export_links())
        assert bad == 0
        bound = 1e-13 if prec == 64 else 1e-5
        assert dev < bound and det < bound
        assert abs(dev - want_dev) < (1e-14 if prec == 64 else 1e-6)
        assert abs(det - want_det) < (1e-13 if prec == 64 else 1e-6)


def test_drift_and_reunitarization(sunlib):
    with sunlib.Lattice(3, (6, 6, 6, 6), 6.0, hot_start=True, seed=3, storage=18, reunit_every=0) as L:
        L.run(6, 1, 4)
        drift, _, _ = L.check_links()
        L.reunitarize()
        after, _, _ = L.check_links()
    assert drift > 10 * after and after < 1e-6


def test_bad_links_are_found(sunlib):
    dims = (4, 4, 4, 4)
    with sunlib.Lattice(3, dims, 6.0, hot_start=True, seed=4, storage=18, precision=64) as L:
        U = L.export_links()
        U[1, 2, 3, 0, 1] *= 2.0  # not unitary: U U^+ = 4 on the diagonal
        U[3, 0, 0, 0, 0, 1, 2] = np.nan
        L.import_links(U)
        dev, det, bad = L.check_links()
        want_dev, want_det, want_bad = numpy_health(L.export_links())
    assert bad == want_bad == 1
    assert abs(dev - want_dev) < 1e-12 and abs(dev - 3.0) < 1e-12
    assert abs(det - want_det) < 1e-12
