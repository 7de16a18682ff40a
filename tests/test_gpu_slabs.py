"""GPU tests of the t-slab decomposition (sun_slabs_*, Sec. 3's multi-GPU
scheme on one GPU): a lattice cut into 1, 2 or 4 slabs with a halo exchange
after every pass is bitwise the same chain as the whole lattice with the same
seed -- hot start, heatbath and overrelaxation, every re-unitarization
placement, the kernels of every Nc -- and its plaquette and Polyakov loop
agree to summation order."""
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


def beta_for(nc):
    return 2.3 if nc == 2 else (6.0 if nc == 3 else 0.7 * nc * nc)


# (nc, storage, precision, variant, re-unitarization modes)
CASES = [(2, 4, 32, 0, (0, 1, 2)), (2, 8, 64, 0, (0,)), (3, 12, 32, 1, (0, 1, 2)), (3, 18, 32, 16, (1,)),
         (3, 12, 64, 0, (0,)), (3, 12, 32, 9, (1,)), (4, 32, 32, 0, (1,)), (4, 32, 32, 1, (0, 2)),
         (6, 72, 32, 0, (0,))]


@pytest.mark.parametrize("nc,st,prec,var,modes", CASES)
@pytest.mark.parametrize("n_slabs", [1, 2, 4])
def test_slabs_follow_the_whole_lattice(sunlib, nc, st, prec, var, modes, n_slabs):
    dims = (4, 6, 4, 8)
    kw = dict(storage=st, precision=prec, variant=var)
    for mode in modes:
        with sunlib.Lattice(nc, dims, beta_for(nc), hot_start=True, seed=17, reunit_mode=mode, **kw) as L:
            U0 = L.export_links()
            p1, l1 = L.run(3, 1, 2)
            U1 = L.export_links()
        with sunlib.Slabs(nc, dims, n_slabs, beta_for(nc), hot_start=True, seed=17, reunit_mode=mode, **kw) as S:
            assert np.array_equal(S.export_links(), U0)
            p2, l2 = S.run(3, 1, 2)
            assert np.array_equal(S.export_links(), U1), (mode, n_slabs)
        assert np.abs(p1 - p2).max() < 1e-13
        assert np.abs(l1 - l2).max() < (1e-12 if prec == 64 else 2e-6)


def test_slabs_import_export_and_graphs(sunlib):
    dims = (6, 4, 4, 12)
    with sunlib.Lattice(3, dims, 6.0, hot_start=True, seed=3) as L:
        L.run(1, 1, 1)
        U = L.export_links()
        p1, _ = L.run(2, 1, 3)
        ref = L.export_links()
        step = L.heatbath_step
    for graphs in (True, False):
        with sunlib.Slabs(3, dims, 3, 6.0, hot_start=False, seed=3, use_graphs=graphs) as S:
            S.import_links(U)
            assert np.array_equal(S.export_links(), U)
            # the slabs' heatbath counters start at 0: advance them as the lattice's did
            S.run(1, 1, 0, plaquette=False, polyakov=False)
            S.import_links(U)
            p2, _ = S.run(2, 1, 3)
            assert np.array_equal(S.export_links(), ref)
            assert np.abs(p1 - p2).max() < 1e-13
    assert step == 3


def test_slab_arguments_are_checked(sunlib):
    for n in (3, 8, 0):
        with pytest.raises(sunlib.SunError):
            sunlib.Slabs(3, (4, 4, 4, 8), n, 6.0)


@pytest.mark.parametrize("nc,st,prec,n_hb,n_or", [(3, 18, 64, 1, 2), (3, 12, 64, 1, 2), (2, 4, 64, 1, 2),
                                                  (3, 12, 32, 0, 1)])
@pytest.mark.parametrize("n_slabs", [2, 4])
def test_slabs_follow_the_oracle(sunlib, nc, st, prec, n_hb, n_or, n_slabs):
    """The oracle's cold-start-thermalised configuration loaded into 2 or 4
    slabs; one sweep with the halo exchange after every pass and the
    re-unitarization, against the oracle's sweep of the whole lattice from the
    same links: FP64 links to 1e-11 (a heatbath and two overrelaxation steps),
    FP32 links to 1e-5 (one overrelaxation step: no accept/reject branch);
    the plaquette and Polyakov loop of the result against the oracle's."""
    import oracle as orc
    from tests.oracle_configs import cold_thermal
    dims = (4, 6, 4, 8)
    beta = beta_for(nc)
    U = cold_thermal(nc, dims, beta)
    with sunlib.Slabs(nc, dims, n_slabs, beta, hot_start=False, seed=23, storage=st, precision=prec) as S:
        S.import_links(U)
        p, l = S.run(1, n_hb, n_or)
        got = S.export_links()
    orc.sweep(U, beta, n_hb, n_or, True, 23, 0)
    assert np.abs(got - U).max() < (1e-11 if prec == 64 else 1e-5)
    assert abs(p[0] - orc.plaquette(U)) < (1e-12 if prec == 64 else 2e-6)
    assert abs(l[0] - orc.polyakov(U)) < (1e-12 if prec == 64 else 2e-5)
