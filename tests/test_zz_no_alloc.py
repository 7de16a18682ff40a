"""sun_plaquette_noalloc: the plaquette for callers that cannot allocate device
memory (memory arenas they do not own, work enqueued during CUDA-graph stream
capture, allocation-free latency-critical loops).  Called through the C ABI on
a lattice's own link storage and compared with sun_plaquette, twice in a row
(the fixed scratch array keeps the previous call's contents and must be
re-armed each time).  Kept in the last-collected file so that a run stopping at
the first failure has run every other test first."""
import ctypes

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


@pytest.mark.parametrize("nc,dims,prec,storage,beta,tol", [
    (3, (8, 6, 4, 10), 32, 12, 6.0, 2e-6),
    (3, (16, 16, 16, 16), 32, 18, 6.0, 2e-6),
    (2, (8, 8, 8, 8), 64, 4, 2.3, 1e-14),
    (4, (4, 4, 6, 4), 32, 32, 11.2, 2e-6),
])
def test_noalloc_plaquette_matches_sun_plaquette(sunlib, nc, dims, prec, storage, beta, tol):
    import torch
    lib = sunlib.load_library()
    with sunlib.Lattice(nc, dims, beta, hot_start=True, seed=5, precision=prec, storage=storage) as L:
        L.sweep(1, 2)
        want = L.plaquette()
        info = L.info()
        out = torch.full((2,), -7.0, dtype=torch.float64, device="cuda")
        d = (ctypes.c_int * 4)(*dims)
        results = []
        for k in range(2):
            ptr = ctypes.cast(out.data_ptr() + 8 * k, ctypes.POINTER(ctypes.c_double))
            st = lib.sun_plaquette_noalloc(ctypes.c_void_p(info.links), nc, d, prec, storage, ptr,
                                           ctypes.c_void_p(L.stream.cuda_stream))
            assert st == 0, lib.sun_last_error()
        L.stream.synchronize()
        results = out.cpu().numpy()
    assert np.abs(results - want).max() < tol, (results, want)
    assert results[0] == results[1]  # same reduction order both times


def test_noalloc_rejects_lattices_beyond_its_scratch(sunlib):
    lib = sunlib.load_library()
    d = (ctypes.c_int * 4)(64, 64, 64, 66)  # 17,301,504 sites > 16,777,216
    dummy = ctypes.cast(ctypes.c_void_p(256), ctypes.POINTER(ctypes.c_double))
    st = lib.sun_plaquette_noalloc(ctypes.c_void_p(256), 3, d, 32, 12, dummy, None)
    assert st == 1
    assert b"at most 16777216 sites" in lib.sun_last_error()
