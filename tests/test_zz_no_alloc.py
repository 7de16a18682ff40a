"""sun_plaquette_noalloc: the plaquette for callers that cannot allocate device
memory (code confined to a memory arena it does not own, latency-critical
loops that cannot afford an allocation's implicit synchronisation).  Called
through the C ABI on a lattice's own link storage and compared with
sun_plaquette and with the oracle's plaquette of the same links, twice in a
row (the fixed scratch array keeps the previous call's contents and must be
re-armed each time), from 960 sites up to exactly the array's limit of
16,777,216 sites (65,536 reduction blocks, far beyond sun_plaquette's grid of
at most 1024).  Kept in the last-collected file so that a run stopping at the
first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

import oracle as orc
from tests.oracle_configs import cold_thermal, tiled

pytestmark = pytest.mark.gpu

CAP_SITES = 16777216


@pytest.fixture(scope="module")
def sunlib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1112_4533_gb300 import build as b
    b.build()
    import paper_1112_4533_gb300 as p
    p.load_library()
    return p


def noalloc_twice(lib, L, nc, dims, prec, storage):
    """Two calls in a row on the lattice's stream into a caller-owned device buffer."""
    import torch
    info = L.info()
    out = torch.full((2,), -7.0, dtype=torch.float64, device="cuda")
    d = (ctypes.c_int * 4)(*dims)
    for k in range(2):
        ptr = ctypes.cast(out.data_ptr() + 8 * k, ctypes.POINTER(ctypes.c_double))
        st = lib.sun_plaquette_noalloc(ctypes.c_void_p(info.links), nc, d, prec, storage, ptr,
                                       ctypes.c_void_p(L.stream.cuda_stream))
        assert st == 0, lib.sun_last_error()
    L.stream.synchronize()
    return out.cpu().numpy()


# (nc, dims, precision, storage, beta, oracle tile, tolerance)
CASES = [
    (3, (8, 6, 4, 10), 32, 12, 6.0, None, 2e-6),
    (3, (16, 16, 16, 16), 32, 18, 6.0, None, 2e-6),
    (2, (8, 8, 8, 8), 64, 4, 2.3, None, 1e-14),
    (4, (4, 4, 6, 4), 32, 32, 11.2, None, 2e-6),
    # 63,488 reduction blocks, then exactly the limit (65,536 blocks)
    (2, (64, 64, 64, 62), 32, 4, 2.3, (16, 16, 16, 62), 2e-6),
    (2, (64, 64, 64, 64), 32, 4, 2.3, (16, 16, 16, 16), 2e-6),
]


@pytest.mark.parametrize("nc,dims,prec,storage,beta,tile,tol", CASES)
def test_noalloc_plaquette_matches_sun_plaquette_and_oracle(sunlib, nc, dims, prec, storage, beta, tile, tol):
    lib = sunlib.load_library()
    if tile is None:
        U = cold_thermal(nc, dims, beta)
    else:
        U = tiled(cold_thermal(nc, tile, beta), tuple(a // b for a, b in zip(dims, tile)))
    assert U.shape[1:5] == tuple(reversed(dims))
    want_oracle = orc.plaquette(U)
    with sunlib.Lattice(nc, dims, beta, seed=5, precision=prec, storage=storage) as L:
        L.import_links(U)
        del U
        want = L.plaquette()
        results = noalloc_twice(lib, L, nc, dims, prec, storage)
    assert np.abs(results - want).max() < tol, (results, want)
    assert np.abs(results - want_oracle).max() < tol, (results, want_oracle)
    assert results[0] == results[1]  # same reduction order both times


@pytest.mark.parametrize("dims", [(64, 64, 64, 66), (2, 4, 2, 1048578)])
def test_noalloc_rejects_lattices_beyond_its_scratch(sunlib, dims):
    """Above 16,777,216 sites (the second shape is 32 sites above) the call is
    refused before any device work."""
    v = dims[0] * dims[1] * dims[2] * dims[3]
    assert v > CAP_SITES
    lib = sunlib.load_library()
    d = (ctypes.c_int * 4)(*dims)
    dummy = ctypes.cast(ctypes.c_void_p(256), ctypes.POINTER(ctypes.c_double))
    st = lib.sun_plaquette_noalloc(ctypes.c_void_p(256), 3, d, 32, 12, dummy, None)
    assert st == 1
    assert b"at most 16777216 sites" in lib.sun_last_error()
