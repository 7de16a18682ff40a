"""GPU tests of the packed-FP32 overrelaxation pass (variant bit 16, SU(3) FP32):
two links per thread with {add,sub,mul,fma}.rn.f32x2 must give bitwise the
links of the one-link kernel -- both storage formats, every re-unitarization
placement, ragged tails (lane 1 idle), a subgroup skipped in one lane only,
graphs, batches -- and hence the oracle's links within the FP32 bound."""
import numpy as np
import pytest

import oracle as orc
from tests.inputs import random_gauge_config

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


def evolve(p, dims, storage, variant, reunit_mode=0, sweeps=2, n_hb=1, n_or=3, seed=5, **kw):
    with p.Lattice(3, dims, 6.0, hot_start=True, seed=seed, storage=storage, variant=variant,
                   reunit_mode=reunit_mode, **kw) as L:
        plaq, poly = L.run(sweeps, n_hb, n_or)
        return L.export_links(), plaq, poly


@pytest.mark.parametrize("storage", [12, 18])
@pytest.mark.parametrize("reunit_mode", [0, 1, 2])
def test_packed_equals_one_link_kernel(sunlib, storage, reunit_mode):
    # 6x6x4x8: 576 links per pass, two 256-link blocks and a ragged third
    for dims in [(6, 6, 4, 8), (8, 8, 8, 8)]:
        a = evolve(sunlib, dims, storage, 1, reunit_mode)
        b = evolve(sunlib, dims, storage, 17, reunit_mode)
        assert np.array_equal(a[0], b[0]), dims
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_packed_with_graphs_off_and_small_blocks(sunlib):
    dims = (4, 4, 4, 6)
    a = evolve(sunlib, dims, 12, 0, block_threads=64)
    b = evolve(sunlib, dims, 12, 16, use_graphs=False)
    assert np.array_equal(a[0], b[0])


def test_packed_pass_follows_the_oracle(sunlib):
    dims = (8, 6, 4, 6)
    U0 = random_gauge_config(3, dims, 31)
    for storage in (12, 18):
        with sunlib.Lattice(3, dims, 6.0, seed=4, storage=storage, variant=16) as L:
            L.import_links(U0)
            L.update_pass(sunlib.OVERRELAX, 3, 0)
            got = L.export_links()
        want = U0.copy()
        orc.update_pass(want, 6.0, orc.OVERRELAX, 3, 0, 0, 4)
        assert np.abs(got - want).max() < 1e-5


def test_subgroup_skipped_in_one_lane(sunlib):
    """At one site the (0,1) block of the staple cancels (U_mu(x - nu) =
    diag(-1, -1, 1) for every nu != mu, all else 1): that lane skips its first
    subgroup while its partner lane updates."""
    dims = (4, 4, 4, 4)
    U = orc.init(3, dims, False, 1)
    mu, x = 0, (2, 2, 2, 2)
    for nu in (1, 2, 3):
        c = list(x)
        c[nu] -= 1
        U[mu, c[3], c[2], c[1], c[0]] = np.diag([-1.0, -1.0, 1.0])  # SU(3): det = 1
    out = []
    for variant in (0, 16):
        with sunlib.Lattice(3, dims, 6.0, seed=2, storage=18, variant=variant) as L:
            L.import_links(U)
            L.update_pass(sunlib.OVERRELAX, mu, 0)
            out.append(L.export_links())
    assert np.array_equal(out[0], out[1])


def test_batch_of_packed_lattices_evolves_as_alone(sunlib):
    specs = [((4, 4, 4, 4), 11), ((6, 4, 6, 4), 12), ((24, 24, 24, 24), 13)]
    alone = []
    for dims, seed in specs:
        with sunlib.Lattice(3, dims, 6.1, hot_start=True, seed=seed, variant=17) as L:
            L.run(2, 1, 2)
            alone.append(L.export_links())
    lats = [sunlib.Lattice(3, dims, 6.1, hot_start=True, seed=seed, variant=17) for dims, seed in specs]
    with sunlib.Batch(lats) as B:
        B.run(2, 1, 2)
    for L, U in zip(lats, alone):
        assert np.array_equal(L.export_links(), U)
        L.close()
