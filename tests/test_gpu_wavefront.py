"""GPU tests of the wavefront launches (variant bit 8): the even and the odd pass
of one direction (Sec. 3) in a single launch, odd units of slice t started
once the even units of slices t-1, t, t+1 are done.

Each link is then updated from the same neighbour values as with two separate
passes, so every case here demands bitwise equality with the two-pass
schedule (itself held to the oracle by the parity tests), across kernels,
re-unitarization placements, ragged t-slices (a slice's half-sites not a
multiple of the block), lags, block sizes, more units than resident blocks,
batches and graphs.  The bounded device-side wait is checked by making it run
out on purpose: with wave_skip_units the first unit (the even links of slice
0) is left out, so the odd units that need it never see it finish; the launch
must end, report SUN_ERR_TIMEOUT once and leave the context usable.
"""
import numpy as np
import pytest

import oracle as orc

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


def evolve(p, nc, dims, storage, prec, variant, reunit_mode=0, sweeps=2, n_hb=1, n_or=2, seed=5, **kw):
    with p.Lattice(nc, dims, beta_for(nc), hot_start=True, seed=seed, storage=storage, precision=prec,
                   variant=variant, reunit_mode=reunit_mode, **kw) as L:
        plaq, poly = L.run(sweeps, n_hb, n_or)
        return L.export_links(), plaq, poly


def assert_same(a, b):
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


# (nc, storage, precision, base variant, re-unitarization modes)
KERNELS = [(2, 4, 32, 0, (0, 1, 2)), (2, 4, 64, 0, (0, 1)), (2, 8, 32, 0, (0, 1)), (3, 12, 32, 0, (0, 1, 2)),
           (3, 12, 32, 1, (0, 1)), (3, 18, 32, 1, (0, 1)), (3, 12, 64, 0, (0, 1)), (4, 32, 32, 0, (0, 1)),
           (5, 50, 32, 0, (0,)), (6, 72, 32, 4, (0, 1)), (6, 72, 64, 4, (0,))]


@pytest.mark.parametrize("nc,st,prec,var,modes", KERNELS)
def test_wavefront_equals_two_passes(sunlib, nc, st, prec, var, modes):
    # 6x6x4: 72 half-sites per slice (a ragged chunk for every block size)
    dims = (6, 6, 4, 8)
    for mode in modes:
        two = evolve(sunlib, nc, dims, st, prec, var, mode)
        wave = evolve(sunlib, nc, dims, st, prec, var | 8, mode)
        assert_same(two, wave)


@pytest.mark.parametrize("lag", [1, 2, 7, 100])
def test_wavefront_lag_does_not_change_results(sunlib, lag):
    dims = (8, 4, 6, 8)
    ref = evolve(sunlib, 3, dims, 12, 32, 1)
    assert_same(ref, evolve(sunlib, 3, dims, 12, 32, 9, wave_lag=lag))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 2), (2, 6, 2, 12)])
def test_wavefront_on_thin_lattices(sunlib, dims):
    for nc, st in ((2, 4), (3, 12)):
        assert_same(evolve(sunlib, nc, dims, st, 32, 0), evolve(sunlib, nc, dims, st, 32, 8))


@pytest.mark.parametrize("block", [32, 64, 256])
def test_wavefront_block_sizes(sunlib, block):
    dims = (6, 6, 6, 6)
    ref = evolve(sunlib, 3, dims, 12, 32, 0)
    assert_same(ref, evolve(sunlib, 3, dims, 12, 32, 8, block_threads=block))


def test_wavefront_with_more_units_than_resident_blocks(sunlib):
    """32^3 x 16 SU(3): 128 units per slice and parity, 4096 blocks per launch,
    several times what the GPU holds at once; with graphs and without."""
    dims = (32, 32, 32, 16)
    ref = evolve(sunlib, 3, dims, 12, 32, 1, reunit_mode=1, sweeps=2, n_hb=1, n_or=3)
    assert_same(ref, evolve(sunlib, 3, dims, 12, 32, 9, reunit_mode=1, sweeps=2, n_hb=1, n_or=3))
    assert_same(ref, evolve(sunlib, 3, dims, 12, 32, 9, reunit_mode=1, sweeps=2, n_hb=1, n_or=3, use_graphs=False))


def test_wavefront_pass_follows_the_oracle(sunlib):
    """One FP64 sweep with wavefront launches against the oracle directly."""
    dims = (4, 6, 4, 6)
    from tests.inputs import random_gauge_config
    U0 = random_gauge_config(3, dims, 80)
    with sunlib.Lattice(3, dims, 6.0, seed=9, precision=64, storage=18, variant=8) as L:
        L.import_links(U0)
        L.sweep(1, 2)
        got = L.export_links()
    want = U0.copy()
    orc.sweep(want, 6.0, 1, 2, True, 9, 0)
    assert np.abs(got - want).max() < 1e-11


def test_large_chain_in_a_batch_uses_wavefront_launches(sunlib):
    # SU(4) 20^4 fills the GPU on its own: it runs its own (wavefront) launches in the batch
    specs = [(4, (20, 20, 20, 20), 11.0, 41), (4, (4, 4, 4, 6), 11.0, 42)]
    alone = []
    for nc, dims, beta, seed in specs:
        with sunlib.Lattice(nc, dims, beta, hot_start=True, seed=seed) as L:
            alone.append((L.run(2, 1, 1), L.export_links()))
    lats = [sunlib.Lattice(nc, dims, beta, hot_start=True, seed=seed, variant=8) for nc, dims, beta, seed in specs]
    with sunlib.Batch(lats) as B:
        plaq, poly = B.run(2, 1, 1)
    for i, L in enumerate(lats):
        (p1, l1), U = alone[i]
        assert np.array_equal(L.export_links(), U)
        assert np.abs(plaq[:, i] - p1).max() < 1e-12
        assert np.abs(poly[:, i] - l1).max() < 1e-12
        L.close()


def test_wavefront_wait_that_runs_out_is_reported(sunlib):
    dims = (4, 4, 4, 4)  # 32 half-sites per slice: one unit per (parity, slice)
    with sunlib.Lattice(3, dims, 6.0, hot_start=True, seed=3, variant=8, wave_skip_units=1) as L:
        L.sweep(0, 1)  # even slice 0 is never updated: the odd slices 3, 0, 1 wait for it
        with pytest.raises(sunlib.SunError) as e:
            L.synchronize()
        assert e.value.status == 4  # SUN_ERR_TIMEOUT
        L.synchronize()  # reported once, then cleared
    # the context is still usable
    ref = evolve(sunlib, 3, dims, 12, 32, 0)
    assert_same(ref, evolve(sunlib, 3, dims, 12, 32, 8))
