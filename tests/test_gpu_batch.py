"""GPU tests of batches (sun_batch_*): many independent chains of mixed Nc,
extent, beta and seed swept by shared kernel launches.  A chain in a batch must
evolve exactly as it does alone (bitwise links: the same per-link kernels, its
own seed and heatbath counter), its observables must agree to rounding, and a
batch must match the oracle."""
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


# (nc, dims, beta, seed, storage, precision)
MIX = [
    (3, (4, 4, 4, 4), 5.7, 11, 12, 32),
    (3, (6, 6, 6, 6), 6.1, 12, 12, 32),
    (3, (8, 4, 6, 4), 6.3, 13, 12, 32),
    (2, (8, 8, 8, 8), 2.3, 14, 4, 32),
    (4, (4, 4, 4, 6), 11.0, 15, 32, 32),
    (3, (4, 6, 4, 8), 5.9, 16, 12, 32),
    (6, (4, 4, 4, 4), 25.0, 17, 72, 32),
]


def make(p, spec, **kw):
    nc, dims, beta, seed, st, prec = spec
    return p.Lattice(nc, dims, beta, hot_start=True, seed=seed, storage=st, precision=prec, **kw)


@pytest.mark.parametrize("reunit_mode", [0, 1])
def test_each_chain_in_a_mixed_batch_evolves_as_alone(sunlib, reunit_mode):
    sweeps = 3
    alone = []
    for spec in MIX:
        with make(sunlib, spec, reunit_mode=reunit_mode) as L:
            plaq, poly = L.run(sweeps, 1, 2)
            alone.append((L.export_links(), plaq, poly, L.heatbath_step))
    lats = [make(sunlib, spec, reunit_mode=reunit_mode) for spec in MIX]
    with sunlib.Batch(lats) as B:
        plaq, poly = B.run(sweeps, 1, 2)
    assert plaq.shape == (sweeps, len(MIX)) and poly.shape == (sweeps, len(MIX))
    for i, L in enumerate(lats):
        U, p1, l1, step = alone[i]
        assert np.array_equal(L.export_links(), U), i
        assert np.abs(plaq[:, i] - p1).max() < 1e-12, i
        assert np.abs(poly[:, i] - l1).max() < 1e-12, i
        assert L.heatbath_step == step == sweeps
        L.close()


def test_batch_graph_replay_equals_direct_launches(sunlib):
    out = []
    for graphs in (True, False):
        lats = [make(sunlib, spec) for spec in MIX[:4]]
        with sunlib.Batch(lats, use_graphs=graphs) as B:
            plaq, poly = B.run(4, 1, 3)
        out.append((plaq, poly, [L.export_links() for L in lats]))
        for L in lats:
            L.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    for a, b in zip(out[0][2], out[1][2]):
        assert np.array_equal(a, b)


def test_fp64_batch_matches_oracle(sunlib):
    specs = [(2, (4, 4, 4, 6), 2.3, 21, 4, 64), (3, (4, 6, 4, 4), 6.0, 22, 18, 64)]
    lats = [make(sunlib, s) for s in specs]
    # the oracle's own Haar starts, loaded into the chains
    starts = [orc.init(s[0], s[1], True, s[3]) for s in specs]
    for L, U in zip(lats, starts):
        L.import_links(U)
    with sunlib.Batch(lats) as B:
        plaq, _ = B.run(1, 1, 1)
    for i, (L, s) in enumerate(zip(lats, specs)):
        want = starts[i].copy()
        orc.sweep(want, s[2], 1, 1, True, s[3], 0)
        assert np.abs(L.export_links() - want).max() < 1e-10
        assert abs(plaq[0, i] - orc.plaquette(want)) < 1e-10
        L.close()


# (nc, dims, beta, seed, storage, variant): FP32 chains of every kernel kind a
# batch launches, the SU(3) one with the headline's variant (two-row staple products)
MIX32 = [
    (3, (8, 6, 4, 10), 6.0, 31, 12, 3),
    (3, (4, 6, 4, 8), 6.0, 32, 12, 0),
    (2, (8, 6, 4, 6), 2.3, 33, 4, 0),
    (4, (4, 4, 6, 4), 11.2, 34, 32, 0),
    (6, (4, 4, 4, 6), 25.2, 35, 72, 0),
]


@pytest.mark.parametrize("reunit_mode", [0, 1])
def test_fp32_batch_matches_oracle(sunlib, reunit_mode):
    """A mixed FP32 batch loaded with the oracle's thermalised configurations:
    one sweep of one overrelaxation step (no accept/reject branch) and the
    re-unitarization, every chain link by link against the oracle's sweep
    (1e-5; the batched passes, row-parallel pass, re-unitarization and
    plaquette kernels), and each chain's plaquette against the oracle's."""
    from tests.oracle_configs import cold_thermal
    specs = [sp for sp in MIX32 if reunit_mode == 0 or sp[0] <= 4]  # row-parallel SU(6): placement 0 only
    lats, starts = [], []
    for nc, dims, beta, seed, st, var in specs:
        L = sunlib.Lattice(nc, dims, beta, seed=seed, storage=st, precision=32, variant=var,
                           reunit_mode=reunit_mode)
        U = cold_thermal(nc, dims, beta)
        L.import_links(U)
        lats.append(L)
        starts.append(U)
    with sunlib.Batch(lats) as B:
        plaq, _ = B.run(1, 0, 1)
    for i, (L, sp) in enumerate(zip(lats, specs)):
        nc, dims, beta, seed = sp[:4]
        want = starts[i].copy()
        orc.sweep(want, beta, 0, 1, orc.REUNIT_FUSED if reunit_mode == 1 else True, seed, 0)
        got = L.export_links()
        assert np.abs(got - want).max() < 1e-5, (sp, float(np.abs(got - want).max()))
        assert abs(plaq[0, i] - orc.plaquette(want)) < 2e-6, sp
        L.close()


def test_batch_argument_errors(sunlib):
    a = make(sunlib, MIX[0])
    b = make(sunlib, MIX[1], reunit_mode=1)
    with pytest.raises(sunlib.SunError):
        sunlib.Batch([a, a])
    with pytest.raises(sunlib.SunError):
        sunlib.Batch([a, b])
    c = make(sunlib, MIX[2], reunit_every=2)
    with pytest.raises(sunlib.SunError):
        sunlib.Batch([c])
    for L in (a, b, c):
        L.close()


def test_large_chains_in_a_batch_run_as_alone(sunlib):
    """Chains that fill the GPU on their own (here SU(3) 24^4 and SU(6) 16^4)
    run the single-lattice kernels inside the batch; with small chains packed
    beside them every chain still evolves exactly as alone."""
    specs = [(3, (24, 24, 24, 24), 6.0, 31, 12, 32), (3, (4, 4, 4, 6), 5.8, 32, 12, 32),
             (6, (16, 16, 16, 16), 25.0, 33, 72, 32), (6, (4, 4, 4, 4), 25.0, 34, 72, 32)]
    alone = []
    for spec in specs:
        with make(sunlib, spec) as L:
            plaq, poly = L.run(2, 1, 1)
            alone.append((L.export_links(), plaq, poly))
    lats = [make(sunlib, spec) for spec in specs]
    with sunlib.Batch(lats) as B:
        plaq, poly = B.run(2, 1, 1)
    for i, L in enumerate(lats):
        U, p1, l1 = alone[i]
        assert np.array_equal(L.export_links(), U), i
        assert np.abs(plaq[:, i] - p1).max() < 1e-12, i
        assert np.abs(poly[:, i] - l1).max() < 1e-12, i
        L.close()
