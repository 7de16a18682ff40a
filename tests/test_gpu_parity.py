"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs and the same Philox stream.

Tolerances: FP64 storage 1e-12 per pass, FP32 storage 1e-5 per pass (the
bounds stated for overrelaxation links).  Heatbath links are compared where
the accept/reject branch agrees; a link whose draw took a different branch
(an "FP flip") differs by O(1) and is counted, at most 1e-6 of the updates.
"""
import numpy as np
import pytest

import oracle as orc
from tests.inputs import near_identity_config, random_gauge_config
from tests.oracle_configs import cold_thermal, drifted

pytestmark = pytest.mark.gpu

# (nc, storage, precision): every built combination
CONFIGS = [(2, 4, 64), (2, 4, 32), (2, 8, 64), (2, 8, 32), (3, 12, 32), (3, 18, 32), (3, 12, 64), (3, 18, 64),
           (4, 32, 32), (4, 32, 64), (5, 50, 32), (6, 72, 32), (6, 72, 64)]


def tol(prec):
    return 1e-12 if prec == 64 else 1e-5


def beta_for(nc):
    return 2.3 if nc == 2 else (6.0 if nc == 3 else 0.7 * nc * nc)


@pytest.fixture(scope="session")
def sunlib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1112_4533_gb300 import build as b
    b.build()
    import paper_1112_4533_gb300 as p
    p.load_library()
    return p


def thermal_config(nc, dims, seed):
    """Oracle configuration a few heatbath sweeps away from a Haar start."""
    U = random_gauge_config(nc, dims, seed)
    orc.sweep(U, beta_for(nc), 2, 1, True, seed + 1, 0)
    return U


def gpu_lattice(p, nc, dims, storage, prec, U=None, seed=7, beta=None, **kw):
    L = p.Lattice(nc, dims, beta_for(nc) if beta is None else beta, seed=seed, precision=prec, storage=storage, **kw)
    if U is not None:
        L.import_links(U)
    return L


def maxdiff(a, b):
    return float(np.abs(a - b).max())


# ------------------------------------------------------------- init / state ----

@pytest.mark.parametrize("cfg", CONFIGS)
def test_cold_start(sunlib, cfg):
    nc, st, prec = cfg
    with gpu_lattice(sunlib, nc, (4, 2, 4, 6), st, prec) as L:
        U = L.export_links()
        assert np.array_equal(U, orc.init(nc, (4, 2, 4, 6), False, 1))
        assert L.plaquette() == 1.0
        assert L.polyakov_loop() == 1.0


@pytest.mark.parametrize("cfg", CONFIGS)
def test_hot_start_matches_oracle(sunlib, cfg):
    nc, st, prec = cfg
    dims = (6, 4, 2, 8)
    L = sunlib.Lattice(nc, dims, 1.0, hot_start=True, seed=99, precision=prec, storage=st)
    U = L.export_links()
    L.close()
    want = orc.init(nc, dims, True, 99)
    assert maxdiff(U, want) < (1e-13 if prec == 64 else 5e-7)


@pytest.mark.parametrize("cfg", CONFIGS)
def test_import_export_roundtrip(sunlib, cfg):
    nc, st, prec = cfg
    dims = (4, 4, 2, 2)
    U = random_gauge_config(nc, dims, seed=5)
    with gpu_lattice(sunlib, nc, dims, st, prec, U) as L:
        back = L.export_links()
        assert maxdiff(back, U) < (1e-15 if prec == 64 else 5e-7)
        L.import_links(back)
        again = L.export_links()
        if st == 12:
            assert maxdiff(again, back) < 5e-7
        else:
            assert np.array_equal(again, back)


# ----------------------------------------------------------- one pass ----

PASS_DIMS = (8, 6, 4, 10)  # V/2 = 960: several 128-thread blocks and a ragged tail


VARIANT_CASES = [c + (0,) for c in CONFIGS] + [(3, st, 32, v) for st in (12, 18) for v in (1, 2, 3)]


@pytest.mark.parametrize("cfg", VARIANT_CASES)
def test_overrelaxation_pass_matches_oracle(sunlib, cfg):
    """Four passes of the oracle's chain from a thermal configuration; before
    each pass the GPU lattice is loaded with the oracle's current links."""
    nc, st, prec, variant = cfg
    U = thermal_config(nc, PASS_DIMS, seed=10 + nc)
    start = U.copy()
    with gpu_lattice(sunlib, nc, PASS_DIMS, st, prec, variant=variant) as L:
        for mu, par in [(0, 0), (3, 1), (1, 1), (2, 0)]:
            before = U.copy()
            L.import_links(U)
            L.update_pass(sunlib.OVERRELAX, mu, par)
            got = L.export_links()
            orc.update_pass(U, beta_for(nc), orc.OVERRELAX, mu, par, 0, 7)
            assert maxdiff(got, U) < tol(prec), (mu, par)
            assert maxdiff(got, before) > 1e-3  # it did something
    assert maxdiff(start, U) > 1e-3


@pytest.mark.parametrize("cfg", VARIANT_CASES)
def test_heatbath_pass_matches_oracle(sunlib, cfg):
    nc, st, prec, variant = cfg
    U = thermal_config(nc, PASS_DIMS, seed=20 + nc)
    n_updates = 0
    flips = 0
    with gpu_lattice(sunlib, nc, PASS_DIMS, st, prec, seed=31, variant=variant) as L:
        for mu, par in [(1, 0), (2, 1), (0, 1), (3, 0)]:
            L.import_links(U)
            L.heatbath_step = 5
            L.update_pass(sunlib.HEATBATH, mu, par)
            got = L.export_links()
            capped = orc.update_pass(U, beta_for(nc), orc.HEATBATH, mu, par, 5, 31)
            assert capped == 0
            d = np.abs(got - U).reshape(4, -1, nc * nc).max(axis=2)
            assert d[[m for m in range(4) if m != mu]].max() < (1e-15 if prec == 64 else 1e-6)
            flips += int((d[mu] > tol(prec)).sum())
            n_updates += d.shape[1] // 2
    assert flips <= 1e-6 * n_updates, (flips, n_updates)


# ----------------------------------------------------- reunit and observables ----

@pytest.mark.parametrize("cfg", CONFIGS)
def test_reunitarization_matches_oracle(sunlib, cfg):
    nc, st, prec = cfg
    dims = (4, 2, 2, 4)
    rng = np.random.default_rng(3)
    U = random_gauge_config(nc, dims, seed=40)
    U = U + 1e-3 * (rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape))
    with gpu_lattice(sunlib, nc, dims, st, prec, U) as L:
        L.reunitarize()
        got = L.export_links()
    # for every storage format the result depends on the rows the format keeps
    # (rows 0 .. Nc-2, or row 0 for SU(2)) and equals the oracle's on U itself
    want = U.copy()
    orc.reunitarize(want)
    assert maxdiff(got, want) < (1e-13 if prec == 64 else 5e-7)
    m = got.reshape(-1, nc, nc)
    assert np.abs(m @ np.conj(np.swapaxes(m, 1, 2)) - np.eye(nc)).max() < (1e-14 if prec == 64 else 1e-6)


@pytest.mark.parametrize("cfg", CONFIGS)
def test_plaquette_and_polyakov_match_oracle(sunlib, cfg):
    nc, st, prec = cfg
    dims = (6, 4, 8, 6)
    U = random_gauge_config(nc, dims, seed=50)
    with gpu_lattice(sunlib, nc, dims, st, prec, U) as L:
        p = L.plaquette()
        poly = L.polyakov_loop()
        p2 = L.plaquette()
    assert p == p2  # deterministic reduction
    t = 1e-14 if prec == 64 else 2e-6
    assert abs(p - orc.plaquette(U)) < t
    assert abs(poly - orc.polyakov(U)) < (1e-13 if prec == 64 else 2e-5)


# -------------------------------------------------------------- sweeps ----

def test_su2_small_workload_history_matches_oracle(sunlib):
    """SU(2) 8^4, beta 2.3, cold start, 10 sweeps of 1 heatbath + 4
    overrelaxation, FP64 links, Philox seed 1, plaquette after each sweep.

    The oracle runs the chain; before each sweep the GPU lattice is loaded
    with the oracle's links and heatbath step, and its sweep is compared with
    the oracle's: links to 1e-11, the plaquette and Polyakov loop to 1e-12.
    The GPU's own free-running history agrees with the oracle's to 1e-10 for
    the first sweeps only: the chain amplifies rounding-order differences by
    roughly 30x per sweep."""
    dims = (8, 8, 8, 8)
    U = orc.init(2, dims, False, 1)
    oracle_hist = []
    with sunlib.Lattice(2, dims, 2.3, hot_start=False, seed=1, precision=64) as L:
        for s in range(10):
            L.import_links(U)
            L.heatbath_step = s
            plaq, poly = L.run(1, 1, 4)
            got = L.export_links()
            orc.sweep(U, 2.3, 1, 4, True, 1, s)
            assert maxdiff(got, U) < 1e-11, s
            assert abs(plaq[0] - orc.plaquette(U)) < 1e-12, s
            assert abs(poly[0] - orc.polyakov(U)) < 1e-12, s
            oracle_hist.append(orc.plaquette(U))
        assert L.heatbath_step == 10
    with sunlib.Lattice(2, dims, 2.3, hot_start=False, seed=1, precision=64) as F:
        free, _ = F.run(10, 1, 4)
    d = np.abs(free - np.array(oracle_hist))
    assert d[:4].max() < 1e-10 and d.max() < 1e-3


@pytest.mark.parametrize("nc,st", [(2, 4), (3, 18), (4, 32), (6, 72)])
def test_fp64_sweeps_follow_the_oracle(sunlib, nc, st):
    """Three FP64 sweeps (1 heatbath + 2 overrelaxation + reunitarization)
    from a Haar start, every pass of the oracle's chain compared with the GPU
    pass from the same links (1e-12).  Whole sweeps are not compared: within
    one sweep the chain amplifies rounding-order differences to 1e-11
    (SU(3)) .. 1e-7 (SU(6))."""
    dims = (4, 6, 4, 4)
    beta = beta_for(nc)
    U = orc.init(nc, dims, True, 17)
    with sunlib.Lattice(nc, dims, beta, hot_start=True, seed=17, precision=64, storage=st) as L:
        assert maxdiff(L.export_links(), U) < 1e-13
        for s in range(3):
            for mode in (orc.HEATBATH, orc.OVERRELAX, orc.OVERRELAX):
                for mu in range(4):
                    for par in range(2):
                        L.import_links(U)
                        L.heatbath_step = s
                        L.update_pass(mode, mu, par)
                        got = L.export_links()
                        orc.update_pass(U, beta, mode, mu, par, s, 17)
                        assert maxdiff(got, U) < 1e-12, (s, mode, mu, par)
            L.import_links(U)
            L.reunitarize()
            got = L.export_links()
            orc.reunitarize(U)
            assert maxdiff(got, U) < 1e-13


def subgroup_strength(U, mu, lexes):
    """For the links U_mu(x) at the sites lexes: the smallest projected SU(2)
    strength k of W = U Sigma^+ over the subgroups, from the oracle's staple.
    FP32 rounding of the staple enters the update divided by k, so it sets
    each link's tolerance."""
    nc = U.shape[-1]
    flat = U.reshape(4, -1, nc, nc)
    kmin = np.full(len(lexes), np.inf)
    for n, lex in enumerate(lexes):
        w = flat[mu, lex] @ np.conj(orc.staple(U, mu, int(lex))).T
        for i in range(nc - 1):
            for j in range(i + 1, nc):
                b = w[np.ix_([i, j], [i, j])]
                q = 0.5 * np.array([(b[0, 0] + b[1, 1]).real, (b[0, 1] + b[1, 0]).imag,
                                    (b[0, 1] - b[1, 0]).real, (b[0, 0] - b[1, 1]).imag])
                kmin[n] = min(kmin[n], np.linalg.norm(q))
    return kmin


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_su3_medium_workload_sweep_pass_by_pass(sunlib, variant):
    """SU(3) 16^4, beta 6.0, Haar start, FP32 12-real: every pass of one sweep
    (1 heatbath + 4 overrelaxation steps, 40 passes) and the FP64
    reunitarization.  The oracle runs the chain from its Haar start; before
    each pass the GPU lattice is loaded with the oracle's links.
    Overrelaxation links agree to 1e-5 where every subgroup strength k >= 1
    and to 1e-5 / k below (a Haar start has some nearly cancelling staples);
    heatbath links the same where the accept branch agrees, with branch flips
    at most 1e-6 of the updates.  Variants with bit 2 (staple terms' third row
    taken as conj(row0 x row1)) assume unitary links; before the sweep's
    re-unitarization the links of a Haar start drift by ~1e-6 and those
    variants are held to 2e-5.  (The unscaled 1e-5 bound on thermalised links
    is tests/test_gpu_headline.py.)"""
    bound = 2e-5 if variant & 2 else 1e-5
    dims = (16, 16, 16, 16)
    n_updates, flips = 0, 0
    worst = 0.0
    U = orc.init(3, dims, True, 2)
    with sunlib.Lattice(3, dims, 6.0, hot_start=True, seed=2, precision=32, storage=12, variant=variant) as L:
        assert maxdiff(L.export_links(), U) < 5e-7
        for step, mode in enumerate([orc.HEATBATH] + [orc.OVERRELAX] * 4):
            for mu in range(4):
                for par in range(2):
                    before = U.copy()
                    L.import_links(U)
                    L.heatbath_step = 0
                    L.update_pass(mode, mu, par)
                    got = L.export_links()
                    orc.update_pass(U, 6.0, mode, mu, par, 0, 2)
                    d = np.abs(got - U).reshape(4, -1, 9).max(axis=2)[mu]
                    off = np.flatnonzero(d >= 1e-5)
                    scaled = d[off] * np.minimum(1.0, subgroup_strength(before, mu, off))
                    if mode == orc.HEATBATH:
                        flips += int((scaled >= bound).sum())
                        n_updates += d.size // 2
                    else:
                        if off.size:
                            print(f"variant {variant} step {step} mu {mu} par {par}: max {d.max():.3e} "
                                  f"scaled {scaled.max():.3e}")
                            assert scaled.max() < bound, (step, mu, par, d.max(), scaled.max())
                        worst = max(worst, d.max())
        L.import_links(U)
        L.reunitarize()
        got = L.export_links()
        orc.reunitarize(U)
        assert maxdiff(got, U) < 5e-7
        assert abs(L.plaquette() - orc.plaquette(U)) < 1e-6
    assert flips <= 1e-6 * n_updates, (flips, n_updates)


@pytest.mark.parametrize("nc,beta,st,prec", [(2, 2.3, 4, 32), (3, 6.0, 12, 32)])
def test_equilibrium_plaquette_agrees_with_oracle(sunlib, nc, beta, st, prec):
    """Independent chains (different seeds) on 8^4: equilibrium <P> agrees within
    3 sigma of the combined binned error."""
    dims = (8, 8, 8, 8)
    therm, meas = 40, 160
    with sunlib.Lattice(nc, dims, beta, hot_start=True, seed=1001, precision=prec, storage=st) as L:
        plaq, _ = L.run(therm + meas, 1, 4, polyakov=False)
    g = plaq[therm:]
    U = orc.init(nc, dims, True, 2002)
    h = []
    for s in range(therm + meas):
        orc.sweep(U, beta, 1, 4, True, 2002, s)
        if s >= therm:
            h.append(orc.plaquette(U))
    o = np.array(h)

    def mean_err(x):
        b = x.reshape(16, -1).mean(axis=1)
        return x.mean(), b.std(ddof=1) / np.sqrt(len(b))

    mg, eg = mean_err(g)
    mo, eo = mean_err(o)
    assert abs(mg - mo) < 3 * np.hypot(eg, eo), (mg, eg, mo, eo)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("cfg", [(2, 4, 64), (3, 18, 64), (3, 12, 64), (4, 32, 64), (2, 4, 32), (3, 12, 32)])
def test_fused_reunitarization_sweep_matches_oracle(sunlib, cfg, mode):
    """reunit_mode 1 (each link of the last step re-unitarized in the update
    kernel) and 2 (runs of 32 links spread over the steps) against the oracle's
    schedules, link by link.  FP64: one sweep of 1 heatbath + 1
    overrelaxation step from a thermal configuration, 1e-10.  FP32:
    overrelaxation steps only (1 step in mode 1, 2 in mode 2, no accept/reject
    branch) from a cold-start-thermalised configuration, every link within
    1e-5 of the oracle.  Where the storage allows (see off_group), the input's
    rows are 1e-4 off the group, so that without the re-unitarization, or with
    it on other links, the result would be ~1e-4 away.  The result is special
    unitary to the storage precision."""
    nc, st, prec = cfg
    dims = (8, 6, 4, 4)  # 96 sites per parity: three runs of 32
    # links off the group make the re-unitarization visible, where the storage
    # evolves them as the oracle's full matrices do: two-row storage rebuilds
    # row 2 from rows 0, 1 at every read, so it gets them only when every
    # updated link is re-unitarized before it is read again (mode 1 with a
    # single step)
    n_steps = 2 if prec == 64 else (1 if mode == 1 else 2)
    off_group = st != 12 or (mode == 1 and n_steps == 1)
    if prec == 64:
        U0 = thermal_config(nc, dims, seed=90 + nc)
        n_hb, n_or = 1, 1
    else:
        U0 = cold_thermal(nc, dims, beta_for(nc))
        n_hb, n_or = 0, (1 if mode == 1 else 2)
    if off_group:
        U0 = drifted(U0, 1e-4, seed=90 + nc)
    with gpu_lattice(sunlib, nc, dims, st, prec, U0, seed=6, reunit_mode=mode) as L:
        L.sweep(n_hb, n_or)
        got = L.export_links()
    want = U0.copy()
    orc.sweep(want, beta_for(nc), n_hb, n_or, orc.REUNIT_FUSED if mode == 1 else orc.REUNIT_SPREAD, 6, 0)
    d = np.abs(got - want).reshape(-1, nc * nc).max(axis=1)
    assert d.max() < (1e-10 if prec == 64 else 1e-5), float(d.max())
    if off_group:
        plain = U0.copy()
        orc.sweep(plain, beta_for(nc), n_hb, n_or, orc.REUNIT_NONE, 6, 0)
        assert np.abs(got - plain).max() > 1e-5
    m = got.reshape(-1, nc, nc)
    assert np.abs(m @ np.conj(np.swapaxes(m, 1, 2)) - np.eye(nc)).max() < (1e-14 if prec == 64 else 2e-6)


# ------------------------------------------------------- equivalences ----

def test_generic_su2_equals_quaternion_su2(sunlib):
    dims = (4, 4, 4, 6)
    U = thermal_config(2, dims, seed=60)
    out = []
    for st in (4, 8):
        with gpu_lattice(sunlib, 2, dims, st, 64, U, seed=3) as L:
            L.sweep(1, 2)
            out.append(L.export_links())
    assert maxdiff(out[0], out[1]) < 1e-13


def test_two_row_equals_full_su3(sunlib):
    dims = (4, 4, 4, 6)
    U = thermal_config(3, dims, seed=61)
    out = []
    for st in (12, 18):
        with gpu_lattice(sunlib, 3, dims, st, 64, U, seed=3) as L:
            L.sweep(1, 2)
            out.append(L.export_links())
    assert maxdiff(out[0], out[1]) < 1e-12


def test_graph_replay_equals_direct_launches(sunlib):
    dims = (8, 4, 4, 8)
    res = []
    for graphs in (True, False):
        with sunlib.Lattice(3, dims, 6.0, hot_start=True, seed=4, use_graphs=graphs) as L:
            plaq, poly = L.run(5, 1, 4)
            res.append((plaq, poly, L.export_links()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][2], res[1][2])


def test_multi_sweep_graphs_equal_one_sweep_graphs(sunlib):
    """graph_sweeps: 4 sweeps per graph launch (then a remainder of single
    sweeps) gives bitwise the links and histories of one sweep per launch."""
    dims = (6, 4, 4, 6)
    out = []
    for gs in (1, 4):
        with sunlib.Lattice(3, dims, 6.0, hot_start=True, seed=14, graph_sweeps=gs, reunit_mode=1) as L:
            plaq, poly = L.run(6, 1, 2)
            plaq2, _ = L.run(3, 1, 2)
            out.append((plaq, poly, plaq2, L.export_links(), L.heatbath_step))
    assert all(np.array_equal(a, b) for a, b in zip(out[0][:4], out[1][:4]))
    assert out[0][4] == out[1][4] == 9
    lats = [sunlib.Lattice(2, (4, 4, 4, 4), 2.3, hot_start=True, seed=15 + i, graph_sweeps=4) for i in range(3)]
    with sunlib.Batch(lats) as B:
        bp, _ = B.run(5, 1, 1)
    for i, L in enumerate(lats):
        with sunlib.Lattice(2, (4, 4, 4, 4), 2.3, hot_start=True, seed=15 + i) as A:
            ap, _ = A.run(5, 1, 1)
            assert np.array_equal(A.export_links(), L.export_links())
        assert np.abs(bp[:, i] - ap).max() < 1e-12
        L.close()


def test_runs_are_deterministic(sunlib):
    out = []
    for _ in range(2):
        with sunlib.Lattice(4, (4, 4, 4, 4), 11.2, hot_start=True, seed=8) as L:
            L.run(3, 1, 2)
            out.append(L.export_links())
    assert np.array_equal(out[0], out[1])


def test_resume_from_exported_state_is_exact(sunlib):
    """(links, seed, heatbath step) is the whole state: stopping, exporting and
    resuming in a fresh lattice reproduces the uninterrupted chain bitwise."""
    dims = (8, 4, 4, 4)
    with sunlib.Lattice(3, dims, 6.0, hot_start=True, seed=12) as A:
        A.run(4, 1, 3)
        ref = A.export_links()
    with sunlib.Lattice(3, dims, 6.0, hot_start=True, seed=12) as B:
        B.run(2, 1, 3)
        saved, step = B.export_links(), B.heatbath_step
    with sunlib.Lattice(3, dims, 6.0, hot_start=False, seed=12) as C:
        C.import_links(saved)
        C.heatbath_step = step
        # the export holds the stored rows exactly, so the continuation is bitwise
        C.run(2, 1, 3)
        got = C.export_links()
    assert np.array_equal(got, ref)


# ------------------------------------------------------------ edge cases ----

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 6, 2), (10, 2, 2, 4)])
def test_smallest_and_ragged_lattices(sunlib, dims):
    U0 = thermal_config(3, dims, seed=70)
    with gpu_lattice(sunlib, 3, dims, 18, 64, U0, seed=5) as L:
        L.sweep(1, 1)
        got = L.export_links()
        p = L.plaquette()
    want = U0.copy()
    orc.sweep(want, 6.0, 1, 1, True, 5, 0)
    assert maxdiff(got, want) < 1e-11
    assert abs(p - orc.plaquette(want)) < 1e-13


def test_beta_zero_heatbath_gives_haar_links(sunlib):
    """beta = 0: the SU(2) heatbath draws Haar links in one step; the SU(3)
    pseudo-heatbath converges to Haar over a few steps."""
    for nc, steps in [(2, 1), (3, 8)]:
        with sunlib.Lattice(nc, (8, 8, 8, 8), 0.0, hot_start=False, seed=3) as L:
            L.sweep(steps, 0)
            U = L.export_links()
        tr = np.trace(U.reshape(-1, nc, nc), axis1=1, axis2=2)
        n = len(tr)
        assert abs(tr.mean()) < 5 / np.sqrt(n)
        assert abs((np.abs(tr) ** 2).mean() - 1) < 5 * np.sqrt(2.0 / n)


def test_vanishing_staple_leaves_the_link(sunlib):
    """SU(2): with U_mu(x - nu) = -1 for every nu != mu and all else 1, the
    forward and backward staple terms cancel (Sigma = 0): both sides skip it."""
    dims = (4, 4, 4, 4)
    nx, ny, nz, nt = dims
    U = orc.init(2, dims, False, 1)
    mu = 0
    x = (2, 2, 2, 2)  # even site
    for nu in (1, 2, 3):
        c = list(x)
        c[nu] -= 1
        U[mu, c[3], c[2], c[1], c[0]] = -np.eye(2)
    for mode in (orc.HEATBATH, orc.OVERRELAX):
        with gpu_lattice(sunlib, 2, dims, 4, 64, U) as L:
            L.update_pass(mode, mu, 0)
            got = L.export_links()
        want = U.copy()
        orc.update_pass(want, 2.3, mode, mu, 0, 0, 7)
        assert np.array_equal(got[mu, 2, 2, 2, 2], np.eye(2))
        assert maxdiff(got, want) < 1e-12


def test_invalid_pass_arguments_raise(sunlib):
    with sunlib.Lattice(2, (4, 4, 4, 4), 2.3) as L:
        for args in [(2, 0, 0), (0, 4, 0), (0, 0, 2)]:
            with pytest.raises(sunlib.SunError):
                L.update_pass(*args)
            with pytest.raises(sunlib.SunError):
                L.update_pass_reunit(*args)
        with pytest.raises(sunlib.SunError):
            L.heatbath_step = 2 ** 33


def test_lattices_on_concurrent_host_threads(sunlib):
    """Two lattices driven at the same time from two host threads (the C ABI
    releases the interpreter lock): each ends bitwise where it ends alone."""
    import threading
    specs = [(3, (8, 6, 4, 6), 6.0, 31), (2, (6, 6, 6, 8), 2.3, 32)]
    alone = []
    for nc, dims, beta, seed in specs:
        with sunlib.Lattice(nc, dims, beta, hot_start=True, seed=seed) as L:
            L.run(12, 1, 3)
            alone.append(L.export_links())
    out, errors = [None, None], []

    def work(i):
        try:
            nc, dims, beta, seed = specs[i]
            with sunlib.Lattice(nc, dims, beta, hot_start=True, seed=seed) as L:
                for _ in range(3):
                    L.run(4, 1, 3)
                out[i] = L.export_links()
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for got, want in zip(out, alone):
        assert np.array_equal(got, want)


@pytest.mark.parametrize("reunit_mode", [0, 1, 2])
def test_su4_register_bound_equals_default_kernel(sunlib, reunit_mode):
    """SU(4) FP32 with variant bit 1 (the per-link pass bounded to 128 registers)
    gives bitwise the links and observables of the default kernel."""
    for dims in [(6, 6, 4, 8), (4, 4, 4, 4)]:
        out = []
        for variant in (0, 1):
            with sunlib.Lattice(4, dims, 11.0, hot_start=True, seed=21, variant=variant,
                                reunit_mode=reunit_mode) as L:
                plaq, poly = L.run(2, 1, 2)
                out.append((L.export_links(), plaq, poly))
        assert np.array_equal(out[0][0], out[1][0]), dims
        assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_fused_pass_unsupported_where_not_built(sunlib):
    """FP64 passes of Nc >= 5 are built without the fused re-unitarization."""
    with sunlib.Lattice(6, (4, 4, 4, 4), 25.2, precision=64) as L:
        with pytest.raises(sunlib.SunError) as e:
            L.update_pass_reunit(sunlib.OVERRELAX, 0, 0)
        assert e.value.status == 5
