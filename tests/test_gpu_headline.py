"""GPU parity of the kernels the headline sweep launches (SU(3), FP32 two-row
storage, FP64 re-unitarization fused into the update kernels), link by link
against the FP64 oracle.

Inputs are the oracle's own thermalised configurations (tests/oracle_configs.py),
imported into the GPU lattice; the oracle never reads a GPU result.  Bounds:
every link of an overrelaxation pass within 1e-5 of the oracle (no scaling by
the subgroup strength: cold-start-thermalised inputs have k >= 1); heatbath
links within 1e-5 wherever the accept/reject branch agrees, no link in the
band between agreement and a branch flip (1e-3), and flips at most 1e-6 of
the updates (Eqs. 12-17, and the re-unitarization at the end of Sec. 2, in
the placements the oracle mirrors).

Inputs whose rows are 1e-4 off the group make a re-unitarization visible (it
moves such a link by ~1e-4).  Two-row storage keeps rows 0 and 1 and takes
row 2 as conj(row0 x row1) whenever it reads a link; for links off the group
that is not the row 2 the full-matrix oracle carries through an update.  So
off-group inputs are used only where every updated link is re-unitarized
before anything reads it (the fused pass, reunit_mode 1) or where the storage
holds the whole matrix (full SU(3) storage, SU(2) quaternions); elsewhere the
inputs are on the group.
"""
import numpy as np
import pytest

import oracle as orc
from tests.oracle_configs import cold_thermal, drifted, min_subgroup_strength, tiled

pytestmark = pytest.mark.gpu

OR_TOL = 1e-5
FLIP = 1e-3       # a link further than this from the oracle took another heatbath branch
FLIP_RATE = 1e-6  # flips allowed per link update


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


def link_diff(got, want):
    nc = got.shape[-1]
    return np.abs(got - want).reshape(-1, nc * nc).max(axis=1)


def check_heatbath(d, n_updates, what, agree=OR_TOL):
    gray = int(((d > agree) & (d < FLIP)).sum())
    flips = int((d >= FLIP).sum())
    assert gray == 0, (what, "links between agreement and a branch flip", gray, float(d[d < FLIP].max()))
    assert flips <= FLIP_RATE * n_updates, (what, flips, n_updates)
    return flips


def unitarity(U):
    nc = U.shape[-1]
    m = U.reshape(-1, nc, nc)
    return float(np.abs(m @ np.conj(np.swapaxes(m, 1, 2)) - np.eye(nc)).max())


SMALL, MEDIUM = (8, 6, 4, 10), (16, 16, 16, 16)
PASSES = [(0, 0), (3, 1), (1, 1), (2, 0)]


def test_thermal_inputs_have_strong_subgroups():
    """The premise of the unscaled bound, on the small input: every subgroup
    strength k >= 1 (oracle only)."""
    U = cold_thermal(3, SMALL, 6.0)
    assert min(min_subgroup_strength(U, mu, par) for mu in range(4) for par in range(2)) >= 1.0


# (nc, storage, variant, dims): the headline's two-row SU(3) kernels (variant 1
# = the register-bounded kernel the benchmark runs, 16 = packed overrelaxation),
# full SU(3) storage, SU(2) quaternions, SU(4)
FUSED_PASS_CASES = [(3, 12, 0, SMALL), (3, 12, 1, SMALL), (3, 12, 1, MEDIUM), (3, 12, 16, SMALL), (3, 18, 1, SMALL),
                    (2, 4, 0, SMALL), (4, 32, 0, SMALL), (4, 32, 1, SMALL)]


@pytest.mark.parametrize("nc,st,variant,dims", FUSED_PASS_CASES)
@pytest.mark.parametrize("mode", [orc.OVERRELAX, orc.HEATBATH])
def test_fused_reunitarization_pass_is_elementwise(sunlib, nc, st, variant, dims, mode):
    """FP32 passes with the FP64 re-unitarization fused into the update kernel
    (the kernels a re-unitarizing step launches), each from the oracle's links,
    1e-4 off the group: every updated link re-unitarized right after its
    update, against the oracle's pass with the same placement."""
    beta = beta_for(nc)
    U = drifted(cold_thermal(nc, dims, beta), 1e-4, seed=3)
    n_updates, flips = 0, 0
    with sunlib.Lattice(nc, dims, beta, seed=6, precision=32, storage=st, variant=variant) as L:
        for mu, par in PASSES:
            before = U.copy()
            L.import_links(U)
            L.heatbath_step = 4
            L.update_pass_reunit(mode, mu, par)
            got = L.export_links()
            orc.update_pass(U, beta, mode, mu, par, 4, 6, reunit_after=True)
            d = link_diff(got, U)
            if mode == orc.OVERRELAX:
                assert d.max() < OR_TOL, (mu, par, float(d.max()))
            else:
                n_updates += d.size // 8
                flips += check_heatbath(d, n_updates, (mu, par))
            # the re-unitarization is visible: without it the oracle lands ~1e-4 away
            orc.update_pass(before, beta, mode, mu, par, 4, 6)
            assert link_diff(got, before).max() > 1e-5


@pytest.mark.parametrize("dims", [SMALL, MEDIUM])
@pytest.mark.parametrize("mode", [orc.OVERRELAX, orc.HEATBATH])
def test_two_row_staple_fused_pass(sunlib, dims, mode):
    """Variant 3 (register bound + two-row staple products, the headline's
    kernels): the fused pass link by link on links on the group, where the
    conj(row0 x row1) third row of each staple term is exact (1e-5); and on
    links 1e-4 off the group, every updated link ends on the group."""
    U = cold_thermal(3, dims, 6.0)
    V = drifted(U, 1e-4, seed=3)
    n_updates, flips = 0, 0
    with sunlib.Lattice(3, dims, 6.0, seed=6, precision=32, storage=12, variant=3) as L:
        for mu, par in PASSES:
            L.import_links(U)
            L.heatbath_step = 4
            L.update_pass_reunit(mode, mu, par)
            got = L.export_links()
            orc.update_pass(U, 6.0, mode, mu, par, 4, 6, reunit_after=True)
            d = link_diff(got, U)
            if mode == orc.OVERRELAX:
                assert d.max() < OR_TOL, (mu, par, float(d.max()))
            else:
                n_updates += d.size // 8
                flips += check_heatbath(d, n_updates, (mu, par))
            L.import_links(V)
            L.update_pass_reunit(mode, mu, par)
            moved = L.export_links().reshape(4, -1, 3, 3)
            m = moved[mu].reshape(dims[3], dims[2], dims[1], dims[0], 3, 3)
            t, z, y, x = np.meshgrid(*[np.arange(n) for n in (dims[3], dims[2], dims[1], dims[0])], indexing="ij")
            updated = m[(x + y + z + t) % 2 == par]
            assert unitarity(updated) < 2e-6
            assert unitarity(V.reshape(4, -1, 3, 3)[mu]) > 1e-5


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("dims", [SMALL, MEDIUM])
def test_fused_step_reunitarizes_every_link(sunlib, dims, variant):
    """reunit_mode 1: one overrelaxation step (eight passes, each link
    re-unitarized right after its update) from links 1e-4 off the group, every
    link within 1e-5 of the oracle's step with the same placement; the result
    is on the group to FP32 rounding."""
    U0 = drifted(cold_thermal(3, dims, 6.0), 1e-4, seed=3)
    with sunlib.Lattice(3, dims, 6.0, seed=6, precision=32, storage=12, variant=variant, reunit_mode=1) as L:
        L.import_links(U0)
        L.sweep(0, 1)
        got = L.export_links()
    want = U0.copy()
    orc.sweep(want, 6.0, 0, 1, orc.REUNIT_FUSED, 6, 0)
    d = link_diff(got, want)
    assert d.max() < OR_TOL, (dims, variant, float(d.max()))
    assert unitarity(got) < 2e-6
    plain = U0.copy()
    orc.sweep(plain, 6.0, 0, 1, orc.REUNIT_NONE, 6, 0)
    assert link_diff(got, plain).max() > 1e-5


@pytest.mark.parametrize("mode,n_hb,n_or", [(1, 1, 0), (2, 1, 1), (2, 0, 2)])
@pytest.mark.parametrize("dims,trials", [(SMALL, 2), (MEDIUM, 4)])
def test_reunitarizing_sweeps_follow_the_oracle(sunlib, dims, trials, mode, n_hb, n_or):
    """Whole re-unitarizing sweeps of the two-row FP32 chain with the fused
    placements (mode 1: every link of the last step; mode 2: runs of 32 links
    spread over the steps), from the oracle's thermalised links (on the group),
    for several heatbath step counters.  The sweep chains eight passes per step,
    each reading links the earlier passes wrote, so a link carries the earlier
    passes' rounding too: a single overrelaxation step within 1e-5 (as one
    pass), longer chains and steps with a heatbath within 2e-5 where the
    branches agree (measured: 1.1e-5 after two overrelaxation steps)."""
    U0 = cold_thermal(3, dims, 6.0)
    agree = OR_TOL if (n_hb, n_or) == (0, 1) else 2e-5
    n_updates, flips = 0, 0
    with sunlib.Lattice(3, dims, 6.0, seed=8, precision=32, storage=12, variant=1, reunit_mode=mode) as L:
        for s in range(trials if n_hb else 1):
            L.import_links(U0)
            L.heatbath_step = 10 + s
            L.sweep(n_hb, n_or)
            got = L.export_links()
            want = U0.copy()
            orc.sweep(want, 6.0, n_hb, n_or, orc.REUNIT_FUSED if mode == 1 else orc.REUNIT_SPREAD, 8, 10 + s)
            n_updates += (n_hb + n_or) * got.size // 9
            flips += check_heatbath(link_diff(got, want), n_updates, (dims, mode, s), agree)
            assert unitarity(got) < 2e-6
    assert flips <= FLIP_RATE * n_updates


@pytest.mark.parametrize("nc,st,prec", [(3, 18, 64), (2, 4, 64), (2, 4, 32)])
@pytest.mark.parametrize("n_hb,n_or", [(1, 1), (0, 2), (2, 1)])
def test_spread_schedule_picks_the_oracles_links(sunlib, nc, st, prec, n_hb, n_or):
    """reunit_mode 2 from links 1e-4 off the group, in storage that holds the
    whole matrix (full SU(3), SU(2) quaternions), where re-unitarizing a run of
    links in another step than the oracle moves them by ~1e-4: FP64 within
    1e-10, FP32 within 1e-5 (overrelaxation only) of the oracle's spread
    schedule."""
    beta = beta_for(nc)
    dims = (8, 6, 4, 4)  # 96 half-sites per parity: three runs of 32
    if prec == 32 and n_hb:
        pytest.skip("FP32 heatbath sweeps: tests above")
    U0 = drifted(cold_thermal(nc, dims, beta), 1e-4, seed=9)
    with sunlib.Lattice(nc, dims, beta, seed=5, precision=prec, storage=st, reunit_mode=2) as L:
        L.import_links(U0)
        L.sweep(n_hb, n_or)
        got = L.export_links()
    want = U0.copy()
    orc.sweep(want, beta, n_hb, n_or, orc.REUNIT_SPREAD, 5, 0)
    assert link_diff(got, want).max() < (1e-10 if prec == 64 else OR_TOL)
    # another schedule is far away
    other = U0.copy()
    orc.sweep(other, beta, n_hb, n_or, orc.REUNIT_FUSED, 5, 0)
    assert link_diff(got, other).max() > 1e-6


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_thermal_medium_lattice_every_pass_unscaled(sunlib, variant):
    """SU(3) 16^4, beta 6.0, FP32 two-row: every pass of one sweep of 1 heatbath
    + 4 overrelaxation steps and the re-unitarization.  The oracle runs its own
    chain from a cold-start-thermalised configuration; before each pass the GPU
    lattice is loaded with the oracle's current links.  Overrelaxation links
    within 1e-5 without scaling by k; variant bit 2 (two-row staple products)
    included, as its accuracy holds on re-unitarized links."""
    dims = MEDIUM
    U = cold_thermal(3, dims, 6.0)
    n_updates, flips, worst = 0, 0, 0.0
    with sunlib.Lattice(3, dims, 6.0, seed=2, precision=32, storage=12, variant=variant) as L:
        for step, mode in enumerate([orc.HEATBATH] + [orc.OVERRELAX] * 4):
            for mu in range(4):
                for par in range(2):
                    L.import_links(U)
                    L.heatbath_step = 0
                    L.update_pass(mode, mu, par)
                    got = L.export_links()
                    orc.update_pass(U, 6.0, mode, mu, par, 0, 2)
                    d = link_diff(got, U)
                    if mode == orc.HEATBATH:
                        n_updates += d.size // 8
                        flips += check_heatbath(d, n_updates, (step, mu, par))
                    else:
                        assert d.max() < OR_TOL, (variant, step, mu, par, float(d.max()))
                        worst = max(worst, float(d.max()))
        L.import_links(U)
        L.reunitarize()
        got = L.export_links()
        orc.reunitarize(U)
        assert link_diff(got, U).max() < 5e-7
        assert abs(L.plaquette() - orc.plaquette(U)) < 1e-6
    assert flips <= FLIP_RATE * n_updates
    print(f"variant {variant}: worst overrelaxation link {worst:.2e}, {flips} flips in {n_updates} updates")


# ---------------------------------------------------------------- full size ----

FULL = (48, 48, 48, 96)
TILE = (16, 16, 16, 32)
REPS = (3, 3, 3, 3)


def test_full_size_headline_configuration(sunlib):
    """SU(3) 48^3x96, beta 6.2, FP32: the configuration the library's autotuner
    picks for the benchmark's sweep (1 heatbath + 5 overrelaxation steps), and
    every kind of update kernel that sweep launches, on the whole lattice
    against the oracle, each from the oracle's links: one heatbath pass, one
    overrelaxation pass, and the re-unitarizing step (the sweep's last step,
    with the tuned placement; its input 1e-4 off the group where that
    placement re-unitarizes every link of the step); then the plaquette and
    the Polyakov loop.  The input is the oracle's thermalised 16^3x32 (beta
    6.2, cold start, six sweeps) tiled 3 x 3 x 3 x 3."""
    beta, seed = 6.2, 1
    tuned = sunlib.autotune(3, FULL, beta, 1, 5, precision=32, storage=12, reunit_mode=1, tune_storage=True,
                            tune_reunit_mode=True, two_row=True)
    kw = dict(precision=32, storage=tuned["storage"], variant=tuned["variant"], reunit_mode=tuned["reunit_mode"],
              block_threads=tuned["block_threads"], graph_sweeps=tuned["graph_sweeps"])
    small = cold_thermal(3, TILE, beta)
    U = tiled(small, REPS)
    n_pass = U.size // 9 // 8  # links of one (direction, parity) pass
    with sunlib.Lattice(3, FULL, beta, seed=seed, **kw) as L:
        L.import_links(U)
        assert abs(L.plaquette() - orc.plaquette(U)) < 2e-6
        assert abs(L.polyakov_loop() - orc.polyakov(U)) < 2e-5
        # heatbath pass (direction 1, even sites), heatbath step 3
        L.heatbath_step = 3
        L.update_pass(sunlib.HEATBATH, 1, 0)
        got = L.export_links()
        want = U.copy()
        orc.update_pass(want, beta, orc.HEATBATH, 1, 0, 3, seed)
        check_heatbath(link_diff(got, want), n_pass, "heatbath pass")
        del got, want
        # overrelaxation pass (direction 2, odd sites)
        L.import_links(U)
        L.update_pass(sunlib.OVERRELAX, 2, 1)
        got = L.export_links()
        want = U.copy()
        orc.update_pass(want, beta, orc.OVERRELAX, 2, 1, 3, seed)
        d = link_diff(got, want)
        assert d.max() < OR_TOL, float(d.max())
        del got, want, U
        # the re-unitarizing step: one overrelaxation step with the tuned placement;
        # links off the group only where every link is re-unitarized before it is
        # read and the staple products use all three rows of each term (with
        # variant bit 2 a term's third row is conj(row0 x row1), exact on the group)
        mode = kw["reunit_mode"]
        two_row_staple = (kw["variant"] & 2) != 0
        off_group = mode == 1 and not two_row_staple
        V = tiled(drifted(small, 1e-4, seed=5) if off_group else small, REPS)
        L.import_links(V)
        L.sweep(0, 1)
        got = L.export_links()
        orc.sweep(V, beta, 0, 1, {0: orc.REUNIT_AFTER, 1: orc.REUNIT_FUSED, 2: orc.REUNIT_SPREAD}[mode], seed, 3)
        d = link_diff(got, V)
        assert d.max() < OR_TOL, float(d.max())
        assert unitarity(got) < 2e-6
        del got
        # observables of the GPU's result against the oracle's on its own links
        assert abs(L.plaquette() - orc.plaquette(V)) < 2e-6
        assert abs(L.polyakov_loop() - orc.polyakov(V)) < 2e-5
        del V
        if mode == 1 and not off_group:
            # every link of the step is re-unitarized: from links 1e-4 off the
            # group the step ends on the group
            L.import_links(tiled(drifted(small, 1e-4, seed=5), REPS))
            L.sweep(0, 1)
            assert unitarity(L.export_links()) < 2e-6
