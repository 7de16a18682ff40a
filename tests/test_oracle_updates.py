"""Pins of the oracle's link updates: overrelaxation invariants, the SU(2)
heatbath distribution of Eq. 13, the Cabibbo-Marinari single-link equilibrium
(Bessel-determinant closed form of the SU(Nc) one-link integral), the strong-
and weak-coupling limits of the plaquette, and the independence of a
checkerboard pass from the order of its links and the thread count.
"""
import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle as orc
from tests.inputs import random_gauge_config, random_su_n


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def action(U, beta):
    """Wilson action, Eq. 3: (beta/Nc) sum_x sum_{mu<nu} ReTr(1 - P)."""
    V = U.shape[1] * U.shape[2] * U.shape[3] * U.shape[4]
    return beta * 6 * V * (1.0 - orc.plaquette(U))


# ------------------------------------------------------------ overrelaxation ----

@pytest.mark.parametrize("nc", [2, 3, 4])
def test_overrelaxation_conserves_the_action(nc):
    """Eq. 17 leaves ReTr(U Sigma^+) unchanged for each link and each subgroup,
    and no link of a pass is in another's staple, so a whole OR step (8 passes,
    no reunitarization) conserves the action to rounding (1e-10 relative)."""
    beta = 2.3 if nc == 2 else 0.7 * nc * nc
    U = random_gauge_config(nc, (4, 4, 2, 4), seed=100 + nc)
    orc.sweep(U, beta, 1, 0, False, seed=5, hb_step0=0)  # leave the Haar start
    s0 = action(U, beta)
    orc.sweep(U, beta, 0, 1, False, seed=5, hb_step0=0)
    s1 = action(U, beta)
    assert abs(s1 - s0) / abs(s0) < 1e-10
    # and it is not the identity
    U2 = U.copy()
    orc.sweep(U2, beta, 0, 1, False, seed=5, hb_step0=0)
    assert np.abs(U2 - U).max() > 1e-2


def test_su2_overrelaxation_is_an_involution():
    """For SU(2) the reflection U -> (Sigma/k) U^+ (Sigma/k) squares to one."""
    rng = np.random.default_rng(7)
    for _ in range(10):
        U = random_su_n(2, rng, 1)[0]
        S = sum(random_su_n(2, rng, 6))
        U1, _ = orc.update_link(U, S, 2.0, orc.OVERRELAX, 1, 0, 0)
        U2, _ = orc.update_link(U1, S, 2.0, orc.OVERRELAX, 1, 0, 0)
        assert np.abs(U1 - U).max() > 1e-3
        assert np.abs(U2 - U).max() < 1e-13
        # and it equals the closed form of Eq. 17 in the orientation exp(ReTr U Sigma^+)
        k = np.sqrt(np.linalg.det(S).real)
        assert np.abs(U1 - (S / k) @ dag(U) @ (S / k)).max() < 1e-13


def test_su2_overrelaxation_is_gauge_covariant():
    """For Nc = 2, W = U Sigma^+ goes to G(x) W G(x)^+ under a gauge transform,
    so its normalised projection and (vhat^+)^2 do too, and the overrelaxed
    link of the transformed field is the transform of the overrelaxed link:
    OR(U^G) = OR(U)^G exactly, up to rounding, for every pass.  (The heatbath
    is covariant only in distribution: its draw b is taken in a fixed frame.)"""
    from tests.inputs import random_site_field
    dims = (4, 4, 2, 6)
    U = random_gauge_config(2, dims, seed=77)
    G = random_site_field(2, dims, seed=78)

    def transform(V):
        out = np.empty_like(V)
        for mu in range(4):
            Gp = np.roll(G, -1, axis=3 - mu)  # x+mu: axes of G are (t, z, y, x)
            out[mu] = G @ V[mu] @ dag(Gp)
        return out

    A, B = U.copy(), transform(U)
    assert np.abs(B - U).max() > 0.1
    for mu in range(4):
        for par in (0, 1):
            orc.update_pass(A, 2.3, orc.OVERRELAX, mu, par, 0, 5)
            orc.update_pass(B, 2.3, orc.OVERRELAX, mu, par, 0, 5)
    assert np.abs(transform(A) - B).max() < 1e-12


@pytest.mark.parametrize("nc", [3, 4])
def test_sun_overrelaxation_keeps_retr_u_sigma(nc):
    rng = np.random.default_rng(8 + nc)
    U = random_su_n(nc, rng, 1)[0]
    S = sum(random_su_n(nc, rng, 6))
    U1, _ = orc.update_link(U, S, 6.0, orc.OVERRELAX, 1, 0, 0)
    assert abs(np.trace(U1 @ dag(S)).real - np.trace(U @ dag(S)).real) < 1e-12
    assert np.abs(U1 @ dag(U1) - np.eye(nc)).max() < 1e-13


# --------------------------------------------------------------- heatbath ----

def _b0_cdf(alpha):
    """CDF of the density sqrt(1-b^2) exp(alpha b) on [-1, 1] (Eq. 13), tabulated."""
    x = np.linspace(-1.0, 1.0, 200001)
    f = np.sqrt(np.clip(1 - x * x, 0, None)) * np.exp(alpha * (x - 1))
    c = integrate.cumulative_trapezoid(f, x, initial=0.0)
    c /= c[-1]
    return lambda q: np.interp(q, x, c)


@pytest.mark.parametrize("alpha", [0.0, 0.2, 1.0, 1.49, 1.5, 4.0, 12.0])
def test_su2_heatbath_element_distribution(alpha):
    """b0 follows sqrt(1-b0^2) e^{alpha b0} (KS test, both samplers, each side
    of the switch) with mean I_2(alpha)/I_1(alpha); the vector part is
    isotropic on the sphere of radius sqrt(1-b0^2)."""
    n = 40000
    b = np.empty((n, 4))
    for i in range(n):
        b[i], used = orc.su2_heatbath(alpha, 11, i, 3, 0)
        assert used >= 1
    assert np.abs((b ** 2).sum(axis=1) - 1).max() < 1e-13
    ks = stats.kstest(b[:, 0], _b0_cdf(alpha))
    assert ks.pvalue > 1e-3
    mean = special.iv(2, alpha) / special.iv(1, alpha) if alpha > 0 else 0.0
    assert abs(b[:, 0].mean() - mean) < 5 * b[:, 0].std() / np.sqrt(n)
    vec = b[:, 1:] / np.linalg.norm(b[:, 1:], axis=1, keepdims=True)
    assert np.abs(vec.mean(axis=0)).max() < 5 / np.sqrt(3 * n)
    assert np.abs(vec.T @ vec / n - np.eye(3) / 3).max() < 5 * 0.3 / np.sqrt(n)


def test_su2_heatbath_is_independent_of_old_link_and_uses_the_staple():
    """For SU(2) the heatbath result b Sigma/k does not depend on the old link
    (Eq. 14), and ReTr(U' Sigma^+)/(2k) is the drawn b0."""
    rng = np.random.default_rng(12)
    S = sum(random_su_n(2, rng, 6))
    k = np.sqrt(np.linalg.det(S).real)
    beta = 2.3
    Ua, Ub = random_su_n(2, rng, 2)
    na, _ = orc.update_link(Ua, S, beta, orc.HEATBATH, 9, 77, 4)
    nb, _ = orc.update_link(Ub, S, beta, orc.HEATBATH, 9, 77, 4)
    assert np.abs(na - nb).max() < 1e-13
    b, _ = orc.su2_heatbath(beta * k, 9, 77, 4, 0)
    assert abs(np.trace(na @ dag(S)).real / (2 * k) - b[0]) < 1e-13


def _sun_onelink_mean_retr(nc, c):
    """<ReTr V> under exp(c ReTr V) dV on SU(nc): d ln Z / dc with
    Z(c) = sum_q det[I_{q+i-j}(c)] (Toeplitz/Bessel form of the one-link integral)."""
    def Z(cc):
        tot = 0.0
        for q in range(-30, 31):
            m = np.array([[special.iv(q + i - j, cc) for j in range(nc)] for i in range(nc)])
            tot += np.linalg.det(m)
        return tot
    h = 1e-4 * max(c, 1.0)
    return (np.log(Z(c + h)) - np.log(Z(c - h))) / (2 * h)


def test_one_link_integral_formula_reduces_to_su2_closed_form():
    # SU(2): Z(c) = I_1(2c)/c, so <ReTr V> = 2 I_2(2c)/I_1(2c)
    for c in [0.3, 1.0, 2.5]:
        assert abs(_sun_onelink_mean_retr(2, c) - 2 * special.iv(2, 2 * c) / special.iv(1, 2 * c)) < 1e-7


@pytest.mark.parametrize("nc,beta,s", [(2, 2.0, 1.3), (3, 6.0, 0.9), (4, 11.0, 0.8)])
def test_cabibbo_marinari_single_link_equilibrium(nc, beta, s):
    """Repeated pseudo-heatbath updates of one link with a fixed staple
    Sigma = s G^+ sample exp((beta/nc) ReTr(U Sigma^+)) dU, so V = U G has
    <ReTr V> = d ln Z/dc at c = beta s / nc (closed form above)."""
    rng = np.random.default_rng(200 + nc)
    G = random_su_n(nc, rng, 1)[0]
    S = s * dag(G)
    U = np.eye(nc, dtype=np.complex128)
    n, burn = 30000, 200
    vals = np.empty(n)
    for m in range(n + burn):
        U, capped = orc.update_link(U, S, beta, orc.HEATBATH, 21, 5, m)
        assert capped == 0
        if m >= burn:
            vals[m - burn] = np.trace(U @ G).real
    bins = vals.reshape(100, -1).mean(axis=1)
    err = bins.std(ddof=1) / np.sqrt(len(bins))
    want = _sun_onelink_mean_retr(nc, beta * s / nc)
    assert abs(vals.mean() - want) < 5 * err + 1e-3, (vals.mean(), want, err)
    assert np.abs(U @ dag(U) - np.eye(nc)).max() < 1e-12


# ------------------------------------------------------ lattice-wide limits ----

def _run(nc, dims, beta, sweeps, therm, n_hb, n_or, seed, hot):
    U = orc.init(nc, dims, hot=hot, seed=seed)
    hist = []
    step = 0
    for s in range(therm + sweeps):
        orc.sweep(U, beta, n_hb, n_or, True, seed, step)
        step += n_hb
        if s >= therm:
            hist.append(orc.plaquette(U))
    h = np.array(hist)
    bins = h.reshape(20, -1).mean(axis=1)
    return h.mean(), bins.std(ddof=1) / np.sqrt(len(bins))


@pytest.mark.parametrize("nc,beta", [(2, 0.5), (3, 1.0), (4, 1.6)])
def test_strong_coupling_plaquette(nc, beta):
    """At small beta the plaquettes decouple: <P> equals the one-plaquette
    value (1/nc) d ln Z/dc at c = beta/nc (beta/4 for SU(2), beta/18 for
    SU(3), beta/(2 nc^2) for nc >= 3 at leading order), up to O(beta^5)."""
    mean, err = _run(nc, (4, 4, 4, 4), beta, 200, 20, 1, 0, seed=300 + nc, hot=True)
    want = _sun_onelink_mean_retr(nc, beta / nc) / nc
    assert abs(mean - want) < 5 * err + 2e-4, (mean, want, err)
    lead = beta / 4 if nc == 2 else beta / (2 * nc * nc)
    assert abs(want - lead) < 0.1 * lead


@pytest.mark.parametrize("nc,beta", [(2, 80.0), (3, 150.0)])
def test_weak_coupling_plaquette(nc, beta):
    """At large beta: 1 - <P> = (nc^2 - 1)/(4 beta) + O(1/beta^2) (one free
    gluon mode per non-gauge degree of freedom)."""
    mean, err = _run(nc, (4, 4, 4, 4), beta, 100, 40, 1, 1, seed=400 + nc, hot=False)
    want = (nc * nc - 1) / (4 * beta)
    assert abs((1 - mean) - want) < 0.05 * want + 5 * err, (1 - mean, want, err)


# ------------------------------------------------------------ determinism ----

@pytest.mark.parametrize("mode", [orc.HEATBATH, orc.OVERRELAX])
@pytest.mark.parametrize("nc", [2, 3])
def test_pass_result_does_not_depend_on_link_order(nc, mode):
    """Links of one (mu, parity) pass share no staple (Sec. 3): walking the
    pass backwards gives bitwise the same lattice."""
    U = random_gauge_config(nc, (4, 2, 4, 2), seed=500 + nc)
    for mu in range(4):
        for p in range(2):
            A = U.copy()
            B = U.copy()
            orc.update_pass(A, 5.0, mode, mu, p, 3, 17, reverse=False)
            orc.update_pass(B, 5.0, mode, mu, p, 3, 17, reverse=True)
            assert np.array_equal(A, B)
            changed = np.abs(A - U).reshape(4, -1).max(axis=1)
            assert changed[mu] > 0 and all(changed[m] == 0 for m in range(4) if m != mu)


def test_sweep_does_not_depend_on_thread_count():
    U = random_gauge_config(3, (4, 4, 4, 4), seed=600)
    A = U.copy()
    B = U.copy()
    old = orc.get_threads()
    try:
        orc.set_threads(1)
        orc.sweep(A, 6.0, 1, 2, True, 3, 10)
        pa = orc.plaquette(A)
        orc.set_threads(4)
        orc.sweep(B, 6.0, 1, 2, True, 3, 10)
        pb = orc.plaquette(B)
    finally:
        orc.set_threads(old)
    assert np.array_equal(A, B)
    assert pa == pb


def test_time_slab_passes_compose_to_a_full_pass():
    """Updating the t-slabs [0,2) and [2,Nt) one after the other equals one
    full pass (the slab form is what the CPU baseline times)."""
    U = random_gauge_config(2, (2, 2, 2, 6), seed=700)
    A = U.copy()
    B = U.copy()
    orc.update_pass(A, 2.3, orc.HEATBATH, 1, 0, 0, 5)
    orc.update_pass(B, 2.3, orc.HEATBATH, 1, 0, 0, 5, t_begin=0, t_end=2)
    orc.update_pass(B, 2.3, orc.HEATBATH, 1, 0, 0, 5, t_begin=2, t_end=6)
    assert np.array_equal(A, B)


def test_beta_zero_heatbath_is_haar():
    """beta = 0: the SU(2) heatbath draws every link from the Haar measure in
    one step, whatever the staple (E Tr U = 0, E|Tr U|^2 = 1); one
    Cabibbo-Marinari step is not an exact SU(3) heatbath (E|Tr U|^2 < 1 from a
    cold start) but repeated steps converge to Haar."""
    for nc, steps, exact in [(2, 1, True), (3, 1, False), (3, 8, True)]:
        U = orc.init(nc, (6, 6, 6, 6), hot=False, seed=1)
        orc.sweep(U, 0.0, steps, 0, False, seed=9, hb_step0=0)
        m = U.reshape(-1, nc, nc)
        tr = np.trace(m, axis1=1, axis2=2)
        n = len(tr)
        assert abs(tr.mean()) < 5 / np.sqrt(n)
        dev = abs((np.abs(tr) ** 2).mean() - 1)
        if exact:
            assert dev < 5 * np.sqrt(2.0 / n)
        else:
            assert dev > 5 * np.sqrt(2.0 / n)


@pytest.mark.parametrize("nc", [2, 3, 4])
def test_fused_reunitarization_schedule(nc):
    """The fused schedule re-unitarizes every link once per sweep (all links
    special unitary afterwards) and differs from the separate placement only
    at the level of the unitarity drift it removes."""
    beta = 2.3 if nc == 2 else 0.7 * nc * nc
    U = random_gauge_config(nc, (4, 2, 4, 4), seed=800 + nc)
    rng = np.random.default_rng(nc)
    U = U + 1e-9 * (rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape))  # small drift
    A, B = U.copy(), U.copy()
    orc.sweep(A, beta, 1, 2, orc.REUNIT_AFTER, 4, 0)
    orc.sweep(B, beta, 1, 2, orc.REUNIT_FUSED, 4, 0)
    for X in (A, B):
        m = X.reshape(-1, nc, nc)
        assert np.abs(m @ dag(m) - np.eye(nc)).max() < 1e-14
        assert np.abs(np.linalg.det(m) - 1).max() < 1e-14
    assert 0 < np.abs(A - B).max() < 1e-6
    # with the last step's pass order, fused = pass then reunit link by link
    C = U.copy()
    orc.sweep(C, beta, 1, 1, orc.REUNIT_NONE, 4, 0)
    for mu in range(4):
        for p in range(2):
            orc.update_pass(C, beta, orc.OVERRELAX, mu, p, 0, 4, reunit_after=True)
    assert np.array_equal(C, B)


@pytest.mark.parametrize("nc", [2, 3])
def test_spread_reunitarization_schedule(nc):
    """Spread schedule: every link re-unitarized once per sweep, in the step
    given by its run of 32 site indices; a link re-unitarized in step s then
    takes the remaining updates of the sweep, so the drift left is that of at
    most n_steps - 1 updates."""
    beta = 2.3 if nc == 2 else 6.0
    dims = (8, 8, 4, 4)
    U = random_gauge_config(nc, dims, seed=850 + nc)
    rng = np.random.default_rng(nc)
    drift = U + 1e-6 * (rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape))
    A = drift.copy()
    orc.sweep(A, beta, 1, 2, orc.REUNIT_SPREAD, 4, 0)
    m = A.reshape(-1, nc, nc)
    assert np.abs(m @ dag(m) - np.eye(nc)).max() < 1e-12
    # pass by pass it is the same thing
    B = drift.copy()
    for s, mode in enumerate([orc.HEATBATH, orc.OVERRELAX, orc.OVERRELAX]):
        for mu in range(4):
            for p in range(2):
                orc.update_pass(B, beta, mode, mu, p, 0, 4, reunit_mod=3, reunit_rem=s)
    assert np.array_equal(A, B)
    # and without any re-unitarization the 1e-6 drift survives
    C = drift.copy()
    orc.sweep(C, beta, 1, 2, orc.REUNIT_NONE, 4, 0)
    m = C.reshape(-1, nc, nc)
    assert np.abs(m @ dag(m) - np.eye(nc)).max() > 1e-7
