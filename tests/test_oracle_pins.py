"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with a
published value, a closed form, an invariant, a reduction to a library routine
or a brute-force evaluation, chosen so that a dropped term, a wrong sign, a
wrong neighbour or a transposed operand fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle as orc
from tests.inputs import random_gauge_config, random_site_field, random_su_n

HERE = os.path.dirname(os.path.abspath(__file__))


def dims_of(U):
    return (U.shape[4], U.shape[3], U.shape[2], U.shape[1])


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


# ---------------------------------------------------------------- Philox ----

def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors of its authors (SC'11 distribution)."""
    rows = 0
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            lhs, rhs = line.split("|")
            v = [int(s, 16) for s in lhs.split()]
            want = [int(s, 16) for s in rhs.split()]
            assert orc.philox4x32_10(v[:4], v[4:6]) == want
            rows += 1
    assert rows == 3


def test_uniform_is_exact_in_float32():
    for u in [0, 1, 255, 256, 0x12345678, 0xFFFFFF00, 0xFFFFFFFF]:
        r = orc.uniform(u)
        assert 0.0 < r < 1.0
        assert float(np.float32(r)) == r
    assert orc.uniform(0) == 2.0 ** -24
    assert orc.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24


# ----------------------------------------------- plaquette and Polyakov ----

@pytest.mark.parametrize("nc", [2, 3, 4, 6])
def test_cold_start_observables_are_one(nc):
    U = orc.init(nc, (4, 4, 2, 6), hot=False, seed=1)
    assert orc.plaquette(U) == 1.0
    assert orc.polyakov(U) == 1.0


def _abelian_config(nc, dims, seed):
    """Diagonal links diag(e^{i th_1}, ..., e^{i th_nc}) with sum th = 0."""
    nx, ny, nz, nt = dims
    rng = np.random.default_rng(seed)
    th = rng.uniform(-np.pi, np.pi, size=(nc - 1, 4, nt, nz, ny, nx))
    th = np.concatenate([th, -th.sum(axis=0, keepdims=True)], axis=0)
    U = np.zeros((4, nt, nz, ny, nx, nc, nc), dtype=np.complex128)
    for a in range(nc):
        U[..., a, a] = np.exp(1j * th[a])
    return U, th


def _roll_axis(mu):
    # canonical array axes (t, z, y, x) for direction mu = x, y, z, t
    return {0: 3, 1: 2, 2: 1, 3: 0}[mu]


@pytest.mark.parametrize("nc", [2, 3, 4])
def test_plaquette_and_polyakov_abelian_closed_form(nc):
    """For commuting links P_{mu nu} is diag(e^{i F}) with the lattice curl
    F = th_mu(x) + th_nu(x+mu) - th_mu(x+nu) - th_nu(x) (Eq. 4), and the
    Polyakov loop is the mean of exp(i sum_t th_t)."""
    dims = (4, 6, 2, 4)
    U, th = _abelian_config(nc, dims, seed=nc)
    nx, ny, nz, nt = dims
    V = nx * ny * nz * nt
    total = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = (th[:, mu] + np.roll(th[:, nu], -1, axis=1 + _roll_axis(mu))
                 - np.roll(th[:, mu], -1, axis=1 + _roll_axis(nu)) - th[:, nu])
            total += np.cos(F).sum()
    assert abs(orc.plaquette(U) - total / (6 * V * nc)) < 1e-13
    phase = th[:, 3].sum(axis=1)  # sum over t, shape (nc, nz, ny, nx)
    want = np.exp(1j * phase).sum() / (nc * nx * ny * nz)
    assert abs(orc.polyakov(U) - want) < 1e-13


def gauge_transform(U, G):
    """U_mu(x) -> G(x) U_mu(x) G(x+mu)^+."""
    out = np.empty_like(U)
    for mu in range(4):
        Gp = np.roll(G, -1, axis=_roll_axis(mu))
        out[mu] = G @ U[mu] @ dag(Gp)
    return out


@pytest.mark.parametrize("nc", [2, 3, 5])
def test_observables_are_gauge_invariant(nc):
    dims = (4, 2, 4, 6)
    U = random_gauge_config(nc, dims, seed=10 + nc)
    G = random_site_field(nc, dims, seed=20 + nc)
    Ug = gauge_transform(U, G)
    assert abs(orc.plaquette(Ug) - orc.plaquette(U)) < 1e-12
    assert abs(orc.polyakov(Ug) - orc.polyakov(U)) < 1e-12
    # a non-closed loop is not invariant: make sure the transform is not trivial
    assert np.abs(Ug - U).max() > 0.1


@pytest.mark.parametrize("nc", [2, 3, 4])
def test_polyakov_center_symmetry(nc):
    """Multiplying every U_t(x, t=0) by the centre element z = e^{2 pi i/nc}
    leaves the plaquette unchanged and multiplies the Polyakov loop by z."""
    U = random_gauge_config(nc, (2, 4, 2, 4), seed=30 + nc)
    z = np.exp(2j * np.pi / nc)
    Uz = U.copy()
    Uz[3, 0] *= z
    assert abs(orc.plaquette(Uz) - orc.plaquette(U)) < 1e-13
    assert abs(orc.polyakov(Uz) - z * orc.polyakov(U)) < 1e-13


# ---------------------------------------------------------------- staple ----

@pytest.mark.parametrize("nc", [2, 3, 4])
def test_staple_sums_to_four_times_plaquettes(nc):
    """Every plaquette holds four links and the staple of a link collects the
    six plaquettes through it (Eq. 9), so sum_{x,mu} ReTr(U Sigma^+) =
    4 sum_{x, mu<nu} ReTr P = 4 * 6 V nc <P>."""
    dims = (2, 4, 2, 4)
    U = random_gauge_config(nc, dims, seed=40 + nc)
    V = int(np.prod(dims))
    flat = U.reshape(4, V, nc, nc)
    total = 0.0
    for mu in range(4):
        for lex in range(V):
            S = orc.staple(U, mu, lex)
            total += np.trace(flat[mu, lex] @ dag(S)).real
    assert abs(total - 4 * 6 * V * nc * orc.plaquette(U)) < 1e-9


@pytest.mark.parametrize("nc", [2, 3])
def test_staple_gives_local_action_change(nc):
    """Brute force: change one link, recompute the Wilson action (Eq. 3) from
    all plaquettes; the change equals -(beta/nc) ReTr((U' - U) Sigma^+)."""
    dims = (4, 2, 2, 4)
    beta = 2.7
    U = random_gauge_config(nc, dims, seed=50 + nc)
    V = int(np.prod(dims))
    rng = np.random.default_rng(60 + nc)
    for mu, lex in [(0, 0), (1, 7), (2, 13), (3, V - 1)]:
        S = orc.staple(U, mu, lex)
        Unew = U.copy()
        flat = Unew.reshape(4, V, nc, nc)
        old = flat[mu, lex].copy()
        flat[mu, lex] = random_su_n(nc, rng, 1)[0]
        action = lambda W: beta * 6 * V * (1 - orc.plaquette(W))
        dS = action(Unew) - action(U)
        want = -(beta / nc) * np.trace((flat[mu, lex] - old) @ dag(S)).real
        assert abs(dS - want) < 1e-10


# -------------------------------------------------------- reunitarization ----

def _qr_reunit(m):
    """Gram-Schmidt of the rows via numpy's QR of m^+, then det phase on the last row."""
    q, r = np.linalg.qr(dag(m))
    ph = np.diag(r) / np.abs(np.diag(r))
    q = q * ph[None, :]
    out = dag(q)
    det = np.linalg.det(out)
    out[-1] *= np.conj(det) / abs(det)
    return out


@pytest.mark.parametrize("nc", [2, 3, 4, 6])
def test_reunitarization_matches_qr_and_is_special_unitary(nc):
    rng = np.random.default_rng(70 + nc)
    for _ in range(20):
        m = rng.normal(size=(nc, nc)) + 1j * rng.normal(size=(nc, nc))
        u = orc.reunit_link(m)
        assert np.abs(u @ dag(u) - np.eye(nc)).max() < 1e-14
        assert abs(np.linalg.det(u) - 1) < 1e-14
        assert np.abs(u - _qr_reunit(m)).max() < 1e-12
    # idempotent on SU(nc), and repairs a small drift
    g = random_su_n(nc, rng, 5)
    for u in g:
        assert np.abs(orc.reunit_link(u) - u).max() < 1e-14
        drift = u + 1e-6 * (rng.normal(size=(nc, nc)) + 1j * rng.normal(size=(nc, nc)))
        v = orc.reunit_link(drift)
        assert np.abs(v @ dag(v) - np.eye(nc)).max() < 1e-14
        assert np.abs(v - u).max() < 1e-5


def test_su2_reunitarization_rebuilds_second_row():
    """Sec. 2: normalise the first row, rebuild the second from it."""
    rng = np.random.default_rng(3)
    m = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    u = orc.reunit_link(m)
    r0 = m[0] / np.linalg.norm(m[0])
    assert np.allclose(u[0], r0, atol=1e-15)
    assert np.allclose(u[1], [-np.conj(r0[1]), np.conj(r0[0])], atol=1e-15)


# ---------------------------------------------------------------- hot start ----

@pytest.mark.parametrize("nc", [2, 3, 4])
def test_hot_start_is_haar(nc):
    """Haar moments: E Tr U = 0, E|Tr U|^2 = 1, and for SU(3) E (Tr U)^3 = 1
    (the epsilon-tensor invariant that tells SU(3) from U(3))."""
    dims = (6, 6, 6, 6)
    U = orc.init(nc, dims, hot=True, seed=123)
    m = U.reshape(-1, nc, nc)
    assert np.abs(m @ dag(m) - np.eye(nc)).max() < 1e-13
    assert np.abs(np.linalg.det(m) - 1).max() < 1e-13
    tr = np.trace(m, axis1=1, axis2=2)
    n = len(tr)
    assert abs(tr.mean()) < 5 / np.sqrt(n)
    assert abs((np.abs(tr) ** 2).mean() - 1) < 5 * np.sqrt(2.0 / n)
    if nc == 3:
        assert abs((tr ** 3).mean() - 1) < 5 * np.sqrt(6.0 / n)
    # different seeds and different links give different matrices
    U2 = orc.init(nc, dims, hot=True, seed=124)
    assert np.abs(U2 - U).max() > 0.5
