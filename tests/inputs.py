"""Seeded synthetic inputs shared by the oracle pins and the GPU parity tests.

Holds none of the method's arithmetic (no staple, update, reunitarization or
observable): only random SU(Nc) matrices drawn with scipy's Haar sampler and the
lattice shapes of the workloads.
"""
import numpy as np
from scipy.stats import unitary_group


def random_su_n(nc, rng, count):
    """`count` Haar-random SU(nc) matrices, shape (count, nc, nc), complex128."""
    count = int(count)
    if count == 0:
        return np.zeros((0, nc, nc), dtype=np.complex128)
    m = unitary_group.rvs(nc, size=count, random_state=rng)
    m = np.asarray(m, dtype=np.complex128).reshape(count, nc, nc)
    det = np.linalg.det(m)
    m[:, -1, :] *= np.conj(det)[:, None] / np.abs(det)[:, None]
    return m


def random_gauge_config(nc, dims, seed):
    """Haar-random links in canonical layout (4, Nt, Nz, Ny, Nx, nc, nc)."""
    nx, ny, nz, nt = dims
    rng = np.random.default_rng(seed)
    m = random_su_n(nc, rng, 4 * nx * ny * nz * nt)
    return m.reshape(4, nt, nz, ny, nx, nc, nc)


def random_site_field(nc, dims, seed):
    """One Haar-random SU(nc) matrix per site, shape (Nt, Nz, Ny, Nx, nc, nc)."""
    nx, ny, nz, nt = dims
    rng = np.random.default_rng(seed)
    return random_su_n(nc, rng, nx * ny * nz * nt).reshape(nt, nz, ny, nx, nc, nc)


def near_identity_config(nc, dims, seed, eps):
    """Links exp(i eps H) with random Hermitian H: an ordered start as at weak coupling."""
    nx, ny, nz, nt = dims
    rng = np.random.default_rng(seed)
    n = 4 * nx * ny * nz * nt
    a = rng.normal(size=(n, nc, nc)) + 1j * rng.normal(size=(n, nc, nc))
    h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
    w, v = np.linalg.eigh(h)
    u = v @ (np.exp(1j * eps * w)[:, :, None] * np.conj(np.swapaxes(v, 1, 2)))
    det = np.linalg.det(u)
    u[:, -1, :] *= np.conj(det)[:, None] / np.abs(det)[:, None]
    return u.reshape(4, nt, nz, ny, nx, nc, nc)


# Lattice shapes of the workloads (x, y, z, t).
SU2_SMALL = (8, 8, 8, 8)          # SU(2) 8^4, beta 2.3, cold start, FP64
SU3_MEDIUM = (16, 16, 16, 16)     # SU(3) 16^4, beta 6.0, hot start, FP32 12-real
SU3_LARGE = (48, 48, 48, 96)      # SU(3) 48^3 x 96, beta 6.2, cold start
