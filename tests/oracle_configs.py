"""Thermalised gauge configurations made by the FP64 CPU oracle alone, as
inputs of GPU parity tests (the GPU receives them through sun_import_links;
nothing here reads a GPU result).

Cold start, then sweeps of 1 heatbath + 4 overrelaxation steps with the
re-unitarization after each sweep (Sec. 3 protocol).  From a cold start the
configuration reaches the equilibrium plaquette within a few sweeps with
every projected SU(2) strength k of W = U Sigma^+ well above zero (measured:
k >= 1.0 for SU(3) at beta 6.0 and 6.2 after six sweeps on 8x6x4x10, 16^4 and
16^3x32), the regime in which FP32 rounding of the staple moves an updated
link by no more than about 1e-6.
"""
import functools

import numpy as np

import oracle as orc


@functools.lru_cache(maxsize=8)
def _cold_thermal(nc, dims, beta, sweeps, seed):
    U = orc.init(nc, dims, False, seed)
    for s in range(sweeps):
        orc.sweep(U, beta, 1, 4, True, seed, s)
    U.setflags(write=False)
    return U


def cold_thermal(nc, dims, beta, sweeps=6, seed=13):
    """A fresh (writable) copy of the oracle's thermalised configuration."""
    return _cold_thermal(int(nc), tuple(int(d) for d in dims), float(beta), int(sweeps), int(seed)).copy()


def tiled(U, reps):
    """The configuration U (shape (4, Nt, Nz, Ny, Nx, nc, nc)) repeated reps =
    (rx, ry, rz, rt) times along each axis: a periodic configuration of the
    larger lattice whose local neighbourhoods are those of U."""
    rx, ry, rz, rt = reps
    return np.ascontiguousarray(np.tile(U, (1, rt, rz, ry, rx, 1, 1)))


def min_subgroup_strength(U, mu, par):
    """Smallest projected SU(2) strength k over the subgroups of W = U Sigma^+,
    over the links U_mu(x) of parity par (oracle staple)."""
    nc = U.shape[-1]
    nx, ny, nz = U.shape[4], U.shape[3], U.shape[2]
    flat = U.reshape(4, -1, nc, nc)
    kmin = np.inf
    for lex in range(flat.shape[1]):
        x, y, z, t = lex % nx, (lex // nx) % ny, (lex // (nx * ny)) % nz, lex // (nx * ny * nz)
        if (x + y + z + t) % 2 != par:
            continue
        w = flat[mu, lex] @ np.conj(orc.staple(U, mu, lex)).T
        for i in range(nc - 1):
            for j in range(i + 1, nc):
                b = w[np.ix_([i, j], [i, j])]
                q = 0.5 * np.array([(b[0, 0] + b[1, 1]).real, (b[0, 1] + b[1, 0]).imag,
                                    (b[0, 1] - b[1, 0]).real, (b[0, 0] - b[1, 1]).imag])
                kmin = min(kmin, float(np.linalg.norm(q)))
    return kmin


def drifted(U, eps, seed):
    """U with its rows 0 .. nc-2 moved off the group by eps-sized complex
    Gaussian noise; for nc = 2 row 1 set to (-conj(u01), conj(u00)) and for
    nc = 3 row 2 to conj(row0 x row1): the full matrices that quaternion and
    two-row storage of the moved rows stand for.  Used
    to make a re-unitarization visible (it moves such links by ~eps)."""
    nc = U.shape[-1]
    rng = np.random.default_rng(seed)
    V = U.copy()
    noise = rng.normal(size=V[..., :nc - 1, :].shape) + 1j * rng.normal(size=V[..., :nc - 1, :].shape)
    V[..., :nc - 1, :] += eps * noise
    if nc == 2:
        V[..., 1, 0] = -np.conj(V[..., 0, 1])
        V[..., 1, 1] = np.conj(V[..., 0, 0])
    if nc == 3:
        V[..., 2, :] = np.conj(np.cross(V[..., 0, :], V[..., 1, :]))
    return V
