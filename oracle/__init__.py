"""ctypes wrapper of the FP64 CPU oracle (oracle/sun_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The product library never imports it.

Links are numpy complex128 arrays of shape (4, Nt, Nz, Ny, Nx, nc, nc), the
canonical order [mu][t][z][y][x][row][col] (x fastest among the sites).
"""
import ctypes
import os

import numpy as np

from . import build as _build

HEATBATH = 0
OVERRELAX = 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = os.environ.get("SUN_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i4 = ctypes.POINTER(ctypes.c_int)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_version.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_get_threads.restype = ctypes.c_int
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_uniform.argtypes = [ctypes.c_uint32]
        L.orc_uniform.restype = ctypes.c_double
        L.orc_init.argtypes = [d, ctypes.c_int, i4, ctypes.c_int, ctypes.c_uint64]
        L.orc_pass.argtypes = [d, ctypes.c_int, i4, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_pass.restype = ctypes.c_int64
        L.orc_sweep.argtypes = [d, ctypes.c_int, i4, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32]
        L.orc_reunitarize.argtypes = [d, ctypes.c_int, i4]
        L.orc_plaquette.argtypes = [d, ctypes.c_int, i4]
        L.orc_plaquette.restype = ctypes.c_double
        L.orc_polyakov.argtypes = [d, ctypes.c_int, i4, d, d]
        L.orc_staple.argtypes = [d, ctypes.c_int, i4, ctypes.c_int, ctypes.c_int64, d]
        L.orc_update_link.argtypes = [d, d, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_update_link.restype = ctypes.c_int
        L.orc_su2_heatbath.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_int, d]
        L.orc_su2_heatbath.restype = ctypes.c_int
        L.orc_reunit_link.argtypes = [d, ctypes.c_int]
        L.orc_random_sun.argtypes = [d, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32]
        _lib = L
    return _lib


def _dptr(a):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(v) for v in dims])


def set_threads(n):
    return lib().orc_set_threads(int(n))


def get_threads():
    return lib().orc_get_threads()


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(u):
    return lib().orc_uniform(int(u))


def new_lattice(nc, dims):
    nx, ny, nz, nt = dims
    return np.zeros((4, nt, nz, ny, nx, nc, nc), dtype=np.complex128)


def init(nc, dims, hot, seed):
    U = new_lattice(nc, dims)
    lib().orc_init(_dptr(U), nc, _dims(dims), int(bool(hot)), int(seed))
    return U


def update_pass(U, beta, mode, mu, parity, hb_step, seed, t_begin=0, t_end=-1, reverse=False,
                reunit_after=False, reunit_mod=0, reunit_rem=0):
    """reunit_after re-unitarizes every updated link; reunit_mod/reunit_rem select
    runs of 32 even/odd site indices ((lex >> 1) >> 5) % reunit_mod == reunit_rem."""
    nc = U.shape[-1]
    dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    if reunit_after:
        reunit_mod, reunit_rem = 1, 0
    return lib().orc_pass(_dptr(U), nc, _dims(dims), float(beta), int(mode), int(mu), int(parity),
                          int(hb_step), int(seed), int(t_begin), int(t_end), int(bool(reverse)),
                          int(reunit_mod), int(reunit_rem))


REUNIT_NONE, REUNIT_AFTER, REUNIT_FUSED, REUNIT_SPREAD = 0, 1, 2, 3


def sweep(U, beta, n_hb, n_or, reunit, seed, hb_step0):
    """reunit: False/0 none, True/1 after the sweep, 2 fused into the last step,
    3 spread over the steps (runs of 32 links)."""
    nc = U.shape[-1]
    dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    lib().orc_sweep(_dptr(U), nc, _dims(dims), float(beta), int(n_hb), int(n_or),
                    int(reunit), int(seed), int(hb_step0))


def reunitarize(U):
    nc = U.shape[-1]
    dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    lib().orc_reunitarize(_dptr(U), nc, _dims(dims))


def plaquette(U):
    nc = U.shape[-1]
    dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    return lib().orc_plaquette(_dptr(U), nc, _dims(dims))


def polyakov(U):
    nc = U.shape[-1]
    dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    re = ctypes.c_double()
    im = ctypes.c_double()
    lib().orc_polyakov(_dptr(U), nc, _dims(dims), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def staple(U, mu, lex):
    nc = U.shape[-1]
    dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    S = np.zeros((nc, nc), dtype=np.complex128)
    lib().orc_staple(_dptr(U), nc, _dims(dims), int(mu), int(lex), _dptr(S))
    return S


def update_link(Ulink, S, beta, mode, seed, link_id, hb_step):
    """Returns (new link, number of subgroup heatbaths that hit the attempt cap)."""
    u = np.ascontiguousarray(Ulink, dtype=np.complex128).copy()
    s = np.ascontiguousarray(S, dtype=np.complex128)
    capped = lib().orc_update_link(_dptr(u), _dptr(s), u.shape[-1], float(beta), int(mode),
                                   int(seed), int(link_id), int(hb_step))
    return u, capped


def su2_heatbath(alpha, seed, link_id, hb_step, subgroup):
    b = np.zeros(4)
    used = lib().orc_su2_heatbath(float(alpha), int(seed), int(link_id), int(hb_step),
                                  int(subgroup), _dptr(b))
    return b, used


def reunit_link(Ulink):
    u = np.ascontiguousarray(Ulink, dtype=np.complex128).copy()
    lib().orc_reunit_link(_dptr(u), u.shape[-1])
    return u


def random_sun(nc, seed, link_id):
    u = np.zeros((nc, nc), dtype=np.complex128)
    lib().orc_random_sun(_dptr(u), nc, int(seed), int(link_id))
    return u


def lex_of(dims, x, y, z, t):
    nx, ny, nz, nt = dims
    return x + nx * (y + ny * (z + nz * t))
