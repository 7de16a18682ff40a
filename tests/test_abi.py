"""CPU checks of the C ABI: the library loads, exports every entry point the
public header declares, and rejects invalid arguments on the host before any
device work (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1112_4533_gb300 import build as b
    b.build()
    from paper_1112_4533_gb300 import sun
    return sun.load_library()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(sun_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_method_calls():
    names = declared_functions()
    for need in ["sun_lattice_create", "sun_sweep", "sun_update_pass", "sun_reunitarize", "sun_plaquette",
                 "sun_polyakov_loop", "sun_export_links", "sun_import_links", "sun_run", "sun_lattice_destroy"]:
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1112_4533_gb300 import sun
    bound = {s[0] for s in sun.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_abi_version_and_status_strings(lib):
    assert lib.sun_abi_version() == 1
    for s in range(7):
        assert lib.sun_status_string(s)
    assert lib.sun_status_string(99) == b"unknown status"


def _dims(d):
    return (ctypes.c_int * 4)(*d)


def test_footprint_matches_storage_model(lib):
    from paper_1112_4533_gb300 import sun
    V = 48 * 48 * 48 * 96
    f12 = sun.footprint_bytes(3, (48, 48, 48, 96), 32, 12)
    f18 = sun.footprint_bytes(3, (48, 48, 48, 96), 32, 18)
    assert 4 * V * 48 <= f12 < 4 * V * 48 + (64 << 20)
    assert 4 * V * 72 <= f18 < 4 * V * 72 + (64 << 20)
    assert sun.footprint_bytes(2, (8, 8, 8, 8), 64, 4) >= 4 * 8 ** 4 * 32
    assert sun.footprint_bytes(6, (8, 8, 8, 8), 32, 0) >= 4 * 8 ** 4 * 72 * 4


@pytest.mark.parametrize("nc,dims,prec,storage,want", [
    (3, (3, 4, 4, 4), 32, 0, 1),            # odd extent
    (3, (0, 4, 4, 4), 32, 0, 1),            # empty extent
    (1, (4, 4, 4, 4), 32, 0, 1),            # nc < 2
    (3, (4, 4, 4, 4), 16, 0, 1),            # precision
    (3, (4, 4, 4, 4), 32, 13, 5),           # storage not built
    (2, (4, 4, 4, 4), 32, 12, 5),
    (7, (4, 4, 4, 4), 32, 0, 5),            # nc not built
    (3, (1024, 1024, 1024, 2), 32, 0, 1),   # 4V >= 2^32
])
def test_create_rejects_invalid_arguments_on_the_host(lib, nc, dims, prec, storage, want):
    from paper_1112_4533_gb300 import sun
    o = sun._options(prec, storage)
    h = ctypes.c_void_p(1234)
    st = lib.sun_lattice_create(ctypes.byref(h), nc, _dims(dims), 6.0, 0, 1, ctypes.byref(o))
    assert st == want
    assert h.value is None
    assert lib.sun_last_error()
    assert lib.sun_footprint_bytes(nc, _dims(dims), ctypes.byref(o)) == 0


def test_calls_on_null_handles_fail_cleanly(lib):
    assert lib.sun_sweep(None, 1, 1) == 1
    assert lib.sun_update_pass(None, 0, 0, 0) == 1
    assert lib.sun_update_pass_reunit(None, 0, 0, 0) == 1
    v = ctypes.c_double()
    assert lib.sun_plaquette(None, ctypes.byref(v)) == 1
    assert lib.sun_selftest_conversions(16, 1, None) == 1
    lib.sun_lattice_destroy(None)


def test_negative_beta_rejected(lib):
    from paper_1112_4533_gb300 import sun
    o = sun._options()
    h = ctypes.c_void_p()
    assert lib.sun_lattice_create(ctypes.byref(h), 3, _dims((4, 4, 4, 4)), -1.0, 0, 1, ctypes.byref(o)) == 1


def test_autotune_rejects_invalid_requests_on_the_host(lib):
    from paper_1112_4533_gb300 import sun
    ms = ctypes.c_double()
    o = sun._options()
    d = _dims((4, 4, 4, 4))
    # a sweep without steps, unknown flags, caller memory: refused before any device work
    assert lib.sun_autotune(3, d, 6.0, 0, 0, 0, ctypes.byref(o), ctypes.byref(ms)) == 1
    assert lib.sun_autotune(3, d, 6.0, 1, 1, 64, ctypes.byref(o), ctypes.byref(ms)) == 1
    o.device_buf = ctypes.c_void_p(4096)
    assert lib.sun_autotune(3, d, 6.0, 1, 1, 0, ctypes.byref(o), ctypes.byref(ms)) == 1
    assert lib.sun_autotune(3, d, 6.0, 1, 1, 0, None, ctypes.byref(ms)) == 1
    assert lib.sun_autotune_batch(0, None, None, None, 1, 1, 0, ctypes.byref(sun._options()), None) == 1


def test_wavefront_options_validated_on_the_host(lib):
    from paper_1112_4533_gb300 import sun
    h = ctypes.c_void_p()
    for field, bad in (("variant", 32), ("wave_lag", -1), ("wave_skip_units", -2), ("graph_sweeps", 65)):
        o = sun._options()
        setattr(o, field, bad)
        assert lib.sun_lattice_create(ctypes.byref(h), 3, _dims((4, 4, 4, 4)), 6.0, 0, 1, ctypes.byref(o)) == 1


def test_slab_arguments_rejected_on_the_host(lib):
    from paper_1112_4533_gb300 import sun
    h = ctypes.c_void_p()
    o = sun._options()
    # Nt = 8: 3 slabs do not divide it, 8 slabs would be 1 slice thick (odd), 0 slabs is no decomposition
    for n in (3, 8, 0):
        assert lib.sun_slabs_create(ctypes.byref(h), 3, _dims((4, 4, 4, 8)), n, 6.0, 0, 1, ctypes.byref(o)) == 1
    o.device_buf = ctypes.c_void_p(4096)
    assert lib.sun_slabs_create(ctypes.byref(h), 3, _dims((4, 4, 4, 8)), 2, 6.0, 0, 1, ctypes.byref(o)) == 1
