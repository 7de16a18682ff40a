"""CPU checks of the configuration file format (sun_read_config_header): a
file written here by an independent numpy writer of the documented layout is
accepted, and every kind of damage is rejected on the host."""
import ctypes
import os
import struct

import numpy as np
import pytest


@pytest.fixture(scope="module")
def sun():
    from paper_1112_4533_gb300 import build as b
    b.build()
    from paper_1112_4533_gb300 import sun as s
    s.load_library()
    return s


def fnv1a_words(payload):
    """FNV-1a, 64-bit offset basis and prime, over little-endian 64-bit words."""
    h = 14695981039346656037
    for w in np.frombuffer(payload, dtype="<u8"):
        h ^= int(w)
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def write_file(path, nc=3, dims=(2, 2, 2, 4), precision=32, storage=12, beta=6.0, seed=9, step=5, sweeps=3,
               payload=None, checksum=None, magic=b"SUNCFG01", version=1):
    V = int(np.prod(dims))
    rows = storage // (2 * nc)
    n = 4 * V * rows * nc * 2
    if payload is None:
        rng = np.random.default_rng(1)
        payload = rng.standard_normal(n).astype(np.float32 if precision == 32 else np.float64).tobytes()
    cs = fnv1a_words(payload) if checksum is None else checksum
    hdr = struct.pack("<I3i4idQQQQQ40x", version, nc, precision, storage, *dims, beta, seed, step, sweeps,
                      len(payload), cs)
    assert len(hdr) == 120
    with open(path, "wb") as f:
        f.write(magic + hdr + payload)
    return payload


def test_header_of_a_well_formed_file(sun, tmp_path):
    p = tmp_path / "a.cfg"
    write_file(p)
    h = sun.read_config_header(p)
    assert (h["nc"], h["precision"], h["storage"], h["dims"]) == (3, 32, 12, (2, 2, 2, 4))
    assert (h["beta"], h["seed"], h["heatbath_step"], h["sweeps_done"]) == (6.0, 9, 5, 3)
    assert h["payload_bytes"] == 4 * 32 * 2 * 3 * 2 * 4


def test_fp64_full_storage_file(sun, tmp_path):
    p = tmp_path / "b.cfg"
    write_file(p, nc=2, precision=64, storage=8)
    assert sun.read_config_header(p)["storage"] == 8


@pytest.mark.parametrize("damage", ["magic", "version", "checksum", "truncated", "extra", "size", "nc", "dims"])
def test_damaged_files_are_rejected(sun, tmp_path, damage):
    p = tmp_path / "c.cfg"
    if damage == "magic":
        write_file(p, magic=b"SUNCFG02")
    elif damage == "version":
        write_file(p, version=2)
    elif damage == "checksum":
        write_file(p, checksum=12345)
    elif damage == "truncated":
        write_file(p)
        data = open(p, "rb").read()
        open(p, "wb").write(data[:-8])
    elif damage == "extra":
        write_file(p)
        with open(p, "ab") as f:
            f.write(b"\0" * 8)
    elif damage == "size":
        write_file(p, payload=b"\0" * 64)
    elif damage == "nc":
        write_file(p, nc=1, storage=2)
    elif damage == "dims":
        write_file(p, dims=(3, 2, 2, 4), payload=b"\0" * (4 * 48 * 2 * 3 * 2 * 4))
    with pytest.raises(sun.SunError):
        sun.read_config_header(p)


def test_header_only_read_skips_the_payload_check(sun, tmp_path):
    p = tmp_path / "d.cfg"
    write_file(p, checksum=1)
    assert sun.read_config_header(p, verify=False)["seed"] == 9
    with pytest.raises(sun.SunError):
        sun.read_config_header(p, verify=True)


def test_missing_file(sun, tmp_path):
    with pytest.raises(sun.SunError):
        sun.read_config_header(tmp_path / "none.cfg")
