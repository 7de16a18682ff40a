"""The integer FP32 <-> FP64 conversions of the kernels (to_f64 / to_f32 in
sun_device.cuh) against GB300's conversion instructions, bit for bit, through
sun_selftest_conversions: all 2^32 float encodings to double, and 2^26 seeded
double encodings to float (a quarter of them any encoding, a quarter with the
exponent across and around the float's normal range, a quarter with the 29
dropped fraction bits at or next to a rounding tie, a quarter at the largest and
smallest float exponents with fractions near all ones or zero)."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1112_4533_gb300 import build as b
    b.build()
    import paper_1112_4533_gb300 as p
    torch.cuda.init()
    return p.load_library()


@pytest.mark.parametrize("seed", [1, 20260611])
def test_conversions_match_the_hardware_bit_for_bit(lib, seed):
    out = (ctypes.c_uint64 * 4)()
    st = lib.sun_selftest_conversions(1 << 26, seed, out)
    assert st == 0, lib.sun_last_error()
    none = (1 << 64) - 1
    assert (out[0], out[1]) == (0, 0), (out[0], out[1], hex(out[2]), hex(out[3]))
    assert (out[2], out[3]) == (none, none)


def test_conversion_selftest_runs_without_double_cases(lib):
    """n = 0: only the exhaustive float -> double part."""
    out = (ctypes.c_uint64 * 4)()
    assert lib.sun_selftest_conversions(0, 1, out) == 0, lib.sun_last_error()
    assert out[0] == 0 and out[1] == 0
