"""The FP64 -> FP32 rounding the tensor-core operand prep does on bit patterns
(csrc/fbits.cuh), compiled for the host and checked against the host's IEEE
conversion (numpy float32 casts round to nearest, ties to even)."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1906_08148_gb300", "csrc")


@pytest.fixture(scope="module")
def fb(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("fbits"))
    src = os.path.join(d, "shim.c")
    with open(src, "w") as f:
        f.write('#include "fbits.cuh"\n'
                "uint32_t fb(uint64_t b, int s) { return fbits_from_double_rn(b, s); }\n"
                "int fs(uint64_t b) { return fp16_leaf_shift(b); }\n"
                "void fbv(const uint64_t* b, int64_t n, int s, uint32_t* out) {\n"
                "  for (int64_t i = 0; i < n; ++i) out[i] = fbits_from_double_rn(b[i], s);\n}\n")
    so = os.path.join(d, "libshim.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-x", "c", "-fPIC", "-shared", "-I", CSRC, "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.fb.argtypes = [ctypes.c_uint64, ctypes.c_int]
    lib.fb.restype = ctypes.c_uint32
    lib.fs.argtypes = [ctypes.c_uint64]
    lib.fs.restype = ctypes.c_int
    lib.fbv.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]

    def conv(x, shift=0):
        x = np.ascontiguousarray(x, np.float64)
        out = np.empty(x.shape, np.uint32)
        lib.fbv(x.ctypes.data, x.size, shift, out.ctypes.data)
        return out

    conv.shift = lambda b: lib.fs(int(b))
    return conv


def _host(x):
    with np.errstate(over="ignore"):
        return np.asarray(x, np.float64).astype(np.float32).view(np.uint32)


def test_matches_host_rounding_over_the_normal_range(fb):
    rng = np.random.default_rng(1)
    x = rng.uniform(1.0, 2.0, 400000) * np.exp2(rng.integers(-126, 128, 400000)) * rng.choice([-1.0, 1.0], 400000)
    got, ref = fb(x), _host(x)
    normal = np.abs(ref.view(np.float32)) >= np.float32(2.0 ** -126)
    assert np.array_equal(got[normal], ref[normal])


def test_ties_go_to_even(fb):
    rng = np.random.default_rng(2)
    f = (rng.uniform(1.0, 2.0, 20000) * np.exp2(rng.integers(-100, 100, 20000))).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + up.astype(np.float64)) / 2.0  # exact in FP64
    assert np.array_equal(fb(mid), _host(mid))
    assert np.array_equal(fb(-mid), _host(-mid))
    # the tie keeps whichever neighbour has an even significand
    even = np.where((f.view(np.uint32) & 1) == 0, f, up)
    assert np.array_equal(fb(mid), even.view(np.uint32))


def test_scale_is_folded_in_exactly(fb):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100000) * np.exp2(rng.integers(-60, 60, 100000))
    for s in (-120, -37, -1, 1, 14, 55, 120):
        y = np.ldexp(x, s)
        ok = (np.abs(y) >= 2.0 ** -126) & (np.abs(y) < 2.0 ** 127)
        assert np.array_equal(fb(x, s)[ok], _host(y)[ok]), s


def test_flush_overflow_and_specials(fb):
    assert fb(np.array([2.0 ** -127, -2.0 ** -140, 5e-324, 0.0, -0.0])).tolist() == [0, 0x80000000, 0, 0, 0x80000000]
    assert fb(np.array([2.0 ** 128, -1e300])).tolist() == [0x7F800000, 0xFF800000]
    assert fb(np.array([np.inf, -np.inf])).tolist() == [0x7F800000, 0xFF800000]
    n = fb(np.array([np.nan]))[0]
    assert (n & 0x7F800000) == 0x7F800000 and (n & 0x007FFFFF) != 0
    # the largest float and the carry of rounding into the exponent
    assert np.array_equal(fb(np.array([3.4028234663852886e38, 1.9999999999])), _host([3.4028234663852886e38,
                                                                                     1.9999999999]))


def test_fp16_leaf_shift_matches_frexp(fb):
    rng = np.random.default_rng(4)
    for t in np.concatenate([rng.uniform(0.5, 1.0, 2000) * np.exp2(rng.integers(-200, 200, 2000)),
                             [1.0, 2.0 ** 14, 2.0 ** 15 - 1.0, 2.0 ** 15, 1e-300, 1e300]]):
        x = math.frexp(t)[1]
        want = max(-120, min(120, 15 - x))
        b = np.array([t]).view(np.uint64)[0]
        assert fb.shift(b) == want, t
        if abs(want) < 120:
            assert 2.0 ** 14 <= t * 2.0 ** want < 2.0 ** 15
    assert fb.shift(0) == 0
    assert fb.shift(np.array([5e-324]).view(np.uint64)[0]) == 120
