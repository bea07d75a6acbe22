"""The integer FP32 -> FP64 conversion of the tensor-core forms' finishing pass
(csrc/convert.cuh), compiled for the host: bit-identical to the exact
conversion for zeros, subnormals, normals of every exponent, infinities and
NaNs."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1906_08148_gb300", "csrc")


@pytest.fixture(scope="module")
def conv(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("convert"))
    src = os.path.join(d, "shim.cpp")
    with open(src, "w") as f:
        f.write('#include "convert.cuh"\n'
                'extern "C" void conv(const uint32_t* in, long n, uint64_t* out) {\n'
                "  for (long i = 0; i < n; ++i) out[i] = f32_to_f64_bits(in[i]);\n"
                "}\n")
    so = os.path.join(d, "libshim.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.conv.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p]
    return lib


def _run(lib, bits):
    bits = np.ascontiguousarray(bits, np.uint32)
    out = np.empty(len(bits), np.uint64)
    lib.conv(bits.ctypes.data, len(bits), out.ctypes.data)
    return out


def test_every_exponent_and_random_fractions(conv):
    rng = np.random.default_rng(0)
    exps = np.repeat(np.arange(256, dtype=np.uint32), 4000)
    frac = rng.integers(0, 1 << 23, len(exps), dtype=np.uint32)
    sign = rng.integers(0, 2, len(exps), dtype=np.uint32)
    bits = (sign << 31) | (exps << 23) | frac
    got = _run(conv, bits)
    want = bits.view(np.float32).astype(np.float64).view(np.uint64)
    finite = exps < 255
    assert np.array_equal(got[finite], want[finite])
    # infinities and NaNs: same class, sign and payload moved to the top
    g = got[~finite].view(np.float64)
    w = bits[~finite].view(np.float32).astype(np.float64)
    assert np.array_equal(np.isnan(g), np.isnan(w)) and np.array_equal(g[~np.isnan(g)], w[~np.isnan(w)])


def test_subnormals_zeros_and_extremes(conv):
    sub = np.concatenate([np.arange(1, 1 << 12, dtype=np.uint32), (1 << 23) - np.arange(1, 1 << 12, dtype=np.uint32),
                          np.uint32(1) << np.arange(23, dtype=np.uint32)])
    bits = np.concatenate([sub, sub | np.uint32(1 << 31), np.array([0, 1 << 31, 0x7f7fffff, 0x00800000, 0x3f800000],
                                                                   np.uint32)])
    got = _run(conv, bits)
    want = bits.view(np.float32).astype(np.float64).view(np.uint64)
    assert np.array_equal(got, want)
