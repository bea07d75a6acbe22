"""The error-free BF16 split of the tensor-core forms (csrc/slices.cuh),
compiled for the host and checked on the CPU against exact rational
arithmetic (Python fractions) and plain integer sums.

What the split promises, per line of a leaf (a row of an A leaf, a column of
a B leaf) after the per-leaf scale 2^f:
    x 2^f = sum_{s<S} d_s 2^(e - 8 - 9 s) + r,   |r| <= 2^(e - 9 S),
    |x 2^f| < 2^e for every x of the line,
    |d_0| <= 256, -256 <= d_s <= 255 (s >= 1),
every slice d_s 2^(e - 8 - 9 s) a BF16 value, and, for a row r of A and a
column c of B, the K = 64 sums of digit products of one index sum g are
integers of magnitude <= (g + 1) 2^22: exact in FP32 for g <= 1 (and g = 2,
<= 3 * 2^22 < 2^24), which is what makes the tensor-core accumulators of
index sums 0 and 1 exact.  The element-wise bound the GPU test uses,
    |sum_k a_rk b_kc - sum_k sum_{s+t<S} A_s B_t| <= 64 (S + 1.01) 2^(eA + eB - 9 S),
is checked here against the exact product."""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1906_08148_gb300", "csrc")


@pytest.fixture(scope="module")
def sl(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("slices"))
    src = os.path.join(d, "shim.cpp")
    with open(src, "w") as f:
        f.write('#include "slices.cuh"\n'
                'extern "C" {\n'
                "int lshift(int e) { return slice_leaf_shift(e); }\n"
                "int lexp(int e, int f) { return slice_line_exp(e, f); }\n"
                "void digits(int S, const uint64_t* b, const int* emax, int64_t n, int32_t* d) {\n"
                "  for (int64_t i = 0; i < n; ++i) {\n"
                "    if (S == 3) slice_digits<3>(b[i], emax[i], d + 3 * i);\n"
                "    else if (S == 4) slice_digits<4>(b[i], emax[i], d + 4 * i);\n"
                "    else slice_digits<5>(b[i], emax[i], d + 5 * i);\n"
                "  }\n"
                "}\n"
                "void bf16(const int32_t* d, const int* p, int64_t n, uint16_t* out) {\n"
                "  for (int64_t i = 0; i < n; ++i) out[i] = slice_bf16_bits(d[i], p[i]);\n"
                "}\n"
                "}\n")
    so = os.path.join(d, "libshim.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.lshift.argtypes = [ctypes.c_int]
    lib.lexp.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.digits.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.bf16.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return lib


def biased_exp(x):
    return ((np.ascontiguousarray(x, np.float64).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int32)


def split_leaf(lib, a, S, role):
    """Digits (m, m, S) and line exponents of leaf a: role 0 lines are rows,
    role 1 lines are columns.  Returns (digits, e per line, f)."""
    E = biased_exp(a)
    emax_line = E.max(axis=1) if role == 0 else E.max(axis=0)
    f = lib.lshift(int(E.max()))
    e = np.array([lib.lexp(int(v), f) for v in emax_line], np.int32)
    em = np.broadcast_to(emax_line[:, None] if role == 0 else emax_line[None, :], a.shape)
    b = np.ascontiguousarray(a, np.float64).view(np.uint64).ravel()
    em = np.ascontiguousarray(em, np.int32)  # kept alive across the call
    d = np.empty(a.size * S, np.int32)
    lib.digits(S, b.ctypes.data, em.ctypes.data, a.size, d.ctypes.data)
    return d.reshape(a.shape + (S,)), e, f


def leaves(seed):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, (64, 64))
    dist = np.abs(np.subtract.outer(np.arange(64), np.arange(64)))
    yield u                                                 # uniform
    yield u * np.exp(-0.3 * dist)                           # decay across the leaf
    yield u * np.exp(-0.6 * dist) * 1e-9                    # small leaf, wide range
    yield np.ldexp(u, rng.integers(-30, 30, (64, 64)))      # wild exponents
    yield np.where(rng.random((64, 64)) < 0.5, 0.0, u)      # half zeros
    z = np.zeros((64, 64))
    z[5, :] = u[5, :]
    yield z                                                 # one non-zero row (others all zero)
    yield np.full((64, 64), -1.0)                           # every element at the line maximum


@pytest.mark.parametrize("S", [3, 4])
@pytest.mark.parametrize("role", [0, 1])
@pytest.mark.parametrize("seed", [1, 2])
def test_digits_bounded_and_reconstruct_within_half_a_unit(sl, S, role, seed):
    for a in leaves(seed):
        d, e, f = split_leaf(sl, a, S, role)
        assert np.all(np.abs(d[..., 0]) <= 256)
        assert np.all((d[..., 1:] >= -256) & (d[..., 1:] <= 255))
        # exact check on every element: x 2^f - sum_s d_s 2^(e - 8 - 9 s)
        rows, cols = a.shape
        for r in range(0, rows, 7):
            for c in range(cols):
                line = r if role == 0 else c
                el = int(e[line])
                x = Fraction(float(a[r, c])) * Fraction(2) ** f
                assert abs(x) < Fraction(2) ** el or a[r, c] == 0.0
                rep = sum(Fraction(int(d[r, c, s])) * Fraction(2) ** (el - 8 - 9 * s) for s in range(S))
                assert abs(x - rep) <= Fraction(2) ** (el - 9 * S), (r, c)


@pytest.mark.parametrize("S", [3, 4])
def test_slices_are_bf16_values(sl, S):
    rng = np.random.default_rng(3)
    a = np.ldexp(rng.uniform(-1, 1, (64, 64)), rng.integers(-60, 4, (64, 64)))
    d, e, f = split_leaf(sl, a, S, 0)
    p = (e[:, None, None] - 8 - 9 * np.arange(S)[None, None, :]) * np.ones_like(d)
    bits = np.empty(d.size, np.uint16)
    dd, pp = np.ascontiguousarray(d.ravel(), np.int32), np.ascontiguousarray(p.ravel(), np.int32)
    sl.bf16(dd.ctypes.data, pp.ctypes.data, d.size, bits.ctypes.data)
    back = (bits.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    want = np.where(pp >= -126, dd.astype(np.float64) * np.exp2(pp.astype(np.float64)), 0.0)
    assert np.array_equal(back, want)


def test_leaf_shift_puts_the_largest_element_in_one_to_two(sl):
    for x in (1.0, 1.5, 0.75, 3.0e-17, 7.0e10, 2.0 ** -1000):
        f = sl.lshift(int(biased_exp(np.array([x]))[0]))
        assert 1.0 <= x * 2.0 ** f < 2.0 or f in (120, -120)
    assert sl.lshift(0) == 0
    assert sl.lshift(int(biased_exp(np.array([2.0 ** -500]))[0])) == 120
    assert sl.lshift(int(biased_exp(np.array([2.0 ** 300]))[0])) == -120


@pytest.mark.parametrize("S", [3, 4])
def test_level_sums_fit_the_fp32_accumulator_exactly(sl, S):
    """Digit products of one index sum g, summed over K = 64 for one (row, column):
    integers of magnitude <= (g + 1) 2^22, including the extreme case where every
    digit is at its bound."""
    cases = list(zip(leaves(4), leaves(5)))
    for a, b in cases:
        da, _, _ = split_leaf(sl, a, S, 0)
        db, _, _ = split_leaf(sl, b, S, 1)
        for g in range(S):
            tot = np.zeros((64, 64), np.int64)
            for s in range(g + 1):
                tot += da[..., s].astype(np.int64) @ db[..., g - s].astype(np.int64)
            assert np.max(np.abs(tot)) <= (g + 1) * 2 ** 22
            if g <= 2:
                assert np.max(np.abs(tot)) < 2 ** 24  # every such integer is an FP32 value


@pytest.mark.parametrize("S", [3, 4])
def test_element_bound_of_one_leaf_product(sl, S):
    """sum_k a_rk b_kc minus the slice products with index sum < S, exactly,
    against 64 (S + 1.01) 2^(eA_r + eB_c - 9 S) (scales 2^-fA, 2^-fB undone)."""
    rng = np.random.default_rng(6)
    dist = np.abs(np.subtract.outer(np.arange(64), np.arange(64)))
    for a, b in ((rng.uniform(-1, 1, (64, 64)) * np.exp(-0.2 * dist), rng.uniform(-1, 1, (64, 64))),
                 (np.ldexp(rng.uniform(-1, 1, (64, 64)), rng.integers(-20, 5, (64, 64))),
                  rng.uniform(-1, 1, (64, 64)) * 1e-6)):
        da, ea, fa = split_leaf(sl, a, S, 0)
        db, eb, fb = split_leaf(sl, b, S, 1)
        for r in (0, 17, 63):
            for c in (0, 40):
                exact = sum(Fraction(float(a[r, k])) * Fraction(float(b[k, c])) for k in range(64))
                approx = Fraction(0)
                for s in range(S):
                    for t in range(S - s):
                        ip = sum(int(da[r, k, s]) * int(db[k, c, t]) for k in range(64))
                        approx += Fraction(ip) * Fraction(2) ** (int(ea[r]) + int(eb[c]) - 16 - 9 * (s + t))
                approx *= Fraction(2) ** (-fa - fb)
                bound = 64 * (S + 1.01) * 2.0 ** (int(ea[r]) + int(eb[c]) - 9 * S - fa - fb)
                assert abs(float(exact - approx)) <= bound
