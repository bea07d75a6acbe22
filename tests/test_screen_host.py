"""The norm-test screen of the task-list builder (csrc/screen.cuh), compiled
for the host: wherever it decides, its decision equals the FP64 rule
fl(||A|| ||B||) >= tau that the oracle applies (Algorithm 1's test), and it
leaves undecided only pairs whose product lies within about 2^-10 of tau or
that involve zero or subnormal norms."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1906_08148_gb300", "csrc")


@pytest.fixture(scope="module")
def scr(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("screen"))
    src = os.path.join(d, "shim.cpp")
    with open(src, "w") as f:
        f.write('#include "screen.cuh"\n'
                'extern "C" void decide(double tau, const double* a, const double* b, long n, int* out) {\n'
                "  const TauScreen sc = make_screen(tau);\n"
                "  for (long i = 0; i < n; ++i) out[i] = screen_decide(pack_norm(a[i]), pack_norm(b[i]), sc);\n"
                "}\n")
    so = os.path.join(d, "libshim.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC,
                           "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.decide.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p]
    return lib


def _decide(lib, tau, a, b):
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    out = np.empty(len(a), np.int32)
    lib.decide(tau, a.ctypes.data, b.ctypes.data, len(a), out.ctypes.data)
    return out


def _check(lib, tau, a, b):
    d = _decide(lib, tau, a, b)
    truth = (a * b) >= tau  # one FP64 rounding, as the oracle's test
    decided = d >= 0
    assert np.array_equal((d == 1)[decided], truth[decided])
    return d


TAUS = [1e-4, 1e-6, 1e-8, 1e-10, 0.5, 1.0, 2.0 ** -20, 3.0 * 2.0 ** -30, np.nextafter(1e-7, 1.0), 123.456]


@pytest.mark.parametrize("tau", TAUS)
def test_screen_agrees_with_fp64_products_over_the_range(scr, tau):
    rng = np.random.default_rng(1)
    n = 400_000
    a = 10.0 ** rng.uniform(-12, 4, n)
    b = tau / a * 10.0 ** rng.uniform(-3, 3, n)  # products spread over six decades around tau
    d = _check(scr, tau, a, b)
    # almost everything is decided without the FP64 product
    assert np.mean(d < 0) < 1e-3


@pytest.mark.parametrize("tau", TAUS)
def test_screen_near_tau(scr, tau):
    rng = np.random.default_rng(2)
    n = 400_000
    a = 10.0 ** rng.uniform(-6, 3, n)
    rel = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-17, -3, n)
    b = tau * (1.0 + rel) / a
    d = _check(scr, tau, a, b)
    # undecided only inside the margin (2^-10 plus the mantissa truncation)
    close = np.abs(a * b / tau - 1.0) < 2.0 ** -9
    assert np.all(close[d < 0])
    assert np.all(d[np.abs(a * b / tau - 1.0) > 2.0 ** -8] >= 0)


def test_screen_exponent_boundaries_and_special_values(scr):
    tau = 2.0 ** -20
    # products that are exactly tau, one ulp below and above, and powers of two around it
    a = np.array([2.0 ** -10, 2.0 ** -10, 2.0 ** -10, 2.0 ** -9, 2.0 ** -12, 1.0, 2.0 - 2.0 ** -52, 0.0, 5e-324, 1e-310])
    b = np.array([2.0 ** -10, np.nextafter(2.0 ** -10, 0), np.nextafter(2.0 ** -10, 1), 2.0 ** -12, 2.0 ** -7,
                  2.0 ** -22 * (2.0 - 2.0 ** -52), 2.0 ** -22 * (2.0 - 2.0 ** -52), 1.0, 1.0, 1e300])
    d = _check(scr, tau, a, b)
    assert d[7] == -1 and d[8] == -1 and d[9] == -1  # zero and subnormal norms take the FP64 product
    # tau = 0 and subnormal tau: always the FP64 product
    assert np.all(_decide(scr, 0.0, a[:7], b[:7]) == -1)
    assert np.all(_decide(scr, 1e-320, a[:7], b[:7]) == -1)


def test_screen_mutant_margin_is_caught(scr):
    """A screen without its margin (deciding by the FP32 product alone) would
    disagree with FP64 near tau: the near-tau test above has cases that need
    the margin."""
    tau = 1e-6
    rng = np.random.default_rng(3)
    a = 10.0 ** rng.uniform(-6, 3, 200_000)
    b = tau * (1.0 + rng.choice([-1.0, 1.0], 200_000) * 10.0 ** rng.uniform(-9, -6, 200_000)) / a
    fp32 = (a.astype(np.float32) * b.astype(np.float32)).astype(np.float64) >= np.float32(tau)
    assert np.any(fp32 != ((a * b) >= tau))
    _check(scr, tau, a, b)
