"""The oracle's pins catch plausible mistakes: each mutant below is a copy of
the oracle's C source with one planted error (a dropped term, a wrong sign or
index, a transposed operand, the squared form of the test), compiled on the
CPU; the battery of pin checks must reject every mutant and accept the
unmodified source."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth
from oracle import literal

SRC = os.path.join(os.path.dirname(oracle.__file__), "spamm_oracle.c")

MUTANTS = {
    "squared_test": ("return sqrt(sa) * sqrt(sb) >= tau;", "return sa * sb >= tau;"),
    "transposed_B": ("C[r * bs + c] += av * B[kk * bs + c];", "C[r * bs + c] += av * B[c * bs + kk];"),
    "wrong_sign": ("C[r * bs + c] += av * B[kk * bs + c];", "C[r * bs + c] -= av * B[kk * bs + c];"),
    "dropped_square": ("if (len == 1) return x[0] * x[0];", "if (len == 1) return x[0];"),
    "dropped_child": ("if (v >= 0.0) { s += v; any = 1; }", "if (v >= 0.0) { if (cj == 0) s += v; any = 1; }"),
    "wrong_index": ("out_ikj[3 * cnt + 2] = b_bj[q];", "out_ikj[3 * cnt + 2] = b_bi[q];"),
    "swapped_k_child": ("double nb = node(s->gb, t + 1, 2 * K + k, 2 * J + j);",
                        "double nb = node(s->gb, t + 1, 2 * K + (1 - k), 2 * J + j);"),
    "dropped_tail_leaf": ("for (int64_t p = cptr[g]; p < cptr[g + 1]; ++p) {",
                          "for (int64_t p = cptr[g]; p + 1 < cptr[g + 1]; ++p) {"),
}


def _compile(tmp_path, name, mutation):
    src = open(SRC).read()
    if mutation is not None:
        old, new = mutation
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-o", str(so), str(c), "-lm"])
    return oracle._configure(ctypes.CDLL(str(so)))


def _battery() -> list:
    """Pin checks; returns the names of the failing ones."""
    failed = []
    A = synth.dense(synth.DecayParams(n=64, kind=synth.KIND_1D, alpha=0.2, seed=3))
    B = synth.dense(synth.DecayParams(n=64, kind=synth.KIND_1D, alpha=0.2, seed=4))
    try:
        for bs in (4, 8):
            LA, LB = oracle.from_dense(A, bs), oracle.from_dense(B, bs)
            ref_sq = [math.fsum(float(v) ** 2 for v in LA.data[q].ravel()) for q in range(LA.m)]
            if not np.allclose(LA.sq, ref_sq, rtol=1e-13):
                failed.append("leaf norms vs fsum")
            if abs(oracle.frob_norm(LA) - np.linalg.norm(A)) > 1e-12 * np.linalg.norm(A):
                failed.append("root norm")
            C, _ = oracle.multiply(LA, LB, 0.0, oracle.SPAMM)
            if not np.allclose(oracle.to_dense(C), A @ B, rtol=1e-12, atol=1e-14):
                failed.append("tau=0 product")
            for tau in (1e-5, 1e-2):
                flat = oracle.kept_flat(LA, LB, tau, oracle.SPAMM)
                _, kl = literal.spamm_literal(A, B, tau, bs)
                lit = oracle._sort_ijk(np.array(kl, np.int32).reshape(-1, 3))
                if not np.array_equal(flat, lit):
                    failed.append("flat vs literal kept set")
                if not np.array_equal(flat, oracle.kept_recursive(LA, LB, tau, oracle.SPAMM)):
                    failed.append("recursive vs flat")
    except AssertionError:
        failed.append("internal consistency assert")
    return failed


@pytest.mark.parametrize("name", ["unmodified"] + sorted(MUTANTS))
def test_pins_reject_each_mutant(tmp_path, name):
    saved = oracle._lib
    try:
        oracle._lib = _compile(tmp_path, name, MUTANTS.get(name))
        failed = _battery()
    finally:
        oracle._lib = saved
    if name == "unmodified":
        assert failed == []
    else:
        assert failed, f"mutant {name} passed every pin"


# Python-level mutants of the skipped-product bound: a copy of
# oracle.skipped_bound with one planted error, swapped in for the pin battery
# of tests/test_oracle_bound.py.
BOUND_MUTANTS = {
    "bound_sums_every_candidate": ("term = np.where(is_kept, 0.0, na * nb)", "term = na * nb"),
    "bound_inverted_is_kept": ("is_kept = np.isin(ck, kk)", "is_kept = ~np.isin(ck, kk)"),
    "bound_squared_norms": ("na = np.sqrt(A.sq[", "na = (A.sq["),
    "bound_sum_not_squares": ("return float(np.sqrt(np.sum(beta * beta)))", "return float(np.sum(beta))"),
}


def _bound_mutant(mutation):
    import inspect
    import textwrap

    src = textwrap.dedent(inspect.getsource(oracle.skipped_bound))
    old, new = mutation
    assert src.count(old) == 1, old
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns["skipped_bound"]


@pytest.mark.parametrize("name", ["unmodified"] + sorted(BOUND_MUTANTS))
def test_bound_pins_reject_each_mutant(monkeypatch, name):
    from test_oracle_bound import bound_battery

    if name != "unmodified":
        monkeypatch.setattr(oracle, "skipped_bound", _bound_mutant(BOUND_MUTANTS[name]))
    failed = bound_battery()
    if name == "unmodified":
        assert failed == []
    else:
        assert failed, f"mutant {name} passed every pin of the bound"
