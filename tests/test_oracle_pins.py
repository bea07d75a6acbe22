"""Pins for the CPU oracle: what the paper and plain mathematics fix."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import literal

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pair(n, alpha=0.15, kind=synth.KIND_1D, seeds=(3, 4)):
    A = synth.dense(synth.DecayParams(n=n, kind=kind, alpha=alpha, seed=seeds[0]))
    B = synth.dense(synth.DecayParams(n=n, kind=kind, alpha=alpha, seed=seeds[1]))
    return A, B


# ---------------------------------------------------------------- norms (Sec. 2)
def test_leaf_norm_closed_forms():
    for bs in (1, 4, 32, 64):
        ones = np.ones((1, bs, bs))
        assert oracle.leaf_sqnorms(ones)[0] == bs * bs
        assert oracle.leaf_sqnorms(ones * 0.5)[0] == bs * bs * 0.25
        single = np.zeros((1, bs, bs))
        single[0, bs - 1, 0] = -3.0
        assert oracle.leaf_sqnorms(single)[0] == 9.0


def test_pairwise_sum_against_exactly_rounded_sum():
    rng = np.random.default_rng(2)
    for _ in range(20):
        x = rng.standard_normal(4096) * np.exp(rng.uniform(-20, 5, 4096))
        ref = math.fsum(float(v) * float(v) for v in x)
        got = oracle.leaf_sqnorms(x.reshape(1, 64, 64))[0]
        assert abs(got - ref) <= 1e-14 * ref


def test_norm_recursion_identity():
    """||A^t||^2 = sum of the four children's squared norms; the root is ||A||_F^2."""
    A, _ = _pair(200)
    M = oracle.from_dense(A, 8)
    grids, _ = oracle.tree_norms(M)
    ref = math.fsum(float(v) * float(v) for v in A.ravel())
    assert abs(grids[0][0, 0] - ref) <= 1e-13 * ref
    for t in range(M.L):
        ch = grids[t + 1]
        for I in range(1 << t):
            for J in range(1 << t):
                kids = [ch[2 * I + a, 2 * J + b] for a in (0, 1) for b in (0, 1)]
                if all(v < 0 for v in kids):
                    assert grids[t][I, J] == -1.0
                else:
                    s = 0.0
                    for v in kids:
                        if v >= 0:
                            s += v
                    assert grids[t][I, J] == s


def test_null_leaves_are_the_all_zero_blocks():
    A, _ = _pair(300, alpha=0.3)
    bs = 16
    M = oracle.from_dense(A, bs)
    nb = -(-300 // bs)
    pad = np.zeros((nb * bs, nb * bs))
    pad[:300, :300] = A
    expect = {(I, J) for I in range(nb) for J in range(nb)
              if pad[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs].any()}
    assert set(zip(M.bi.tolist(), M.bj.tolist())) == expect
    assert np.array_equal(oracle.to_dense(M), A)
    assert len(expect) < nb * nb  # decay leaves null blocks


# ------------------------------------------------------------ kept set (Alg. 1)
@pytest.mark.parametrize("bs", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("mode", [oracle.TRUNCATE, oracle.SPAMM, oracle.COMBINED])
def test_recursive_equals_flat_equals_literal(bs, mode):
    A, B = _pair(64, alpha=0.2)
    LA, LB = oracle.from_dense(A, bs), oracle.from_dense(B, bs)
    for tau in (0.0, 1e-9, 1e-5, 1e-3, 1e-1):
        if mode != oracle.SPAMM:
            LA_, LB_ = oracle.truncate_block(LA, tau), oracle.truncate_block(LB, tau)
        else:
            LA_, LB_ = LA, LB
        flat = oracle.kept_flat(LA_, LB_, tau, mode)
        rec = oracle.kept_recursive(LA_, LB_, tau, mode)
        assert np.array_equal(flat, rec)
        if mode == oracle.SPAMM:
            _, kl = literal.spamm_literal(A, B, tau, bs)
            assert np.array_equal(flat, oracle._sort_ijk(np.array(kl, np.int32).reshape(-1, 3)))


def test_tau_zero_keeps_every_nonnull_pair_and_huge_tau_keeps_none():
    A, B = _pair(256, alpha=0.1)
    LA, LB = oracle.from_dense(A, 16), oracle.from_dense(B, 16)
    k0 = oracle.kept_flat(LA, LB, 0.0, oracle.SPAMM)
    # closed-form count: sum over k of (#A leaves in block column k) x (#B leaves in block row k)
    cnt = sum(int(np.sum(LA.bj == k)) * int(np.sum(LB.bi == k)) for k in range(1 << LA.L))
    assert len(k0) == cnt
    assert np.array_equal(k0, oracle.kept_flat(LA, LB, 0.0, oracle.TRUNCATE))
    big = float(np.sqrt(LA.sq.max()) * np.sqrt(LB.sq.max())) * 1.0001
    assert len(oracle.kept_flat(LA, LB, big, oracle.SPAMM)) == 0


def test_kept_sets_are_nested_in_tau_and_combined_is_inside_both():
    A, B = _pair(256, alpha=0.1)
    LA, LB = oracle.from_dense(A, 8), oracle.from_dense(B, 8)
    key = lambda t: set(map(tuple, t.tolist()))
    prev = None
    for tau in (1e-12, 1e-9, 1e-6, 1e-3, 1e-1):
        s = key(oracle.kept_flat(LA, LB, tau, oracle.SPAMM))
        if prev is not None:
            assert s <= prev
        prev = s
        At, Bt = oracle.truncate_block(LA, tau), oracle.truncate_block(LB, tau)
        comb = key(oracle.kept_flat(At, Bt, tau, oracle.COMBINED))
        trunc = key(oracle.kept_flat(At, Bt, tau, oracle.TRUNCATE))
        assert comb <= s and comb <= trunc


def test_structural_examples_of_section_4_4():
    """Equations (nonoptimal_MM) and (nonoptimal_MM2): the predictor gives the
    exact output structure although no input is empty."""
    with open(os.path.join(GOLDEN, "nonoptimal_mm.json")) as f:
        gold = json.load(f)
    bs = 4
    rng = np.random.default_rng(9)
    for case in gold["cases"]:
        A = np.zeros((2 * bs, 2 * bs))
        B = np.zeros((2 * bs, 2 * bs))
        for I in range(2):
            for J in range(2):
                if case["A"][I][J]:
                    A[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs] = rng.uniform(-1, 1, (bs, bs))
                if case["B"][I][J]:
                    B[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs] = rng.uniform(-1, 1, (bs, bs))
        LA, LB = oracle.from_dense(A, bs), oracle.from_dense(B, bs)
        C, ikj = oracle.multiply(LA, LB, 0.0, oracle.SPAMM)
        pattern = [[0, 0], [0, 0]]
        for i, j in zip(C.bi.tolist(), C.bj.tolist()):
            pattern[i][j] = 1
        assert pattern == case["C"], case["name"]
        terms = {}
        for i, k, j in ikj.tolist():
            terms.setdefault(f"{i},{j}", []).append([i, k, k, j])
        assert terms == case["C_terms"]
        for key, prods in case["C_terms"].items():
            i, j = map(int, key.split(","))
            ref = sum(A[p[0] * bs:(p[0] + 1) * bs, p[1] * bs:(p[1] + 1) * bs]
                      @ B[p[2] * bs:(p[2] + 1) * bs, p[3] * bs:(p[3] + 1) * bs] for p in prods)
            got = C.data[[q for q in range(C.m) if (C.bi[q], C.bj[q]) == (i, j)][0]]
            assert np.allclose(got, ref, rtol=1e-14, atol=1e-15)


# ---------------------------------------------------------------- the product
@pytest.mark.parametrize("bs", [1, 4, 16, 32, 256])
def test_tau_zero_is_the_dense_product(bs):
    n = 300 if bs == 256 else (130 if bs > 1 else 48)  # 300: two ragged 256-leaves per side
    A, B = _pair(n, alpha=0.05)
    C, _ = oracle.multiply(oracle.from_dense(A, bs), oracle.from_dense(B, bs), 0.0, oracle.SPAMM)
    ref = A @ B
    textbook = np.empty_like(ref)
    oracle._load().orc_dense_product(n, oracle._p(np.ascontiguousarray(A)), oracle._p(np.ascontiguousarray(B)),
                                     oracle._p(textbook))
    got = oracle.to_dense(C)
    scale = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(got - ref) <= 1e-13 * scale + 1e-300)
    assert np.all(np.abs(got - textbook) <= 1e-13 * scale + 1e-300)


def test_element_form_of_theorem_2():
    """bs = 1: C_ij = sum_k chi_ikj, chi = a_ik b_kj if |a_ik||b_kj| >= tau else 0."""
    A, B = _pair(40, alpha=0.1)
    for tau in (1e-6, 1e-3, 5e-2):
        C, _ = oracle.multiply(oracle.from_dense(A, 1), oracle.from_dense(B, 1), tau, oracle.SPAMM)
        mask = (np.abs(A)[:, :, None] * np.abs(B)[None, :, :]) >= tau
        ref = np.einsum("ik,kj,ikj->ij", A, B, mask)
        assert np.allclose(oracle.to_dense(C) if C.m else 0 * A, ref, rtol=1e-13, atol=1e-16)


def test_truncmul_element_rule_is_theorem_1():
    """Element rule: C~ = A~ B~ with a -> 0 iff |a| < tau (eq. truncated_matrices)."""
    A, B = _pair(96, alpha=0.1)
    for bs in (1, 8, 32):
        for tau in (1e-6, 1e-3, 3e-2):
            C, _ = oracle.multiply(oracle.from_dense(A, bs), oracle.from_dense(B, bs), tau, oracle.TRUNCATE,
                                   rule="element")
            At = np.where(np.abs(A) < tau, 0.0, A)
            Bt = np.where(np.abs(B) < tau, 0.0, B)
            ref = At @ Bt
            got = oracle.to_dense(C) if C.m else np.zeros_like(A)
            assert np.all(np.abs(got - ref) <= 1e-13 * (np.abs(At) @ np.abs(Bt)) + 1e-300)


def test_complement_identity():
    """Kept plus skipped sub-products reassemble the exact product."""
    A, B = _pair(200, alpha=0.08)
    LA, LB = oracle.from_dense(A, 8), oracle.from_dense(B, 8)
    for tau in (1e-8, 1e-4, 1e-2):
        kept = oracle.kept_flat(LA, LB, tau, oracle.SPAMM)
        allp = oracle.kept_flat(LA, LB, 0.0, oracle.SPAMM)
        ks = set(map(tuple, kept.tolist()))
        dropped = np.array([t for t in allp.tolist() if tuple(t) not in ks], np.int32).reshape(-1, 3)
        Ck = oracle.to_dense(oracle.product(LA, LB, kept))
        Cd = oracle.to_dense(oracle.product(LA, LB, dropped)) if len(dropped) else 0.0
        assert np.allclose(Ck + Cd, A @ B, rtol=0, atol=1e-13 * np.abs(A).max() * np.abs(B).max() * 200)


@pytest.mark.parametrize("mode", ["truncate", "spamm", "combined"])
@pytest.mark.parametrize("rule", ["block", "element"])
def test_error_below_skipped_bound(mode, rule):
    A, B = _pair(256, alpha=0.06, kind=synth.KIND_1D)
    LA, LB = oracle.from_dense(A, 16), oracle.from_dense(B, 16)
    Cx = oracle.exact(LA, LB)
    for tau in (1e-8, 1e-5, 1e-3):
        C, _ = oracle.multiply(LA, LB, tau, oracle.MODES[mode], rule)
        err = oracle.error(Cx, C)
        bound = oracle.skipped_bound(LA, LB, tau, oracle.MODES[mode], rule)
        slack = 1e-13 * np.sqrt(np.sum((np.abs(A) @ np.abs(B)) ** 2))
        assert err <= bound + slack
        if mode != "truncate":
            assert bound > 0


def test_error_function_closed_forms():
    A, B = _pair(100, alpha=0.2)
    X, Y = oracle.from_dense(A, 8), oracle.from_dense(B, 8)
    assert oracle.error(X, X) == 0.0
    ref = math.sqrt(math.fsum(float(v) ** 2 for v in (A - B).ravel()))
    assert abs(oracle.error(X, Y) - ref) <= 1e-13 * ref
    Z = oracle.LeafMatrix(100, 8, np.zeros(0), np.zeros(0), np.zeros((0, 8, 8)))
    assert abs(oracle.error(X, Z) - oracle.frob_norm(X)) <= 1e-14 * oracle.frob_norm(X)
    assert abs(oracle.frob_norm(X) - np.linalg.norm(A)) <= 1e-13 * np.linalg.norm(A)


def test_single_leaf_matrix_takes_the_leaf_test():
    """n <= bs: the one leaf pair is tested like every other leaf pair."""
    A, B = _pair(20, alpha=0.3)
    LA, LB = oracle.from_dense(A, 32), oracle.from_dense(B, 32)
    assert LA.L == 0 and LA.m == 1
    prod = np.sqrt(LA.sq[0]) * np.sqrt(LB.sq[0])
    for tau, expect in ((prod * 0.999, 1), (prod * 1.001, 0)):
        for f in (oracle.kept_flat, oracle.kept_recursive):
            assert len(f(LA, LB, tau, oracle.SPAMM)) == expect
        _, kl = literal.spamm_literal(A, B, tau, 32)
        assert len(kl) == expect
    assert len(oracle.kept_recursive(LA, LB, prod * 2, oracle.TRUNCATE)) == 1


# ---------------------------------------------------------------- error-controlled truncation
def test_error_controlled_truncation_is_the_largest_admissible_drop():
    """Brute force over every subset of a small leaf set: the rule drops the
    largest number of leaves whose squared norms sum to <= tau^2 (dropping
    the smallest first is optimal for the count), and ||M - M~||_F <= tau."""
    import itertools
    rng = np.random.default_rng(7)
    for trial in range(40):
        m = int(rng.integers(1, 9))
        bs = 2
        data = rng.standard_normal((m, bs, bs)) * np.exp(rng.uniform(-3, 1, (m, 1, 1)))
        M = oracle.from_leaves(16, bs, np.arange(m), np.arange(m), data)
        tau = float(np.sqrt(np.sum(M.sq)) * rng.uniform(0.0, 1.1))
        T = oracle.truncate(M, tau, "error")
        dropped = M.m - T.m
        best = max(len(c) for r in range(m + 1) for c in itertools.combinations(range(m), r)
                   if np.sum(M.sq[list(c)]) <= tau * tau)
        assert dropped == best
        assert oracle.error(M, T) <= tau * (1 + 1e-15)


def test_error_controlled_truncation_edges_and_nesting():
    p = synth.lattice_3d(1024, alpha=1.0, seed=3)
    M = oracle.from_dense(synth.dense(p), 32)
    assert oracle.truncate(M, 0.0, "error").m == M.m
    assert oracle.truncate(M, oracle.frob_norm(M) * (1 + 1e-12), "error").m == 0
    prev = M.m
    for tau in [1e-12, 1e-9, 1e-6, 1e-3, 1e-1]:
        T = oracle.truncate(M, tau, "error")
        assert T.m <= prev and oracle.error(M, T) <= tau
        prev = T.m
    # equal norms fall in Morton order: identical leaves, budget for exactly two
    one = np.ones((4, 2, 2))
    E = oracle.from_leaves(8, 2, [1, 0, 1, 0], [1, 1, 0, 0], one)
    T = oracle.truncate(E, np.sqrt(8.0), "error")
    assert sorted(zip(T.bi.tolist(), T.bj.tolist())) == [(1, 0), (1, 1)]
