"""Tensor-core precision forms (BF16 error-free splits with 3 and 4 slices,
FP16 per-leaf scaled) against the FP64 oracle on the same kept set.

Tolerances are the element-wise bounds derived from each form's arithmetic
in tests/tcbound.py.  The Frobenius error against the oracle is also
reported and checked to stay below the method's own truncation error at the
same tau (Theorems 1-3 give that error; Section 5 compares methods at equal
accuracy), on the full product at n = 4096 and on windows of output leaves
at n = 16384 for tau down to 1e-8.  Integer inputs whose split is exact check
that the slice products of index sum 0 (and 1 for 4 slices) accumulate
exactly and that the two-float epilogue loses nothing."""
import numpy as np
import pytest

import oracle
import synth
import tcbound
from oracle import sampled

pytestmark = pytest.mark.gpu

TC = ["bf16_split", "bf16_split4", "fp16_scaled"]


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm
    return spamm


@pytest.fixture(scope="module")
def ctx(S):
    return S.Context(0)


def _check(S, ctx, GA, GB, MA, MB, tau, mode, prec):
    C = S.spamm_multiply(ctx, GA, GB, tau, mode, prec)
    ref, ikj = oracle.multiply(MA, MB, tau, oracle.MODES[mode])
    At = MA if mode == "spamm" else oracle.truncate_block(MA, tau)
    Bt = MB if mode == "spamm" else oracle.truncate_block(MB, tau)
    bnd = tcbound.bound(prec, At, Bt, ikj, ref)
    bi, bj, pay, _ = S.spamm_to_blocks(ctx, C)
    key = lambda r, c: (int(r), int(c))
    gpu = {key(r, c): pay[q] for q, (r, c) in enumerate(zip(bi, bj))}
    assert set(gpu) == {key(r, c) for r, c in zip(ref.bi, ref.bj)}
    num = 0.0
    worst = 0.0
    for q in range(ref.m):
        d = np.abs(gpu[key(ref.bi[q], ref.bj[q])] - ref.data[q])
        worst = max(worst, float(np.max(d / bnd[q])))
        num += float(np.sum(d ** 2))
    rel = np.sqrt(num) / max(oracle.frob_norm(ref), 1e-300)
    return worst, rel, ref


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("mode,bs", [("spamm", 64), ("combined", 64), ("truncate", 64), ("combined", 128)])
def test_tensor_forms_within_derived_bound(S, ctx, prec, mode, bs):
    pa, pb = synth.lattice_3d(4096, alpha=0.9, seed=1), synth.lattice_3d(4096, alpha=0.9, seed=2)
    GA, GB = S.spamm_generate(ctx, pa, bs), S.spamm_generate(ctx, pb, bs)
    MA, MB = oracle.from_dense(synth.dense(pa), bs), oracle.from_dense(synth.dense(pb), bs)
    for tau in (1e-4, 1e-6):
        worst, rel, _ = _check(S, ctx, GA, GB, MA, MB, tau, mode, prec)
        print(f"{prec} {mode} bs={bs} tau={tau}: rel Frobenius error vs FP64 oracle {rel:.3e}, "
              f"worst/bound {worst:.3f}")
        assert worst <= 1.0


@pytest.mark.parametrize("prec", TC)
def test_tensor_error_below_truncation_error(S, ctx, prec):
    """Section 5's accuracy target: the arithmetic error stays below the
    method's own truncation error ||AB - C||_F at the same tau."""
    pa, pb = synth.lattice_3d(4096, alpha=0.9, seed=1), synth.lattice_3d(4096, alpha=0.9, seed=2)
    GA, GB = S.spamm_generate(ctx, pa, 64), S.spamm_generate(ctx, pb, 64)
    MA, MB = oracle.from_dense(synth.dense(pa), 64), oracle.from_dense(synth.dense(pb), 64)
    exact = oracle.exact(MA, MB)
    for tau in (1e-3, 1e-4):
        _, rel, ref = _check(S, ctx, GA, GB, MA, MB, tau, "combined", prec)
        trunc = oracle.error(exact, ref)
        arith = rel * oracle.frob_norm(ref)
        print(f"{prec} tau={tau}: arithmetic error {arith:.3e} vs truncation error {trunc:.3e}")
        assert arith < trunc


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("bs", [64, 128])
def test_single_leaf_product_layout(S, ctx, prec, bs):
    """One leaf pair with distinct entries: any operand layout, tile or
    descriptor mistake shows up as an O(1) error."""
    rng = np.random.default_rng(11)
    A = rng.uniform(-1, 1, (bs, bs))
    B = rng.uniform(-1, 1, (bs, bs))
    GA, GB = S.spamm_from_dense(ctx, A, bs), S.spamm_from_dense(ctx, B, bs)
    C = S.spamm_to_dense(ctx, S.spamm_multiply(ctx, GA, GB, 0.0, "spamm", prec))
    MA, MB = oracle.from_dense(A, bs), oracle.from_dense(B, bs)
    ref, ikj = oracle.multiply(MA, MB, 0.0, oracle.SPAMM)
    bnd = tcbound.bound(prec, MA, MB, ikj, ref)[0]
    assert np.all(np.abs(C - A @ B) <= bnd)


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("cols", ["odd", "even", "alternating", "all"])
def test_steps_with_one_b_leaf(S, ctx, prec, cols):
    """Quads of 64-leaves whose steps need only one of their two B leaves
    (kept products in one output column): the other leaf is not loaded, so
    its half of the stage holds an earlier step's terms, which must reach
    only discarded quadrants.  B's leaf columns only odd (the second leaf of
    every pair), only even, alternating with k (both kinds within one quad),
    and all present.
    Integer entries: the BF16 splits are exact (C = AB bit for bit); FP16
    within its derived bound."""
    rng = np.random.default_rng(23)
    bs, nl = 64, 6
    n = bs * nl
    A = rng.integers(-255, 256, (n, n)).astype(np.float64)
    B = rng.integers(-255, 256, (n, n)).astype(np.float64)
    for kb in range(nl):
        for jb in range(nl):
            keep = {"odd": jb % 2 == 1, "even": jb % 2 == 0, "alternating": jb % 2 == kb % 2, "all": True}[cols]
            if not keep:
                B[kb * bs:(kb + 1) * bs, jb * bs:(jb + 1) * bs] = 0.0
    GA, GB = S.spamm_from_dense(ctx, A, bs), S.spamm_from_dense(ctx, B, bs)
    C = S.spamm_to_dense(ctx, S.spamm_multiply(ctx, GA, GB, 0.0, "spamm", prec))
    if prec != "fp16_scaled":
        assert np.array_equal(C, A @ B)
    else:
        MA, MB = oracle.from_dense(A, bs), oracle.from_dense(B, bs)
        ref, ikj = oracle.multiply(MA, MB, 0.0, oracle.SPAMM)
        bnd = oracle.to_dense(oracle.LeafMatrix(n, bs, ref.bi, ref.bj, tcbound.bound(prec, MA, MB, ikj, ref)))
        assert np.all(np.abs(C - A @ B) <= bnd)


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("bs", [64, 128])
def test_tensor_ragged_and_empty(S, ctx, prec, bs):
    rng = np.random.default_rng(5)
    n = 200 if bs == 64 else 330  # ragged: 4 x 4 (3 x 3) leaves, the last ones padded
    A = rng.uniform(-1, 1, (n, n)) * np.exp(-0.05 * np.abs(np.subtract.outer(np.arange(n), np.arange(n))))
    GA = S.spamm_from_dense(ctx, A, bs)
    C = S.spamm_to_dense(ctx, S.spamm_multiply(ctx, GA, GA, 0.0, "spamm", prec))
    MA = oracle.from_dense(A, bs)
    ref, ikj = oracle.multiply(MA, MA, 0.0, oracle.SPAMM)
    bnd = oracle.to_dense(oracle.LeafMatrix(n, bs, ref.bi, ref.bj, tcbound.bound(prec, MA, MA, ikj, ref)))
    assert np.all(np.abs(C - A @ A) <= bnd)
    E = S.spamm_multiply(ctx, GA, GA, 1e9, "spamm", prec)
    assert E.info()["nleaves"] == 0
    G32 = S.spamm_from_dense(ctx, A, 32)  # 32 x 32 leaves: FP64 only
    with pytest.raises(S.SpammError) as err:
        S.spamm_multiply(ctx, G32, G32, 0.0, "spamm", prec)
    assert err.value.status == S.E_UNSUPPORTED


def test_tensor_forms_deterministic(S, ctx):
    p = synth.lattice_3d(4096, alpha=0.7, seed=3)
    G = S.spamm_generate(ctx, p, 64)
    for prec in TC:
        outs = [S.spamm_to_blocks(ctx, S.spamm_multiply(ctx, G, G, 1e-6, "combined", prec))[2] for _ in range(2)]
        assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", TC)
def test_power_of_two_scaling_is_exact(S, ctx, prec):
    """Scaling A by 2^-40 and B by 2^40 (exact in FP64, in range for FP32) gives
    bit for bit the same C: both forms only shift exponents."""
    A, B = (synth.dense(synth.lattice_3d(4096, alpha=0.9, seed=s)) for s in (1, 2))
    tau = 1e-6
    ref = S.spamm_to_dense(ctx, S.spamm_multiply(ctx, S.spamm_from_dense(ctx, A, 64), S.spamm_from_dense(ctx, B, 64),
                                                 tau, "spamm", prec))
    As, Bs = np.ldexp(A, -40), np.ldexp(B, 40)
    got = S.spamm_to_dense(ctx, S.spamm_multiply(ctx, S.spamm_from_dense(ctx, As, 64), S.spamm_from_dense(ctx, Bs, 64),
                                                 tau, "spamm", prec))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec,amax", [("bf16_split", 255), ("bf16_split4", 65535)])
@pytest.mark.parametrize("bs", [64, 128])
def test_integer_inputs_are_exact(S, ctx, prec, amax, bs):
    """Integer A (|a| <= amax: one digit for the 3-slice split, two for the
    4-slice split) and integer B (|b| <= 255, one digit): the split is exact,
    every slice product of index sum 0 (and 1) sums over K = 64 to at most
    2^22 units of its grid, exact in its FP32 accumulator, the larger index
    sums are all zero, and the two-float sum over the four k leaves loses
    nothing: C equals A B bit for bit.  The all-maximal 3-slice case puts the
    first accumulator at 64 * 255^2 = 4,161,600, next to 2^22."""
    rng = np.random.default_rng(8)
    n = 4 * bs
    for A, B in ((rng.integers(-amax, amax + 1, (n, n)).astype(np.float64),
                  rng.integers(-255, 256, (n, n)).astype(np.float64)),
                 (np.full((n, n), float(amax)), np.full((n, n), 255.0))):
        GA, GB = S.spamm_from_dense(ctx, A, bs), S.spamm_from_dense(ctx, B, bs)
        C = S.spamm_to_dense(ctx, S.spamm_multiply(ctx, GA, GB, 0.0, "spamm", prec))
        assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("prec,taus", [("bf16_split4", (1e-6, 1e-7, 1e-8)), ("bf16_split", (1e-4, 1e-5)),
                                       ("fp16_scaled", (1e-4, 1e-5))])
def test_tensor_error_below_truncation_error_16384(S, ctx, prec, taus):
    """n = 16384 (32 x 32 x 16 lattice, alpha = 0.9, A != B), combined: on a
    window of output leaves (each form over the tau range its arithmetic
    serves: the 4-slice split down to 1e-8, the 3-slice split and FP16, whose
    errors are about 1.5e-7 of |C|, down to 1e-5) (block rows and columns [0, 8) plus the window
    around the middle of the index range), the form's deviation from the FP64
    oracle stays below the method's truncation error ||AB - C||_F there,
    the exact AB taken over every non-null k of the untruncated inputs."""
    n, alpha = 16384, 0.9
    pa, pb = synth.lattice_3d(n, alpha=alpha, seed=1), synth.lattice_3d(n, alpha=alpha, seed=2)
    GA, GB = S.spamm_generate(ctx, pa, 64), S.spamm_generate(ctx, pb, 64)
    for tau in taus:
        C = S.spamm_multiply(ctx, GA, GB, tau, "combined", prec)
        arith2 = trunc2 = 0.0
        for w0 in (0, 124):
            rows = range(w0, w0 + 8)
            A_rows, B_cols = sampled.window_inputs(pa, pb, 64, rows, rows)
            ref, ikj = sampled.window_product(A_rows, B_cols, tau, oracle.COMBINED)
            X = sampled.window_exact(A_rows, B_cols)
            At, Bt = oracle.truncate_block(A_rows, tau), oracle.truncate_block(B_cols, tau)
            bnd = tcbound.bound(prec, At, Bt, ikj, ref)
            gpu, found = S.spamm_gather_leaves(ctx, C, ref.bi, ref.bj)
            assert found.all()
            assert np.all(np.abs(gpu - ref.data) <= bnd)
            arith2 += float(np.sum((gpu - ref.data) ** 2))
            trunc2 += oracle.error(X, ref) ** 2
        arith, trunc = np.sqrt(arith2), np.sqrt(trunc2)
        print(f"{prec} n={n} tau={tau}: arithmetic error {arith:.3e} vs truncation error {trunc:.3e}")
        assert arith < trunc
        C.close()


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("bs", [64, 128])
def test_symmetric_square_shares_terms(S, ctx, prec, bs):
    """X times X for a symmetric X (the squarings of a purification chain):
    one set of operand terms serves both roles (B's leaf (k, j) uses the
    terms of leaf (j, k)); the output is bit-identical to building the B
    terms separately, and the plan holds fewer bytes.  A leaf set without
    every transpose falls back to separate terms."""
    p = synth.lattice_3d(4096, alpha=0.9, seed=4)
    X = S.spamm_generate(ctx, p, bs)
    tau = 1e-6
    shared, st1 = S.spamm_multiply(ctx, X, X, tau, "combined", prec, stats=True)
    pl1 = S.spamm_plan_create(ctx, X, X, tau, "combined", prec)
    X.set_symmetric(False)
    plain, st0 = S.spamm_multiply(ctx, X, X, tau, "combined", prec, stats=True)
    pl0 = S.spamm_plan_create(ctx, X, X, tau, "combined", prec)
    assert st1["terms_shared"] == 1 and st0["terms_shared"] == 0
    assert pl1.info()["plan_bytes"] < pl0.info()["plan_bytes"]
    a, b = S.spamm_to_blocks(ctx, shared), S.spamm_to_blocks(ctx, plain)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    # the mark on a leaf set that lacks a transpose: separate terms, the product A A
    rng = np.random.default_rng(9)
    D = np.zeros((4 * bs, 4 * bs))
    D[:bs, :bs] = rng.uniform(-1, 1, (bs, bs))
    D[bs:2 * bs, :bs] = rng.uniform(-1, 1, (bs, bs))  # leaf (1, 0) without (0, 1)
    G = S.spamm_from_dense(ctx, D, bs)
    G.set_symmetric(True)
    C, st = S.spamm_multiply(ctx, G, G, 0.0, "spamm", prec, stats=True)
    assert st["terms_shared"] == 0
    M = oracle.from_dense(D, bs)
    ref, ikj = oracle.multiply(M, M, 0.0, oracle.SPAMM)
    bnd = oracle.to_dense(oracle.LeafMatrix(4 * bs, bs, ref.bi, ref.bj, tcbound.bound(prec, M, M, ikj, ref)))
    assert np.all(np.abs(S.spamm_to_dense(ctx, C) - D @ D) <= bnd)


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("bs", [64, 128])
def test_output_norms_are_kernel_a_of_the_finished_leaves(S, ctx, prec, bs):
    """The finishing pass (kernel (d) of the tensor forms) stores each output
    leaf's squared norm in kernel (a)'s order: rebuilding the matrix from its
    own FP64 leaves gives the same norms bit for bit, and they agree with
    NumPy's sums of squares."""
    p = synth.lattice_3d(4096, alpha=0.9, seed=4)
    G = S.spamm_generate(ctx, p, bs)
    C = S.spamm_multiply(ctx, G, G, 1e-7, "combined", prec)
    bi, bj, pay, sq = S.spamm_to_blocks(ctx, C)
    R = S.spamm_from_blocks(ctx, 4096, bs, bi, bj, pay)
    _, _, pay2, sq2 = S.spamm_to_blocks(ctx, R)
    assert np.array_equal(pay, pay2)
    assert np.array_equal(sq, sq2)
    assert np.allclose(sq, np.sum(pay * pay, axis=(1, 2)), rtol=1e-13, atol=0)
    assert S.spamm_frob_norm(ctx, C) == pytest.approx(np.sqrt(np.sum(pay * pay)), rel=1e-13)
