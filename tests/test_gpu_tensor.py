"""Tensor-core precision forms (BF16 three-term split, FP16 per-leaf scaled)
against the FP64 oracle on the same kept set.

Tolerance, derived from the arithmetic (u = 2^-24, the FP32 unit roundoff):
each operand is represented by its terms to about 2^-24 relative (BF16 split,
>= 3 terms of 8 bits) or 2^-22 (FP16, 2 terms of 11 bits); every leaf product
is accumulated in FP32 over K = 64 and added into an FP32 register
accumulator once per kept leaf product.  With n_k kept products for output
leaf (i, j) and |A||B| the product of absolute values over the kept set:
    |C_tc - C_fp64|_ij <= (n_k + c) * 2^-e * (|A||B|)_ij
with (c, e) = (8, 22) for BF16 split and (16, 20) for FP16 scaled.  The
Frobenius error against the oracle is also reported and, where the method's
truncation error is larger, checked to be below it."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

BOUND = {"bf16_split": (8, 22), "fp16_scaled": (16, 20)}


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


def _abs(M):
    return oracle.LeafMatrix(M.n, M.bs, M.bi, M.bj, np.abs(M.data))


def _check(S, ctx, GA, GB, MA, MB, tau, mode, prec):
    C = S.spamm_multiply(ctx, GA, GB, tau, mode, prec)
    ref, ikj = oracle.multiply(MA, MB, tau, oracle.MODES[mode])
    At = MA if mode == "spamm" else oracle.truncate_block(MA, tau)
    Bt = MB if mode == "spamm" else oracle.truncate_block(MB, tau)
    absprod = oracle.product(_abs(At), _abs(Bt), ikj)
    bi, bj, pay, _ = S.spamm_to_blocks(ctx, C)
    key = lambda r, c: (int(r), int(c))
    gpu = {key(r, c): pay[q] for q, (r, c) in enumerate(zip(bi, bj))}
    assert set(gpu) == {key(r, c) for r, c in zip(ref.bi, ref.bj)}
    i, j = ikj[:, 0], ikj[:, 2]
    nk = {}
    for a, b in zip(i.tolist(), j.tolist()):
        nk[(a, b)] = nk.get((a, b), 0) + 1
    c0, e = BOUND[prec]
    num = 0.0
    worst = 0.0
    for q in range(ref.m):
        k = key(ref.bi[q], ref.bj[q])
        d = np.abs(gpu[k] - ref.data[q])
        bound = (nk[k] + c0) * 2.0 ** -e * absprod.data[q] + 1e-300
        worst = max(worst, float(np.max(d / bound)))
        num += float(np.sum((gpu[k] - ref.data[q]) ** 2))
    rel = np.sqrt(num) / max(oracle.frob_norm(ref), 1e-300)
    return worst, rel, ref


@pytest.mark.parametrize("prec", ["bf16_split", "fp16_scaled"])
@pytest.mark.parametrize("mode", ["spamm", "combined", "truncate"])
def test_tensor_forms_within_derived_bound(S, ctx, prec, mode):
    pa, pb = synth.lattice_3d(4096, alpha=0.9, seed=1), synth.lattice_3d(4096, alpha=0.9, seed=2)
    GA, GB = S.spamm_generate(ctx, pa, 64), S.spamm_generate(ctx, pb, 64)
    MA, MB = oracle.from_dense(synth.dense(pa), 64), oracle.from_dense(synth.dense(pb), 64)
    for tau in (1e-4, 1e-6):
        worst, rel, _ = _check(S, ctx, GA, GB, MA, MB, tau, mode, prec)
        print(f"{prec} {mode} tau={tau}: rel Frobenius error vs FP64 oracle {rel:.3e}, worst/bound {worst:.3f}")
        assert worst <= 1.0


@pytest.mark.parametrize("prec", ["bf16_split", "fp16_scaled"])
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


@pytest.mark.parametrize("prec", ["bf16_split", "fp16_scaled"])
def test_single_leaf_product_layout(S, ctx, prec):
    """One 64 x 64 leaf pair with distinct entries: any operand layout or
    descriptor mistake shows up as an O(1) error."""
    rng = np.random.default_rng(11)
    A = rng.uniform(-1, 1, (64, 64))
    B = rng.uniform(-1, 1, (64, 64))
    GA, GB = S.spamm_from_dense(ctx, A, 64), S.spamm_from_dense(ctx, B, 64)
    C = S.spamm_to_dense(ctx, S.spamm_multiply(ctx, GA, GB, 0.0, "spamm", prec))
    ref = A @ B
    c0, e = BOUND[prec]
    assert np.all(np.abs(C - ref) <= (1 + c0) * 2.0 ** -e * (np.abs(A) @ np.abs(B)))


@pytest.mark.parametrize("prec", ["bf16_split", "fp16_scaled"])
def test_tensor_ragged_and_empty(S, ctx, prec):
    rng = np.random.default_rng(5)
    n = 200  # ragged: 4 x 4 leaves, the last ones padded
    A = rng.uniform(-1, 1, (n, n)) * np.exp(-0.05 * np.abs(np.subtract.outer(np.arange(n), np.arange(n))))
    GA = S.spamm_from_dense(ctx, A, 64)
    C = S.spamm_to_dense(ctx, S.spamm_multiply(ctx, GA, GA, 0.0, "spamm", prec))
    c0, e = BOUND[prec]
    assert np.all(np.abs(C - A @ A) <= (4 + c0) * 2.0 ** -e * (np.abs(A) @ np.abs(A)))
    E = S.spamm_multiply(ctx, GA, GA, 1e9, "spamm", prec)
    assert E.info()["nleaves"] == 0
    G32 = S.spamm_from_dense(ctx, A, 32)
    with pytest.raises(S.SpammError) as err:
        S.spamm_multiply(ctx, G32, G32, 0.0, "spamm", prec)
    assert err.value.status == S.E_UNSUPPORTED


def test_tensor_forms_deterministic(S, ctx):
    p = synth.lattice_3d(4096, alpha=0.7, seed=3)
    G = S.spamm_generate(ctx, p, 64)
    for prec in ("bf16_split", "fp16_scaled"):
        outs = [S.spamm_to_blocks(ctx, S.spamm_multiply(ctx, G, G, 1e-6, "combined", prec))[2] for _ in range(2)]
        assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", ["bf16_split", "fp16_scaled"])
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
