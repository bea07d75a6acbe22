"""Purification-chain operations on the GPU (spamm_add, spamm_identity,
spamm_trace, the SP2 and squaring chains) against the oracle chain."""
import numpy as np
import pytest

import oracle
import synth
from oracle import chain as ochain

pytestmark = pytest.mark.gpu


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


def _pair(S, ctx, n, bs, fill, seeds):
    out = []
    for sd in seeds:
        bi, bj, d = synth.block_sparse(n, bs, fill, seed=sd)
        out.append((S.spamm_from_blocks(ctx, n, bs, bi, bj, d), oracle.from_leaves(n, bs, bi, bj, d)))
    return out


@pytest.mark.parametrize("n,bs", [(1000, 32), (2048, 64)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (2.0, -1.0), (-0.37, 1.9)])
def test_add_matches_oracle_bitwise(S, ctx, n, bs, alpha, beta):
    (GX, OX), (GY, OY) = _pair(S, ctx, n, bs, 0.3, (1, 2))
    GZ = S.spamm_add(ctx, alpha, GX, beta, GY)
    OZ = ochain.add(alpha, OX, beta, OY)
    bi, bj, d, sq = S.spamm_to_blocks(ctx, GZ)
    key = lambda i, j: np.asarray(i, np.int64) * 65536 + np.asarray(j, np.int64)
    og = np.argsort(key(bi, bj)), np.argsort(key(OZ.bi, OZ.bj))
    assert np.array_equal(key(bi, bj)[og[0]], key(OZ.bi, OZ.bj)[og[1]])
    assert np.array_equal(d[og[0]], OZ.data[og[1]])
    assert np.allclose(sq[og[0]], OZ.sq[og[1]], rtol=1e-14, atol=0)
    assert S.spamm_frob_norm(ctx, GZ) == pytest.approx(oracle.frob_norm(OZ), rel=1e-13)


def test_add_edge_cases(S, ctx):
    (GX, OX), = _pair(S, ctx, 512, 32, 0.5, (3,))
    assert S.spamm_add(ctx, 1.0, GX, -1.0, GX).info()["nleaves"] == 0
    E = S.spamm_add(ctx, 1.0, GX, -1.0, GX)
    assert S.spamm_add(ctx, 1.0, E, 1.0, E).info()["nleaves"] == 0
    Z = S.spamm_add(ctx, 1.0, E, 2.0, GX)
    assert np.array_equal(S.spamm_to_dense(ctx, Z), 2.0 * oracle.to_dense(OX))
    G64, _ = _pair(S, ctx, 512, 64, 0.5, (4,))[0]
    with pytest.raises(S.SpammError):
        S.spamm_add(ctx, 1.0, GX, 1.0, G64)


@pytest.mark.parametrize("n,bs", [(300, 32), (4096, 64), (1000, 128)])
def test_identity_and_trace(S, ctx, n, bs):
    I = S.spamm_identity(ctx, n, bs)
    assert np.array_equal(S.spamm_to_dense(ctx, I), np.eye(n))
    assert S.spamm_trace(ctx, I) == n
    (GX, OX), = _pair(S, ctx, n, bs, 0.4, (5,))
    assert S.spamm_trace(ctx, GX) == pytest.approx(ochain.trace(OX), rel=1e-13, abs=1e-12)


def test_sp2_chain_matches_oracle(S, ctx):
    from paper_1906_08148_gb300 import chain
    p = synth.model_1d(1024, alpha=0.05, seed=1)
    F = synth.dense(p)
    w = np.linalg.eigvalsh(F)
    lo, hi = 256, 768
    n_occ = lo + int(np.argmax(np.diff(w[lo:hi + 1]))) + 1
    bound = synth.spectral_bound(p)
    tau, iters = 1e-10, 30
    GX, gh = chain.sp2(ctx, S.spamm_from_dense(ctx, F, 32), n_occ, bound, tau, "spamm", "fp64", iters)
    OX, oh = ochain.sp2(oracle.from_dense(F, 32), n_occ, bound, tau, oracle.SPAMM, iters)
    assert [h["branch"] for h in gh] == [h["branch"] for h in oh]
    for g, o in zip(gh, oh):
        assert g["trace"] == pytest.approx(o["trace"], rel=1e-11)
        assert g["idempotency"] == pytest.approx(o["idempotency"], rel=1e-8, abs=1e-12)
    D, R = S.spamm_to_dense(ctx, GX), oracle.to_dense(OX)
    assert np.linalg.norm(D - R) <= 1e-10 * np.linalg.norm(R)
    # (convergence to the spectral projector itself is pinned on the oracle, tests/test_oracle_chain.py)


@pytest.mark.parametrize("prec", ["fp64", "fp16_scaled"])
def test_square_chain_matches_oracle(S, ctx, prec):
    from paper_1906_08148_gb300 import chain
    p = synth.lattice_3d(4096, alpha=1.0, seed=1)
    bound = synth.spectral_bound(p)
    ps = synth.DecayParams(n=p.n, kind=p.kind, alpha=p.alpha, seed=p.seed, c=1.0 / bound)
    G0 = S.spamm_generate(ctx, ps, 64)
    X0 = oracle.from_dense(synth.dense(ps), 64)
    tau = 1e-8
    GX, gh = chain.square_chain(ctx, G0, 4, tau, "combined", prec)
    OX, on = ochain.square_chain(X0, 4, tau, oracle.COMBINED)
    D, R = S.spamm_to_dense(ctx, GX), oracle.to_dense(OX)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.linalg.norm(D - R) <= tol * np.linalg.norm(R), np.linalg.norm(D - R) / np.linalg.norm(R)
    assert gh[0]["n_kept"] == len(oracle.multiply(X0, X0, tau, oracle.COMBINED)[1])
    assert gh[-1]["frob"] == pytest.approx(on[-1], rel=1e-12 if prec == "fp64" else 1e-5)


def _insulator(S, ctx, n, delta, tau, bs=64):
    """F = V + D of the gapped two-sublattice insulator, V generated with its
    leaves below 2 b tau dropped (X0 = (bI - F) / (2b) then keeps the leaves
    of norm >= tau); both sides start from the same leaves."""
    p = synth.lattice_3d(n, alpha=1.0, seed=1)
    bound = delta + synth.spectral_bound(p)
    di, dj, dd, n_occ = synth.onsite_blocks(n, bs, delta)
    V = S.spamm_generate(ctx, p, bs, 2.0 * bound * tau)
    D = S.spamm_from_blocks(ctx, n, bs, di, dj, dd)
    GF = S.spamm_add(ctx, 1.0, V, 1.0, D)
    vi, vj, vd, _ = S.spamm_to_blocks(ctx, V)
    OF = ochain.add(1.0, oracle.from_leaves(n, bs, vi, vj, vd), 1.0, oracle.from_leaves(n, bs, di, dj, dd))
    V.close()
    D.close()
    return GF, OF, n_occ, bound


@pytest.mark.parametrize("prec", ["fp64", "fp16_scaled", "bf16_split4"])
def test_sp2_insulator_matches_oracle(S, ctx, prec):
    """Once X is a projector to within the truncation error the trace rule is
    a tie and either branch is right, so the states are compared over the
    iterations before that (k of them, while ||X - X^2||_F > 1e-3), and the
    converged chains by their trace."""
    from paper_1906_08148_gb300 import chain
    n, delta, tau, iters = 2048, 6.0, 1e-7, 22
    GF, OF, n_occ, bound = _insulator(S, ctx, n, delta, tau)
    OXc, oh = ochain.sp2(OF, n_occ, bound, tau, oracle.COMBINED, iters)
    assert ochain.trace(OXc) == pytest.approx(n_occ, rel=1e-6)
    k = next(i for i, o in enumerate(oh) if o["idempotency"] <= 1e-3)
    assert k >= 6
    GX, gh = chain.sp2(ctx, GF, n_occ, bound, tau, "combined", prec, k)
    OX, _ = ochain.sp2(OF, n_occ, bound, tau, oracle.COMBINED, k)
    assert [g["branch"] for g in gh] == [o["branch"] for o in oh[:k]]
    D, R = S.spamm_to_dense(ctx, GX), oracle.to_dense(OX)
    # each product adds the form's arithmetic error (4-slice: a few 1e-10, FP16:
    # ~1e-6 relative) and SP2 carries the occupied-unoccupied part of an error
    # forward unchanged, so the chains part by up to k times that
    tol = 1e-12 if prec == "fp64" else (k * 5e-10 if prec == "bf16_split4" else k * 5e-6)
    assert np.linalg.norm(D - R) <= tol * np.linalg.norm(R), np.linalg.norm(D - R) / np.linalg.norm(R)
    GXc, _ = chain.sp2(ctx, GF, n_occ, bound, tau, "combined", prec, iters)
    assert S.spamm_trace(ctx, GXc) == pytest.approx(n_occ, rel=1e-6)


def test_sp2_probe_rows_equal_the_oracle_rows(S, ctx):
    """The bench's sampled-row check of a chain product (exact rows, method
    rows in FP64, the form's rows) against the oracle's product rows."""
    import bench
    n, delta, tau = 2048, 6.0, 1e-7
    GF, OF, n_occ, bound = _insulator(S, ctx, n, delta, tau)
    I = S.spamm_identity(ctx, n, 64)
    GX = S.spamm_add(ctx, -0.5 / bound, GF, 0.5, I)
    OX = ochain.add(-0.5 / bound, OF, 0.5, ochain.identity(n, 64))
    GX2 = S.spamm_multiply(ctx, GX, GX, tau, "combined", "fp16_scaled")
    rows = np.array([3, 17], np.int32)
    ea, ef, ex = bench.sp2_probe_rows(S, ctx, GX, GX2, rows, tau, n, 64)
    E = oracle.to_dense(oracle.exact(OX, OX))
    M = oracle.to_dense(oracle.multiply(OX, OX, tau, oracle.COMBINED)[0])
    T = S.spamm_to_dense(ctx, GX2)
    r = np.concatenate([np.arange(64 * i, 64 * i + 64) for i in rows])
    assert ex == pytest.approx(np.sum(E[r] ** 2), rel=1e-12)
    assert ea == pytest.approx(np.sum((E[r] - M[r]) ** 2), rel=1e-6, abs=1e-30)
    assert ef == pytest.approx(np.sum((M[r] - T[r]) ** 2), rel=1e-3, abs=1e-30)
