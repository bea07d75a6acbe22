"""Pins for the purification-chain oracle (oracle/chain.py): addition,
identity and trace against dense arithmetic, SP2 against the spectral
projector from an eigendecomposition, repeated squaring against matrix
powers."""
import numpy as np
import pytest

import oracle
import synth
from oracle import chain


def _rand(n, bs, fill, seed):
    bi, bj, d = synth.block_sparse(n, bs, fill, seed=seed)
    return oracle.from_leaves(n, bs, bi, bj, d)


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (2.0, -1.0), (-0.37, 1.9), (0.0, 3.0)])
def test_add_is_the_dense_sum(alpha, beta):
    X, Y = _rand(300, 32, 0.3, 1), _rand(300, 32, 0.4, 2)
    Z = chain.add(alpha, X, beta, Y)
    want = alpha * oracle.to_dense(X) + beta * oracle.to_dense(Y)
    assert np.array_equal(oracle.to_dense(Z), want)
    # every stored leaf has a non-zero element, every non-zero block is stored
    nzb = {(i, j) for i in range(10) for j in range(10) if np.any(want[32 * i:32 * i + 32, 32 * j:32 * j + 32])}
    assert set(zip(Z.bi.tolist(), Z.bj.tolist())) == nzb
    assert np.allclose(Z.sq, np.sum(Z.data ** 2, axis=(1, 2)), rtol=1e-14, atol=0)


def test_add_cancellation_gives_the_empty_matrix():
    X = _rand(256, 32, 0.5, 3)
    assert chain.add(1.0, X, -1.0, X).m == 0
    assert chain.add(0.0, X, 0.0, X).m == 0


@pytest.mark.parametrize("n,bs", [(256, 32), (300, 32), (1000, 64)])
def test_identity_and_trace(n, bs):
    I = chain.identity(n, bs)
    assert np.array_equal(oracle.to_dense(I), np.eye(n))
    assert chain.trace(I) == n
    X = _rand(n, bs, 0.3, 4)
    assert chain.trace(X) == pytest.approx(np.trace(oracle.to_dense(X)), rel=1e-13, abs=1e-12)


def _gapped_occupation(F):
    w = np.linalg.eigvalsh(F)
    n = len(w)
    lo, hi = n // 4, 3 * n // 4
    k = lo + int(np.argmax(np.diff(w[lo:hi + 1])))  # largest gap between w[k] and w[k+1]
    return k + 1, w


def test_sp2_converges_to_the_spectral_projector():
    p = synth.model_1d(256, alpha=0.05, seed=1)
    F = synth.dense(p)
    n_occ, w = _gapped_occupation(F)
    FL = oracle.from_dense(F, 32)
    X, hist = chain.sp2(FL, n_occ, synth.spectral_bound(p), 0.0, oracle.SPAMM, 80)
    v = np.linalg.eigh(F)[1][:, :n_occ]
    P = v @ v.T
    D = oracle.to_dense(X)
    assert np.linalg.norm(D - P) <= 1e-8 * np.sqrt(n_occ)
    assert chain.trace(X) == pytest.approx(n_occ, abs=1e-8)
    assert hist[-1]["idempotency"] <= 1e-10
    # both branches are used, and idempotency eventually decreases monotonically
    assert {h["branch"] for h in hist} == {"square", "2x-x2"}


def test_square_chain_is_the_matrix_power():
    p = synth.lattice_3d(512, alpha=1.0, seed=1)
    A = synth.dense(p) / synth.spectral_bound(p)
    X, norms = chain.square_chain(oracle.from_dense(A, 64), 4, 0.0, oracle.SPAMM)
    ref = np.linalg.matrix_power(A, 16)
    assert np.linalg.norm(oracle.to_dense(X) - ref) <= 1e-12 * np.linalg.norm(A) ** 16 * 512
    assert norms[-1] == pytest.approx(np.linalg.norm(ref), rel=1e-10)


def test_sp2_gapped_insulator_converges_to_the_projector():
    # two-sublattice on-site term +-delta plus a decay matrix of norm < delta:
    # the gap lies between the n_occ = #(-delta sites) lowest eigenvalues and the rest
    n, delta = 512, 4.0
    p = synth.lattice_3d(n, alpha=1.0, seed=3)
    bi, bj, dd, n_occ = synth.onsite_blocks(n, 64, delta)
    D = oracle.to_dense(oracle.from_leaves(n, 64, bi, bj, dd))
    assert np.array_equal(np.diag(D) < 0, synth.sublattice_parity(n) == 0)
    F = synth.dense(p) + D
    w, v = np.linalg.eigh(F)
    assert w[n_occ] - w[n_occ - 1] > 1.0
    bound = delta + synth.spectral_bound(p)
    assert bound >= max(-w[0], w[-1])
    FL = chain.add(1.0, oracle.from_dense(synth.dense(p), 64), 1.0, oracle.from_leaves(n, 64, bi, bj, dd))
    X, hist = chain.sp2(FL, n_occ, bound, 0.0, oracle.SPAMM, 60)
    P = v[:, :n_occ] @ v[:, :n_occ].T
    assert np.linalg.norm(oracle.to_dense(X) - P) <= 1e-8 * np.sqrt(n_occ)
    assert chain.trace(X) == pytest.approx(n_occ, abs=1e-8)
