"""Pins for the seeded input generator (Definitions 1-3 of the paper)."""
import math

import numpy as np
import pytest

import synth


def test_exp_matches_libm_within_a_few_ulp():
    rng = np.random.default_rng(0)
    xs = np.concatenate([np.linspace(-699.0, 0.0, 20001), -rng.exponential(8.0, 20000)])
    worst = max(abs(synth.exp_nonpos(x) - math.exp(x)) / math.exp(x) for x in xs)
    assert worst <= 4 * 2.0 ** -53
    assert synth.exp_nonpos(0.0) == 1.0
    assert synth.exp_nonpos(-800.0) == 0.0


def test_uniform_range_symmetry_and_moments():
    vals = np.array([synth.uniform(7, i, j) for i in range(60) for j in range(60)])
    assert np.all(vals >= -1.0) and np.all(vals < 1.0)
    assert synth.uniform(7, 3, 11) == synth.uniform(7, 11, 3)
    assert synth.uniform(7, 3, 11) != synth.uniform(8, 3, 11)
    assert abs(vals.mean()) < 0.05
    assert abs(vals.var() - 1.0 / 3.0) < 0.02


def test_lattice_is_a_box_in_morton_order():
    pts = np.array([synth.lattice_point(i) for i in range(65536)])
    assert pts[:, 0].max() == 63 and pts[:, 1].max() == 31 and pts[:, 2].max() == 31
    assert len({tuple(p) for p in pts}) == 65536
    # Morton order with x first: index 1 -> (1,0,0), 2 -> (0,1,0), 4 -> (0,0,1)
    assert synth.lattice_point(1) == (1, 0, 0)
    assert synth.lattice_point(2) == (0, 1, 0)
    assert synth.lattice_point(4) == (0, 0, 1)
    assert synth.lattice_point(7) == (1, 1, 1)


@pytest.mark.parametrize("kind", [synth.KIND_1D, synth.KIND_3D])
def test_distance_is_a_pseudo_metric(kind):
    """Section 3: d >= 0, symmetric, d(i,i) = 0, triangle inequality."""
    p = synth.DecayParams(n=4096, kind=kind)
    rng = np.random.default_rng(1)
    for _ in range(500):
        i, j, k = (int(v) for v in rng.integers(0, 4096, 3))
        dij, dji = synth.distance(p, i, j), synth.distance(p, j, i)
        assert dij >= 0 and dij == dji and synth.distance(p, i, i) == 0.0
        assert dij <= synth.distance(p, i, k) + synth.distance(p, k, j) + 1e-12
    if kind == synth.KIND_1D:
        assert synth.distance(p, 10, 3) == 7.0


def test_finite_neighbourhood_3d():
    """Definition 3 holds on the lattice with beta = 3: |N(i,R)| <= gamma R^3."""
    p = synth.lattice_3d(4096)
    for i in (0, 1000, 4095):
        for R in (1.0, 2.0, 4.0):
            cnt = sum(synth.distance(p, i, j) <= R for j in range(4096))
            assert cnt <= (4.0 / 3.0 * math.pi * (R + 1.0) ** 3) * 1.0 + 1


@pytest.mark.parametrize("params", [synth.model_1d(300, alpha=0.05), synth.lattice_3d(512, alpha=1.0)])
def test_decay_bound_and_cutoff(params):
    """Definition 1 with c = 1: |a_ij| <= exp(-alpha d(i,j)); |a| < cutoff is 0."""
    A = synth.dense(params)
    assert np.array_equal(A, A.T)
    for i in range(0, params.n, 7):
        for j in range(0, params.n, 5):
            bound = math.exp(-params.alpha * synth.distance(params, i, j))
            assert abs(A[i, j]) <= bound * (1 + 1e-14)
    nz = A[A != 0.0]
    assert np.all(np.abs(nz) >= params.cutoff)


def test_leaves_match_dense_with_zero_padding():
    p = synth.model_1d(100, alpha=0.1, seed=5)
    A = synth.dense(p)
    bs = 32
    L = synth.leaves(p, bs, [0, 3, 2], [1, 3, 0])
    assert np.array_equal(L[0], A[0:32, 32:64])
    assert np.array_equal(L[1][:4, :4], A[96:100, 96:100])
    assert not L[1][4:, :].any() and not L[1][:, 4:].any()
    assert np.array_equal(L[2], A[64:96, 0:32])


@pytest.mark.parametrize("params,bs", [(synth.model_1d(600, alpha=0.05), 32), (synth.lattice_3d(4096, alpha=0.7), 64)])
def test_leaf_bound_dominates_every_element(params, bs):
    A = synth.dense(params)
    nb = -(-params.n // bs)
    pad = np.zeros((nb * bs, nb * bs))
    pad[:params.n, :params.n] = np.abs(A)
    tight = 0
    for bi in range(nb):
        for bj in range(nb):
            b = synth.leaf_bound(params, bs, bi, bj)
            m = pad[bi * bs:(bi + 1) * bs, bj * bs:(bj + 1) * bs].max()
            assert m <= b
            tight += m > 0.1 * b
    assert tight > 0


@pytest.mark.parametrize("fill", [0.05, 0.3, 0.9])
def test_block_sparse_fill_and_values(fill):
    """Section 5.2's random block-sparse input: independent uniform block
    positions (fill fraction within a 4-sigma binomial band), elements in
    [-1, 1) with mean ~0, deterministic per seed, different for another seed."""
    n, bs = 2048, 32
    nb = n // bs
    bi, bj, d = synth.block_sparse(n, bs, fill, seed=11)
    m = len(bi)
    sd = np.sqrt(nb * nb * fill * (1 - fill))
    assert abs(m - fill * nb * nb) <= 4 * sd
    assert np.all((d >= -1.0) & (d < 1.0))
    assert abs(d.mean()) < 4 * np.sqrt(1 / 3 / d.size)
    assert len(set(zip(bi.tolist(), bj.tolist()))) == m
    b2 = synth.block_sparse(n, bs, fill, seed=11)
    assert np.array_equal(b2[2], d)
    b3 = synth.block_sparse(n, bs, fill, seed=12)
    assert not (len(b3[0]) == m and np.array_equal(b3[0], bi) and np.array_equal(b3[1], bj))


def test_block_sparse_padding_stays_zero():
    n, bs = 300, 32
    bi, bj, d = synth.block_sparse(n, bs, 0.9, seed=5)
    for q in range(len(bi)):
        r0, c0 = bi[q] * bs, bj[q] * bs
        rows, cols = max(0, min(bs, n - r0)), max(0, min(bs, n - c0))
        assert not np.any(d[q, rows:, :]) and not np.any(d[q, :, cols:])
        assert np.all(d[q, :rows, :cols] != 0.0)


@pytest.mark.parametrize("kind,n,pw", [(synth.KIND_1D, 700, 2), (synth.KIND_3D, 512, 3), (synth.KIND_3D, 1000, 4)])
def test_algebraic_decay_law(kind, n, pw):
    """a_ij = c u_ij / (1 + d)^p: the bound holds, the law's value is exact in
    closed form on sample pairs, the leaf bound dominates, and the spectral
    bound dominates the largest eigenvalue magnitude."""
    p = synth.DecayParams(n=n, kind=kind, alpha=float(pw), seed=5, law=synth.LAW_ALGEBRAIC)
    A = synth.dense(p)
    assert np.array_equal(A, A.T)
    i, j = np.triu_indices(n, 1)
    sel = np.random.default_rng(0).choice(len(i), 2000, replace=False)
    for a, b in zip(i[sel], j[sel]):
        d = synth.distance(p, int(a), int(b))
        want = synth.uniform(p.seed, int(a), int(b)) / (1.0 + d) ** pw
        assert A[a, b] == pytest.approx(want, rel=4e-16 * pw, abs=0)
        assert abs(A[a, b]) <= 1.0 / (1.0 + d) ** pw
    bs = 32
    for bi in range(0, n // bs, 5):
        for bj in range(0, n // bs, 3):
            blk = A[bi * bs:(bi + 1) * bs, bj * bs:(bj + 1) * bs]
            assert np.abs(blk).max() <= synth.leaf_bound(p, bs, bi, bj)
    assert np.abs(np.linalg.eigvalsh(A)).max() <= synth.spectral_bound(p)
