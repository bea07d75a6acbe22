"""Error behaviour of Theorems 1-3 (and Section 5's observations) on the oracle.

||E||_F = O(n^{1/2}) at fixed tau and O(tau^{p/2}) for all p < 2 as tau -> 0,
|E_ij| = O(tau) element-wise; the paper measures slopes ~0.5 in n and ~1 in
tau (Figures of Section 5.3; 0.96-0.99 on the water clusters).  1-D decay
problem of Section 5.3 with a faster decay (alpha = 0.1) so the CPU can form
the exact product."""
import numpy as np
import pytest

import oracle
import synth

ALPHA, BS = 0.1, 16


def _inputs(n):
    nb = -(-n // BS)
    bi, bj = np.meshgrid(np.arange(nb), np.arange(nb), indexing="ij")
    bi, bj = bi.ravel(), bj.ravel()
    band = np.abs(bi - bj) * BS < 400 / ALPHA  # exp(-400) is far below the 1e-16 cutoff
    bi, bj = bi[band], bj[band]
    out = []
    for seed in (11, 12):
        p = synth.model_1d(n, alpha=ALPHA, seed=seed)
        out.append(oracle.from_leaves(n, BS, bi, bj, synth.leaves(p, BS, bi, bj)))
    return out


_cache = {}


def _exact(n):
    if n not in _cache:
        A, B = _inputs(n)
        _cache[n] = (A, B, oracle.exact(A, B))
    return _cache[n]


def _err(n, tau, mode):
    A, B, Cx = _exact(n)
    C, ikj = oracle.multiply(A, B, tau, oracle.MODES[mode])
    return oracle.error(Cx, C), C, Cx, len(ikj)


@pytest.mark.parametrize("mode", ["truncate", "spamm", "combined"])
def test_error_grows_like_sqrt_n(mode):
    ns = [1024, 2048, 4096, 8192]
    errs = [_err(n, 1e-6, mode)[0] for n in ns]
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert 0.35 <= slope <= 0.65, slope


@pytest.mark.parametrize("mode", ["truncate", "spamm", "combined"])
def test_error_falls_like_tau(mode):
    taus = [1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10]
    errs = [_err(2048, t, mode)[0] for t in taus]
    slope = np.polyfit(np.log(taus), np.log(errs), 1)[0]
    assert 0.8 <= slope <= 1.2, slope
    assert all(e2 <= e1 * 1.5 for e1, e2 in zip(errs, errs[1:]))


@pytest.mark.parametrize("mode", ["truncate", "spamm", "combined"])
def test_elementwise_error_is_order_tau_independent_of_n(mode):
    ratios = []
    for n in (1024, 4096):
        tau = 1e-6
        _, C, Cx, _ = _err(n, tau, mode)
        D = oracle.to_dense(Cx) - oracle.to_dense(C)
        ratios.append(np.abs(D).max() / tau)
    assert max(ratios) < 100.0
    assert ratios[1] < 3.0 * ratios[0] + 1.0


def test_truncmul_makes_more_leaf_products_and_needs_smaller_tau():
    """Section 5.3: at equal tau Truncmul multiplies more leaf pairs than SpAMM;
    to reach sigma = 1e-6 SpAMM can use a larger tau than Truncmul."""
    n_t = _err(2048, 1e-8, "truncate")[3]
    n_s = _err(2048, 1e-8, "spamm")[3]
    assert n_t > n_s
    grid = [1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10]
    pick = {m: max(t for t in grid if _err(2048, t, m)[0] <= 1e-6) for m in ("truncate", "spamm")}
    assert pick["spamm"] >= pick["truncate"]
