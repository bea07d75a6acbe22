"""Two-sided pins for the oracle's skipped-product bound.

The bound of the error analysis (Theorem 2's proof in the appendix; Theorem 3
splits the combined method's error the same way) is
    ||AB - C||_F <= sqrt(sum_ij beta_ij^2),
    beta_ij = sum over the products (i, k, j) the method leaves out of ||A_ik||_F ||B_kj||_F,
with original (untruncated) norms.  ``oracle.skipped_bound`` computes it from
the kept set.  Two independent checks pin it from both sides:

* brute force: the same quantity written out as a loop over dense
  sub-blocks of tiny inputs, each norm taken with ``math.fsum`` and each
  leave-out decision taken from the method's definition (Algorithm 1's test;
  the block rule drops a block iff its norm < tau), at bs = 1 and bs = 4;
* equality: inputs built so that every left-out product lands in one output
  block, each a rank-one product u (v^T v) w^T with the same u and w and a
  positive weight.  Then ||A_ik B_kj||_F = ||A_ik||_F ||B_kj||_F for each of
  them, their sum has no cancellation, and the true error equals the bound.
A bound that sums every candidate product, or the kept ones instead of the
left-out ones, fails both.
"""
import math

import numpy as np
import pytest

import oracle


def _block_norm(a, i, k, bs):
    blk = a[i * bs:(i + 1) * bs, k * bs:(k + 1) * bs]
    return math.sqrt(math.fsum(float(x) * float(x) for x in blk.ravel()))


def brute_force_bound(a, b, bs, tau, mode, rule="block"):
    """sqrt(sum_ij beta_ij^2) by a loop over all block triples.

    Block rule: a block is dropped iff its norm < tau.  Element rule
    (Theorem 1): elements with |x| < tau become zero, a block left all-zero is
    dropped, and a kept product of truncated blocks still contributes
    ||A - A~|| ||B|| + ||A~|| ||B - B~|| to beta (the triangle inequality on
    A B - A~ B~ = (A - A~) B + A~ (B - B~))."""
    nb = a.shape[0] // bs
    at = np.where(np.abs(a) < tau, 0.0, a) if rule == "element" else a
    bt = np.where(np.abs(b) < tau, 0.0, b) if rule == "element" else b
    na = [[_block_norm(a, i, k, bs) for k in range(nb)] for i in range(nb)]
    nbm = [[_block_norm(b, k, j, bs) for j in range(nb)] for k in range(nb)]
    nat = [[_block_norm(at, i, k, bs) for k in range(nb)] for i in range(nb)]
    nbt = [[_block_norm(bt, k, j, bs) for j in range(nb)] for k in range(nb)]
    nda = [[_block_norm(a - at, i, k, bs) for k in range(nb)] for i in range(nb)]
    ndb = [[_block_norm(b - bt, k, j, bs) for j in range(nb)] for k in range(nb)]
    total = []
    for i in range(nb):
        for j in range(nb):
            beta = []
            for k in range(nb):
                x, y = na[i][k], nbm[k][j]
                if x == 0.0 or y == 0.0:
                    continue  # a null block: no candidate product
                if mode == oracle.SPAMM:
                    left_out = x * y < tau
                elif rule == "block":
                    dropped = x < tau or y < tau
                    left_out = dropped or (mode == oracle.COMBINED and x * y < tau)
                else:
                    xt, yt = nat[i][k], nbt[k][j]
                    dropped = xt == 0.0 or yt == 0.0
                    left_out = dropped or (mode == oracle.COMBINED and xt * yt < tau)
                if left_out:
                    beta.append(x * y)
                elif rule == "element" and mode != oracle.SPAMM:
                    beta.append(nda[i][k] * y + nat[i][k] * ndb[k][j])
            s = math.fsum(beta)
            total.append(s * s)
    return math.sqrt(math.fsum(total))


def _decay_pair(n, seed):
    rng = np.random.default_rng(seed)
    d = np.abs(np.subtract.outer(np.arange(n), np.arange(n)))
    a = rng.uniform(-1, 1, (n, n)) * np.exp(-0.5 * d)
    b = rng.uniform(-1, 1, (n, n)) * np.exp(-0.5 * d)
    return a, b


def _safe_taus(a, b, bs, candidates):
    """Thresholds no block norm or norm product lies within 1e-9 of (the
    brute force and the oracle sum squares in different orders)."""
    nb = a.shape[0] // bs
    na = np.array([[_block_norm(a, i, k, bs) for k in range(nb)] for i in range(nb)])
    nbm = np.array([[_block_norm(b, k, j, bs) for j in range(nb)] for k in range(nb)])
    vals = np.concatenate([na.ravel(), nbm.ravel(), np.outer(na.ravel(), nbm.ravel()).ravel()])
    vals = vals[vals > 0]
    return [t for t in candidates if np.all(np.abs(vals - t) > 1e-9 * t)]


def bound_battery():
    """Every pin of the bound; returns the names of the failing checks."""
    failed = []
    for bs, n in ((1, 12), (4, 32)):
        a, b = _decay_pair(n, seed=11 + bs)
        LA, LB = oracle.from_dense(a, bs), oracle.from_dense(b, bs)
        for tau in _safe_taus(a, b, bs, (3e-4, 1e-2, 0.07)):
            for mode in (oracle.SPAMM, oracle.COMBINED, oracle.TRUNCATE):
                for rule in ("block", "element"):
                    ref = brute_force_bound(a, b, bs, tau, mode, rule)
                    try:
                        got = oracle.skipped_bound(LA, LB, tau, mode, rule)
                    except Exception:  # a mutant may fail an internal consistency check
                        got = math.nan
                    if not abs(got - ref) <= 1e-13 * max(ref, 1e-300):
                        failed.append(f"brute force bs={bs} tau={tau} mode={mode} rule={rule}")
    for bs in (1, 4):
        a, b, tau = aligned_case(bs)
        LA, LB = oracle.from_dense(a, bs), oracle.from_dense(b, bs)
        exact = oracle.exact(LA, LB)
        for mode in (oracle.SPAMM, oracle.COMBINED):
            C, _ = oracle.multiply(LA, LB, tau, mode)
            err = oracle.error(exact, C)
            bound = oracle.skipped_bound(LA, LB, tau, mode)
            if not (err > 0 and abs(err - bound) <= 1e-12 * bound + rounding_slack(a, b)):
                failed.append(f"equality bs={bs} mode={mode}")
        # every block norm is above tau: Truncmul leaves nothing out
        if oracle.skipped_bound(LA, LB, tau, oracle.TRUNCATE) != 0.0:
            failed.append(f"truncate bound zero bs={bs}")
    return failed


def rounding_slack(a, b):
    """Rounding of the kept products: both C and the exact product carry
    errors of a few ulp of (|A||B|)_ij, far below the left-out part here."""
    return 1e-14 * np.linalg.norm(np.abs(a) @ np.abs(b))


def aligned_case(bs, nb=4):
    """Block-diagonal A and B of norm ~1 plus small rank-one blocks A_0k = c_k u v^T
    and B_k0 = d_k v w^T (k >= 1).  With eps^2 < tau < eps for the small blocks'
    norms eps, the only products left out are A_0k B_k0: all in output block
    (0, 0), all positive multiples of u w^T."""
    rng = np.random.default_rng(5 + bs)
    n = nb * bs
    a = np.zeros((n, n))
    b = np.zeros((n, n))
    for k in range(nb):
        s = slice(k * bs, (k + 1) * bs)
        a[s, s] = rng.uniform(0.5, 1.0, (bs, bs))
        b[s, s] = rng.uniform(0.5, 1.0, (bs, bs))
    u = rng.uniform(0.5, 1.0, bs)
    v = rng.uniform(0.5, 1.0, bs)
    w = rng.uniform(0.5, 1.0, bs)
    nu, nv, nw = np.linalg.norm(u), np.linalg.norm(v), np.linalg.norm(w)
    for k in range(1, nb):
        c = 1e-3 * (1 + 0.25 * k) / (nu * nv)  # ||A_0k|| = 1e-3 (1 + k / 4)
        d = 2e-3 * (1 + 0.5 * k) / (nv * nw)   # ||B_k0|| = 2e-3 (1 + k / 2)
        a[0:bs, k * bs:(k + 1) * bs] = c * np.outer(u, v)
        b[k * bs:(k + 1) * bs, 0:bs] = d * np.outer(v, w)
    tau = 1e-4  # above every small x small product (< 2e-5), below every other one (> 5e-4)
    return a, b, tau


def test_bound_equals_brute_force_loop():
    for bs, n in ((1, 12), (4, 32)):
        a, b = _decay_pair(n, seed=11 + bs)
        LA, LB = oracle.from_dense(a, bs), oracle.from_dense(b, bs)
        taus = _safe_taus(a, b, bs, (3e-4, 1e-2, 0.07))
        assert len(taus) == 3
        for tau in taus:
            for mode in (oracle.SPAMM, oracle.COMBINED, oracle.TRUNCATE):
                for rule in ("block", "element"):
                    ref = brute_force_bound(a, b, bs, tau, mode, rule)
                    got = oracle.skipped_bound(LA, LB, tau, mode, rule)
                    assert abs(got - ref) <= 1e-13 * max(ref, 1e-300), (bs, tau, mode, rule, got, ref)
                    if mode != oracle.TRUNCATE and tau >= 1e-2:
                        assert ref > 0  # the case leaves products out


@pytest.mark.parametrize("bs", [1, 4])
def test_bound_attained_by_aligned_rank_one_products(bs):
    a, b, tau = aligned_case(bs)
    LA, LB = oracle.from_dense(a, bs), oracle.from_dense(b, bs)
    exact = oracle.exact(LA, LB)
    # the construction: exactly the nb - 1 products A_0k B_k0 are left out
    kept = oracle.kept_flat(LA, LB, tau, oracle.SPAMM)
    allp = oracle.kept_flat(LA, LB, 0.0, oracle.SPAMM)
    left = set(map(tuple, allp.tolist())) - set(map(tuple, kept.tolist()))
    assert left == {(0, k, 0) for k in range(1, 4)}
    expect = math.fsum(1e-3 * (1 + 0.25 * k) * 2e-3 * (1 + 0.5 * k) for k in range(1, 4))
    for mode in (oracle.SPAMM, oracle.COMBINED):
        C, _ = oracle.multiply(LA, LB, tau, mode)
        err = oracle.error(exact, C)
        bound = oracle.skipped_bound(LA, LB, tau, mode)
        assert abs(bound - expect) <= 1e-13 * expect
        assert abs(err - bound) <= 1e-12 * bound + rounding_slack(a, b), (err, bound)
    assert oracle.skipped_bound(LA, LB, tau, oracle.TRUNCATE) == 0.0


def test_battery_accepts_the_oracle():
    assert bound_battery() == []
