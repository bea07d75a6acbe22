"""Oracle on a window of output leaves of a large synthetic problem.

TEST INFRASTRUCTURE ONLY.  For output leaves (i, j) with i in `rows` and j
in `cols`, C_ij depends only on A's block rows i and B's block columns j
(every kept triple (i,k,j) reads A_ik and B_kj; truncation and the norm test
are per leaf).  So the oracle regenerates just those leaves from the seeded
generator, restricts A and B to them and runs the ordinary oracle pipeline:
the result equals the corresponding leaves of the full oracle product.

`error_estimate` uses this per output leaf to estimate ||AB - C||_F of a
problem whose exact product is too large to form (every sampled leaf of AB is
exact; the estimate carries a stratified-sampling interval).
"""
from __future__ import annotations

import numpy as np

import oracle
import synth


def _leaves_rows(p: synth.DecayParams, bs: int, rows, transpose: bool) -> oracle.LeafMatrix:
    nb = -(-p.n // bs)
    bi, bj = [], []
    for r in rows:
        for k in range(nb):
            a, b = (k, r) if transpose else (r, k)
            if synth.leaf_bound(p, bs, a, b) >= p.cutoff:
                bi.append(a)
                bj.append(b)
    data = synth.leaves(p, bs, bi, bj)
    return oracle.from_leaves(p.n, bs, bi, bj, data)


def window_inputs(pa, pb, bs, rows, cols):
    """A restricted to block rows `rows`, B restricted to block columns `cols`."""
    return _leaves_rows(pa, bs, rows, False), _leaves_rows(pb, bs, cols, True)


def window_product(A_rows: oracle.LeafMatrix, B_cols: oracle.LeafMatrix, tau: float, mode: int, rule="block"):
    """(C leaves for the window, kept triples): the ordinary oracle pipeline."""
    return oracle.multiply(A_rows, B_cols, tau, mode, rule)


def window_exact(A_rows, B_cols):
    return oracle.exact(A_rows, B_cols)


# ------------------------------------------------- sampled approximation error
def _band(bound: np.ndarray, decades: int, nbands: int) -> np.ndarray:
    """Distance band of an output leaf position from the generator's bound of
    the input leaf at the same position (how far apart the two index blocks
    are): band b holds bounds in (10^-(b+1)d, 10^-bd], the last band
    everything below."""
    lg = -np.log10(np.maximum(bound, 1e-300))
    return np.minimum((np.maximum(lg, 0.0) // decades).astype(np.int64), nbands - 1)


def _strata_row(pa, bs: int, i: int, cols: np.ndarray, decades: int, nbands: int) -> np.ndarray:
    """Strata of the output leaf positions (i, j) of block row i: 0 for the
    diagonal leaf (the largest leaves of AB, all alike), 1 + the distance band
    for the others."""
    st = 1 + _band(synth.leaf_bounds_row(pa, bs, i, cols), decades, nbands)
    if i < len(cols):
        st[i] = 0
    return st


def leaf_sq(pa, pb, bs: int, i: int, j: int, tau: float, mode: int, rule="block"):
    """(||(AB)_ij - C_ij||_F^2, ||(AB)_ij||_F^2) for one output leaf: the exact
    leaf over every non-null k of the untruncated inputs against the method's
    leaf (its truncation and kept set restricted to block row i of A and block
    column j of B, which is all the leaf depends on)."""
    A_row, B_col = window_inputs(pa, pb, bs, [i], [j])
    X = window_exact(A_row, B_col)
    C, _ = window_product(A_row, B_col, tau, mode, rule)
    return oracle.error(X, C) ** 2, oracle.frob_norm(X) ** 2


def leaf_error_sq(pa, pb, bs: int, i: int, j: int, tau: float, mode: int, rule="block") -> float:
    """||(AB)_ij - C_ij||_F^2 for one output leaf (see `leaf_sq`)."""
    return leaf_sq(pa, pb, bs, i, j, tau, mode, rule)[0]


def _positions(pa, bs: int, nb: int, decades: int, nbands: int, ranks: dict) -> dict:
    """Output leaf positions of the given ranks per stratum (rank r of stratum
    h = its r-th position in row-major order)."""
    cols = np.arange(nb, dtype=np.int64)
    seen = np.zeros(nbands + 1, np.int64)
    want = {h: np.sort(np.asarray(r, np.int64)) for h, r in ranks.items() if len(r)}
    out = {h: [] for h in ranks}
    for i in range(nb):
        band = _strata_row(pa, bs, i, cols, decades, nbands)
        for h in want:
            where = np.flatnonzero(band == h)
            hit = np.isin(seen[h] + np.arange(len(where)), want[h], assume_unique=True)
            out[h].extend((i, int(j)) for j in where[hit])
            seen[h] += len(where)
    return out


def error_estimate(pa, pb, bs: int, tau: float, mode: int, samples: int = 256, seed: int = 0, rule="block",
                   decades: int = 4, nbands: int = 5, z: float = 1.959964):
    """Estimate ||AB - C||_F of a problem too large for the full exact
    product, from sampled output leaves (stratified simple random sampling
    without replacement, two-phase Neyman allocation).

    Population: all nb x nb output leaf positions (a position no kept or
    exact product reaches contributes zero).  Strata (`_strata_row`): the
    diagonal leaves, whose products are the largest and alike, and the
    others by decades of the generator's leaf bound at the position.  Phase 1 takes a pilot of
    max(2, samples / (2 H)) positions from each of the H non-empty strata
    (a smaller stratum whole); phase 2 gives the remaining samples to the
    strata in proportion to N_h s_h (stratum size times the pilot's standard
    deviation of e_ij^2), as Neyman allocation prescribes.  With all n_h
    samples of stratum h, mean m_h and variance s_h^2 of e_ij^2:
        T = sum_h N_h m_h,  V = sum_h N_h^2 (1 - n_h / N_h) s_h^2 / n_h,
    and the interval for ||E||_F is sqrt(max(0, T -/+ z sqrt(V))) (a normal
    approximation: for skewed strata and few samples it covers less often
    than its nominal rate; on the 1-D model problem n = 2048 it covered the
    true error in 12, 16 and 19 of 20 seeds with 64, 128 and 256 samples).
    The same samples give the stratified estimate of ||AB||_F^2 (sum of the
    exact leaves' squared norms), hence the relative error.  Returns the
    estimate, the interval, ||AB||_F and the strata."""
    nb = -(-pa.n // bs)
    cols = np.arange(nb, dtype=np.int64)
    counts = np.zeros(nbands + 1, np.int64)
    for i in range(nb):
        counts += np.bincount(_strata_row(pa, bs, i, cols, decades, nbands), minlength=nbands + 1)
    rng = np.random.default_rng(seed)
    live = [int(h) for h in np.flatnonzero(counts)]
    perm = {h: rng.permutation(int(counts[h]))[:samples] for h in live}
    pilot = max(2, samples // (2 * max(1, len(live))))
    n0 = {h: min(int(counts[h]), pilot) for h in live}

    xsq = {h: [] for h in live}

    def evaluate(ranks):
        pos = _positions(pa, bs, nb, decades, nbands, ranks)
        out = {}
        for h in ranks:
            pairs = [leaf_sq(pa, pb, bs, i, j, tau, mode, rule) for i, j in pos[h]]
            out[h] = [e for e, _ in pairs]
            xsq[h].extend(x for _, x in pairs)
        return out

    y = evaluate({h: perm[h][:n0[h]] for h in live})
    rest = samples - sum(n0.values())
    room = {h: min(int(counts[h]), samples) - n0[h] for h in live}
    if rest > 0 and any(room.values()):
        sd = {h: float(np.std(y[h], ddof=1)) if len(y[h]) > 1 else 0.0 for h in live}
        w = {h: counts[h] * sd[h] if room[h] > 0 else 0.0 for h in live}
        if sum(w.values()) <= 0.0:
            w = {h: float(counts[h]) if room[h] > 0 else 0.0 for h in live}
        tot = sum(w.values())
        extra = {h: min(room[h], int(rest * w[h] / tot)) for h in live}
        left = rest - sum(extra.values())
        for h in sorted(live, key=lambda h: -w[h]):  # what rounding left, to the heaviest strata
            add = min(left, room[h] - extra[h])
            extra[h] += add
            left -= add
        more = evaluate({h: perm[h][n0[h]:n0[h] + extra[h]] for h in live if extra[h] > 0})
        for h, v in more.items():
            y[h] = y[h] + v
    strata = []
    total, var, xtotal = 0.0, 0.0, 0.0
    for h in live:
        v = np.asarray(y[h])
        N, m = int(counts[h]), len(v)
        mean = float(np.mean(v))
        s2 = float(np.var(v, ddof=1)) if m > 1 else 0.0
        total += N * mean
        xtotal += N * float(np.mean(xsq[h]))
        var += N * N * (1.0 - m / N) * s2 / m
        strata.append({"stratum": h, "positions": N, "sampled": m, "mean_err_sq": mean, "var_err_sq": s2})
    half = z * np.sqrt(var)
    return {"estimate": float(np.sqrt(total)), "low": float(np.sqrt(max(0.0, total - half))),
            "high": float(np.sqrt(total + half)), "err_sq": total, "err_sq_sd": float(np.sqrt(var)),
            "exact_norm": float(np.sqrt(xtotal)), "samples": int(sum(s["sampled"] for s in strata)),
            "strata": strata}


def _main(argv=None):
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description="Sampled estimate of ||AB - C||_F on a synthetic decay problem.")
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--kind", choices=["1d", "3d"], default="3d")
    ap.add_argument("--alpha", type=float, required=True)
    ap.add_argument("--bs", type=int, default=64)
    ap.add_argument("--tau", type=float, required=True)
    ap.add_argument("--mode", choices=list(oracle.MODES), default="combined")
    ap.add_argument("--samples", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    make = synth.lattice_3d if a.kind == "3d" else (lambda n, alpha, seed: synth.model_1d(n, alpha=alpha, seed=seed))
    pa, pb = make(a.n, alpha=a.alpha, seed=1), make(a.n, alpha=a.alpha, seed=2)
    t0 = time.perf_counter()
    r = error_estimate(pa, pb, a.bs, a.tau, oracle.MODES[a.mode], samples=a.samples, seed=a.seed)
    r.update({"n": a.n, "kind": a.kind, "alpha": a.alpha, "bs": a.bs, "tau": a.tau, "mode": a.mode,
              "seconds": time.perf_counter() - t0, "threads": oracle.num_threads()})
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    _main()
