"""Derived element-wise error bounds of the tensor-core forms against the
FP64 product on the same kept set (a helper for the GPU tests).

FP16 scaled: each operand is represented by its two terms to 2^-22 relative
(after rounding to FP32), each leaf product is accumulated in FP32 over
K = 64 and added into an FP32 register accumulator once per step (one per
kept product, two for 128-leaves), n_k steps in all:
    |C_tc - C_fp64|_ij <= (n_k + 16) 2^-20 (|A||B|)_ij.

BF16 splits with S slices (3: bf16_split, 4: bf16_split4).  For the rows r of
A leaf (i, k) and columns c of B leaf (k, j), with l = the exponent of the
line's largest |x| (x_max < 2^l; 128-leaves are split into 64-wide K halves,
each with its own line exponents, and the terms below add over the halves),
per kept leaf product:
  * dropped digits and slice products (the split's residual, checked against
    exact arithmetic on the CPU in test_slices_host.py):
        64 (S + 1.01) 2^(lA_r + lB_c - 9 S);
  * rounding in the one FP32 accumulator shared by the index sums
    g >= NACC - 1 (NACC = 2 for S = 3, 3 for S = 4; the smaller sums are
    integers on a common grid, exact): at most one rounding of 2^-23 of the
    accumulator's bound per product added, n = 64 x (pairs in it):
        n 2^-23 64 sum_{g >= NACC-1} (g + 1) 2^(lA_r + lB_c - 9 g);
  * digits below the FP32 normal range after the leaf scale (dropped):
        64 S 2^-116 max|A_ik| max|B_kj|;
plus, once per output element, the two-float accumulation (2^-44 relative)
and the final FP64 rounding: 2^-44 (|A||B|)_ij + 2^-52 |C_ij|.
"""
import numpy as np

import oracle

FP16 = (16, 20)
SLICES = {"bf16_split": (3, 2), "bf16_split4": (4, 3)}  # prec -> (S, NACC)


def _line_exp(x, axis):
    """Exponent l of each line's largest |x| (max < 2^l); -inf for a zero line."""
    m = np.max(np.abs(x), axis=axis)
    _, e = np.frexp(m)
    return np.where(m > 0, e.astype(np.float64), -np.inf)


def slice_consts(S, nacc):
    trunc = 64.0 * (S + 1.01) * 2.0 ** (-9 * S)
    pairs = sum(g + 1 for g in range(nacc - 1, S))
    acc = 64.0 * pairs * 2.0 ** -23 * 64.0 * sum((g + 1) * 2.0 ** (-9 * g) for g in range(nacc - 1, S))
    return trunc, acc


def bound(prec, At: oracle.LeafMatrix, Bt: oracle.LeafMatrix, ikj: np.ndarray, ref: oracle.LeafMatrix):
    """Per-element bound for every leaf of ref (the FP64 oracle product on the
    kept triples ikj of the truncated inputs At, Bt), shape (ref.m, bs, bs)."""
    key = {(int(r), int(c)): q for q, (r, c) in enumerate(zip(ref.bi, ref.bj))}
    absA = oracle.LeafMatrix(At.n, At.bs, At.bi, At.bj, np.abs(At.data))
    absB = oracle.LeafMatrix(Bt.n, Bt.bs, Bt.bi, Bt.bj, np.abs(Bt.data))
    absprod = oracle.product(absA, absB, ikj)
    apos = {(int(r), int(c)): q for q, (r, c) in enumerate(zip(absprod.bi, absprod.bj))}
    out = np.zeros_like(ref.data)
    for (r, c), q in key.items():
        out[q] = absprod.data[apos[(r, c)]]
    nkh = At.bs // 64  # K halves: a 128-leaf product runs as two 64-deep steps
    if prec == "fp16_scaled":
        c0, e = FP16
        nk = np.zeros(ref.m)
        for i, _, j in ikj.tolist():
            nk[key[(i, j)]] += nkh
        return (nk[:, None, None] + c0) * 2.0 ** -e * out + 1e-300
    S, nacc = SLICES[prec]
    trunc, acc = slice_consts(S, nacc)
    ia = {(int(r), int(c)): q for q, (r, c) in enumerate(zip(At.bi, At.bj))}
    ib = {(int(r), int(c)): q for q, (r, c) in enumerate(zip(Bt.bi, Bt.bj))}
    # line exponents per 64-wide K half: A rows over columns 64 kh.., B columns over rows 64 kh..
    la = [[_line_exp(At.data[q][:, 64 * h:64 * h + 64], 1) for h in range(nkh)] for q in range(At.m)]
    lb = [[_line_exp(Bt.data[q][64 * h:64 * h + 64, :], 0) for h in range(nkh)] for q in range(Bt.m)]
    ma = np.max(np.abs(At.data), axis=(1, 2))
    mb = np.max(np.abs(Bt.data), axis=(1, 2))
    b = 2.0 ** -44 * out + 2.0 ** -52 * np.abs(ref.data)
    for i, k, j in ikj.tolist():
        qa, qb = ia[(i, k)], ib[(k, j)]
        p2 = sum(np.exp2(la[qa][h][:, None] + lb[qb][h][None, :]) for h in range(nkh))
        b[key[(i, j)]] += (trunc + acc) * p2 + nkh * 64.0 * S * 2.0 ** -116 * ma[qa] * mb[qb]
    return b + 1e-300
