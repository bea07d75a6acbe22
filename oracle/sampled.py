"""Oracle on a window of output leaves of a large synthetic problem.

TEST INFRASTRUCTURE ONLY.  For output leaves (i, j) with i in `rows` and j
in `cols`, C_ij depends only on A's block rows i and B's block columns j
(every kept triple (i,k,j) reads A_ik and B_kj; truncation and the norm test
are per leaf).  So the oracle regenerates just those leaves from the seeded
generator, restricts A and B to them and runs the ordinary oracle pipeline:
the result equals the corresponding leaves of the full oracle product.
"""
from __future__ import annotations

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
