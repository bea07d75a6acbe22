"""Algorithm 1 written out literally over dense numpy sub-blocks (tiny n only).

TEST INFRASTRUCTURE ONLY.  Independent of the C oracle: the norms at every
level are recomputed from the dense sub-block itself (||X||_F via numpy), the
recursion follows Algorithm 1 of the paper (for i, j in {0,1}: T_0, T_1 from
the k = 0 and k = 1 sub-products when ||A_ik|| ||B_kj|| >= tau, else 0;
C_ij = T_0 + T_1), and at the lowest level (block size bs) C = AB.
A sub-block that is identically zero is a null sub-matrix and is never
entered (Section 4.2).  Pure-Python recursion: keep n <= 128.
"""
from __future__ import annotations

import numpy as np


def spamm_literal(A: np.ndarray, B: np.ndarray, tau: float, bs: int, truncmul: bool = False):
    """Returns (C dense, list of kept leaf triples (i, k, j))."""
    n = A.shape[0]
    nb = -(-n // bs)
    side = 1
    while side < nb:
        side *= 2
    N = side * bs
    Ap = np.zeros((N, N))
    Bp = np.zeros((N, N))
    Ap[:n, :n] = A
    Bp[:n, :n] = B
    kept = []

    def rec(a, b, i0, k0, j0, size):
        # a = Ap block at (i0, k0), b = Bp block at (k0, j0), both size x size
        if size == bs:
            kept.append((i0 // bs, k0 // bs, j0 // bs))
            return a @ b
        h = size // 2
        C = np.zeros((size, size))
        for i in range(2):
            for j in range(2):
                T = []
                for k in range(2):
                    aik = a[i * h:(i + 1) * h, k * h:(k + 1) * h]
                    bkj = b[k * h:(k + 1) * h, j * h:(j + 1) * h]
                    if not aik.any() or not bkj.any():
                        T.append(np.zeros((h, h)))
                        continue
                    if truncmul or np.linalg.norm(aik) * np.linalg.norm(bkj) >= tau:
                        T.append(rec(aik, bkj, i0 + i * h, k0 + k * h, j0 + j * h, h))
                    else:
                        T.append(np.zeros((h, h)))
                C[i * h:(i + 1) * h, j * h:(j + 1) * h] = T[0] + T[1]
        return C

    root_ok = Ap.any() and Bp.any()
    if root_ok and N == bs and not truncmul:
        # a single leaf: the root pair is a leaf pair and takes the leaf test
        root_ok = np.linalg.norm(Ap) * np.linalg.norm(Bp) >= tau
    if root_ok:
        C = rec(Ap, Bp, 0, 0, 0, N)
    else:
        C = np.zeros((N, N))
    return C[:n, :n], kept
