"""Oracle for the operations of a density-matrix purification chain.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): plain FP64 NumPy
over leaf lists, no code shared with the CUDA path.

Density-matrix purification is the application that motivates the paper
(Section 1: the density matrix of a Hartree-Fock / Kohn-Sham calculation is
computed by iterated multiplications of matrices with decay, and Section 4.4
lists addition and rescaling beside multiplication among the leaf library's
operations).  SP2 (second-order spectral projection, Niklasson, Phys. Rev. B
66, 155115 (2002)) maps the spectrum of X0 = (b I - F) / (2 b), b >= ||F||_2,
into [0, 1] and iterates X <- X^2 or X <- 2X - X^2, choosing per step the
branch whose trace is closer to the number of occupied states N; it converges
to the projector onto the eigenvectors of the N lowest eigenvalues of F.

Functions:
* add(alpha, X, beta, Y): alpha X + beta Y leaf by leaf, element value
  fl(fl(alpha x) + fl(beta y)) with an absent leaf read as zero, leaves that
  come out exactly zero dropped (a leaf is stored iff it has a non-zero
  element, Section 4.4);
* identity(n, bs), trace(X);
* sp2(F, n_occ, bound, tau, mode, iters): the chain with the paper's
  approximate multiply (``oracle.multiply``) for every product;
* square_chain(X0, steps, tau, mode): X <- X X, the plain repeated squaring.
"""
from __future__ import annotations

import numpy as np

from . import LeafMatrix, error, multiply


def _keys(M: LeafMatrix, side: int) -> np.ndarray:
    return M.bi.astype(np.int64) * side + M.bj


def add(alpha: float, X: LeafMatrix, beta: float, Y: LeafMatrix) -> LeafMatrix:
    assert X.n == Y.n and X.bs == Y.bs
    side = 1 << 20
    kx, ky = _keys(X, side), _keys(Y, side)
    keys = np.union1d(kx, ky)
    bs = X.bs
    out = np.zeros((len(keys), bs, bs))
    ax = np.zeros((len(keys), bs, bs))
    by = np.zeros((len(keys), bs, bs))
    ax[np.searchsorted(keys, kx)] = alpha * X.data
    by[np.searchsorted(keys, ky)] = beta * Y.data
    out = ax + by  # one rounding for each product and one for the sum
    nz = np.any(out != 0.0, axis=(1, 2))
    keys = keys[nz]
    return LeafMatrix(X.n, bs, (keys // side).astype(np.int32), (keys % side).astype(np.int32), out[nz])


def identity(n: int, bs: int) -> LeafMatrix:
    nb = -(-n // bs)
    data = np.zeros((nb, bs, bs))
    for q in range(nb):
        rows = min(bs, n - q * bs)
        data[q, np.arange(rows), np.arange(rows)] = 1.0
    idx = np.arange(nb, dtype=np.int32)
    return LeafMatrix(n, bs, idx, idx, data)


def trace(X: LeafMatrix) -> float:
    diag = X.bi == X.bj
    return float(np.sum(np.trace(X.data[diag], axis1=1, axis2=2)))


def sp2(F: LeafMatrix, n_occ: float, bound: float, tau: float, mode: int, iters: int):
    """SP2 from X0 = (bound I - F) / (2 bound); returns (X, history) with, per
    step, the traces of X and X^2, the branch taken and ||X - X^2||_F."""
    X = add(-0.5 / bound, F, 0.5, identity(F.n, F.bs))
    hist = []
    for _ in range(iters):
        X2, _ = multiply(X, X, tau, mode)
        t1, t2 = trace(X), trace(X2)
        idem = error(X, X2)
        if abs(t2 - n_occ) < abs(2.0 * t1 - t2 - n_occ):
            X, branch = X2, "square"
        else:
            X, branch = add(2.0, X, -1.0, X2), "2x-x2"
        hist.append({"trace": t1, "trace_sq": t2, "branch": branch, "idempotency": idem})
    return X, hist


def square_chain(X0: LeafMatrix, steps: int, tau: float, mode: int):
    X, norms = X0, []
    for _ in range(steps):
        X, _ = multiply(X, X, tau, mode)
        norms.append(float(np.sqrt(np.sum(X.sq))))
    return X, norms
