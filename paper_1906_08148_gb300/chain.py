"""Purification-style chains of approximate products on resident matrices.

Density-matrix purification is the application the paper's multiply serves
(Section 1): the density matrix is computed by a chain of multiplications of
matrices with decay, each approximate (SpAMM / Truncmul / Hybrid with the
same tau), the intermediate matrices kept resident.  Two chains:

* square_chain: X <- X X, `steps` times (the repeated squaring of a matrix
  scaled to spectral radius <= 1);
* sp2: second-order spectral projection (Niklasson, Phys. Rev. B 66, 155115
  (2002)): X0 = (b I - F) / (2 b) with b >= ||F||_2, then per step X <- X^2 or
  X <- 2X - X^2, whichever trace is closer to the number of occupied states,
  converging to the projector onto the eigenvectors of F's lowest eigenvalues.

Every step runs on the device through the C ABI (spamm_multiply, spamm_add,
spamm_identity, spamm_trace, spamm_error); only traces and norms come back.
"""
from __future__ import annotations

from . import spamm as S


def square_chain(ctx, X0, steps: int, tau: float, mode: str = "combined", prec: str = "fp64", keep_input=True):
    """Returns (X_final, per-step stats).  X0 is not released when keep_input."""
    X, hist = X0, []
    for _ in range(steps):
        Y, st = S.spamm_multiply(ctx, X, X, tau, mode, prec, stats=True)
        if X is not X0 or not keep_input:
            X.close()
        X = Y
        hist.append({"n_kept": st["n_kept"], "n_c_leaves": st["n_c_leaves"], "ms_gemm": st["ms_gemm"],
                     "kept_flops": st["kept_flops"], "frob": S.spamm_frob_norm(ctx, X)})
    return X, hist


def sp2(ctx, F, n_occ: float, bound: float, tau: float, mode: str = "combined", prec: str = "fp64",
        iters: int = 40, tol: float = 0.0, X0=None, probe=None):
    """Returns (X, per-step history: traces of X and X^2, branch, ||X - X^2||_F,
    kept products).  Stops early once ||X - X^2||_F <= tol.  X0: start from
    this matrix (released as the chain moves on) instead of (bI - F) / (2b).
    probe(step, X, X2): called after each product, its dict (if any) is
    added to that step's history."""
    if X0 is None:
        info = F.info()
        I = S.spamm_identity(ctx, info["n"], info["bs"])
        X = S.spamm_add(ctx, -0.5 / bound, F, 0.5, I)
        I.close()
    else:
        X = X0
    hist = []
    for it in range(iters):
        X2, st = S.spamm_multiply(ctx, X, X, tau, mode, prec, stats=True)
        extra = probe(it, X, X2) if probe is not None else None
        t1, t2 = S.spamm_trace(ctx, X), S.spamm_trace(ctx, X2)
        idem = S.spamm_error(ctx, X, X2)
        if abs(t2 - n_occ) < abs(2.0 * t1 - t2 - n_occ):
            Xn, branch = X2, "square"
        else:
            Xn, branch = S.spamm_add(ctx, 2.0, X, -1.0, X2), "2x-x2"
            X2.close()
        X.close()
        X = Xn
        hist.append({"trace": t1, "trace_sq": t2, "branch": branch, "idempotency": idem,
                     "n_kept": st["n_kept"], "ms_gemm": st["ms_gemm"], "kept_flops": st["kept_flops"]})
        if extra:
            hist[-1].update(extra)
        if tol and idem <= tol:
            break
    return X, hist
