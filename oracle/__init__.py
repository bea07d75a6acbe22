"""Plain FP64 CPU oracle for SpAMM, Truncmul and their combination.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the library.  It shares no
code with the CUDA path; the only common module is the seeded input generator
``synth`` (which holds none of the method's arithmetic).

What it computes, in the paper's order (Artemov, arXiv:1906.08148):

* leaves and their squared Frobenius norms, parents as sums of the four
  children (Section 2, the norm recursion; Section 4.2: every matrix stores
  its squared norm); a leaf is kept iff it has a non-zero element (Sec. 4.4);
* input truncation with the same tau as the product test (Theorem 1 for the
  element rule; the block rule drops a leaf iff its Frobenius norm < tau);
* the kept set of leaf triples (i,k,j): Algorithm 1's norm test
  ||A_ik|| ||B_kj|| >= tau applied down to leaf pairs (Section 4.4), both as a
  literal recursion of Algorithm 1 and as the flat test over all leaf pairs;
  Truncmul keeps every pair of non-null leaves (Section 5.3);
* the product: each output leaf the sum over its kept k, ascending, of naive
  FP64 leaf products (Algorithm 1, "C = AB" at the lowest level);
* the error ||X - Y||_F and the skipped-product bound.

Pins: every function is checked in ``tests/test_oracle_*.py`` against what
the paper and plain mathematics fix (brute force on tiny inputs, the dense
product at tau = 0, the element form of Theorem 2's proof, the structural
examples of Section 4.4, closed forms, the error bound and the error slopes
of Theorems 1-3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

TRUNCATE, SPAMM, COMBINED = 0, 1, 2
MODES = {"truncate": TRUNCATE, "spamm": SPAMM, "combined": COMBINED}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, OpenMP across output leaves)."""
    src = os.path.join(_HERE, "spamm_oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    lp = ctypes.POINTER(ctypes.c_int64)
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.orc_pairwise_sumsq.argtypes = [dp, i64]
    lib.orc_pairwise_sumsq.restype = f64
    lib.orc_leaf_sqnorms.argtypes = [i64, i32, dp, dp]
    lib.orc_leaves_from_dense.argtypes = [i64, i32, dp, i64, ip, ip, dp]
    lib.orc_leaves_from_dense.restype = i64
    lib.orc_tree_norms.argtypes = [i32, i64, ip, ip, dp, dp]
    lib.orc_kept_flat.argtypes = [i64, ip, ip, dp, i64, ip, ip, dp, i32, f64, i32, ip]
    lib.orc_kept_flat.restype = i64
    lib.orc_kept_recursive.argtypes = [i32, dp, dp, f64, i32, ip]
    lib.orc_kept_recursive.restype = i64
    lib.orc_leaf_products.argtypes = [i32, dp, dp, i64, lp, lp, lp, dp]
    lib.orc_dense_product.argtypes = [i64, dp, dp, dp]
    lib.orc_leaf_diff_sumsq.argtypes = [i32, dp, dp]
    lib.orc_leaf_diff_sumsq.restype = f64
    lib.orc_num_threads.restype = i32
    return lib


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def num_threads() -> int:
    """Host threads the oracle's parallel loops use."""
    return int(_load().orc_num_threads())


def levels(n: int, bs: int) -> int:
    """Quadtree depth L: leaves live on a 2^L x 2^L grid with 2^L >= ceil(n/bs)."""
    nb = -(-n // bs)
    L = 0
    while (1 << L) < nb:
        L += 1
    return L


@dataclass
class LeafMatrix:
    """A quadtree matrix given by its non-null leaves."""
    n: int
    bs: int
    bi: np.ndarray  # int32 block row of each leaf
    bj: np.ndarray  # int32 block column
    data: np.ndarray  # float64 (m, bs, bs), row-major leaves
    sq: np.ndarray = field(default=None)  # squared Frobenius norm per leaf

    def __post_init__(self):
        self.bi = np.ascontiguousarray(self.bi, dtype=np.int32)
        self.bj = np.ascontiguousarray(self.bj, dtype=np.int32)
        self.data = np.ascontiguousarray(self.data, dtype=np.float64).reshape(-1, self.bs, self.bs)
        if self.sq is None:
            self.sq = leaf_sqnorms(self.data)

    @property
    def m(self) -> int:
        return len(self.bi)

    @property
    def L(self) -> int:
        return levels(self.n, self.bs)

    def keys(self) -> np.ndarray:
        return self.bi.astype(np.int64) * (1 << self.L) + self.bj


def leaf_sqnorms(data: np.ndarray) -> np.ndarray:
    """Squared Frobenius norm of each leaf, pairwise summation (Section 2)."""
    data = np.ascontiguousarray(data, dtype=np.float64)
    m = data.shape[0]
    bs = data.shape[1] if data.ndim == 3 else int(round(np.sqrt(data.shape[1])))
    out = np.empty(m, dtype=np.float64)
    _load().orc_leaf_sqnorms(m, bs, _p(data), _p(out))
    return out


def from_dense(a: np.ndarray, bs: int) -> LeafMatrix:
    """Leaves of a dense matrix; a leaf is kept iff it has a non-zero (Sec. 4.4)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = a.shape[0]
    lib = _load()
    m = lib.orc_leaves_from_dense(n, bs, _p(a), n, None, None, None)
    bi = np.empty(m, np.int32)
    bj = np.empty(m, np.int32)
    data = np.empty((m, bs, bs), np.float64)
    lib.orc_leaves_from_dense(n, bs, _p(a), n, _p(bi, ctypes.c_int32), _p(bj, ctypes.c_int32), _p(data))
    return LeafMatrix(n, bs, bi, bj, data)


def from_leaves(n: int, bs: int, bi, bj, data) -> LeafMatrix:
    """Leaf list -> LeafMatrix, dropping leaves that are identically zero."""
    data = np.ascontiguousarray(data, dtype=np.float64).reshape(-1, bs, bs)
    nz = np.any(data != 0.0, axis=(1, 2))
    return LeafMatrix(n, bs, np.asarray(bi)[nz], np.asarray(bj)[nz], data[nz])


def to_dense(M: LeafMatrix) -> np.ndarray:
    nb = -(-M.n // M.bs)
    full = np.zeros((nb * M.bs, nb * M.bs), dtype=np.float64)
    for q in range(M.m):
        r, c = M.bi[q] * M.bs, M.bj[q] * M.bs
        full[r:r + M.bs, c:c + M.bs] = M.data[q]
    return full[:M.n, :M.n]


def tree_norms(M: LeafMatrix):
    """Squared norms on every quadtree level (Section 2); -1 marks a null node.

    Returns a list: entry t is the 2^t x 2^t grid of level t (0 = root)."""
    L = M.L
    total = ((1 << (2 * (L + 1))) - 1) // 3
    grid = np.empty(total, dtype=np.float64)
    _load().orc_tree_norms(L, M.m, _p(M.bi, ctypes.c_int32), _p(M.bj, ctypes.c_int32), _p(M.sq), _p(grid))
    out = []
    for t in range(L + 1):
        off = ((1 << (2 * t)) - 1) // 3
        out.append(grid[off:off + (1 << (2 * t))].reshape(1 << t, 1 << t))
    return out, grid


def frob_norm(M: LeafMatrix) -> float:
    """||M||_F = sqrt of the root's squared norm (0 for the empty matrix)."""
    if M.m == 0:
        return 0.0
    grids, _ = tree_norms(M)
    return float(np.sqrt(grids[0][0, 0]))


def truncate_block(M: LeafMatrix, tau: float) -> LeafMatrix:
    """Block rule: drop a leaf iff its Frobenius norm sqrt(s) < tau."""
    keep = ~(np.sqrt(M.sq) < tau)
    return LeafMatrix(M.n, M.bs, M.bi[keep], M.bj[keep], M.data[keep], M.sq[keep])


def truncate_element(M: LeafMatrix, tau: float) -> LeafMatrix:
    """Element rule, Theorem 1 eq. (truncated matrices): a_ij -> 0 iff |a_ij| < tau;
    leaves left without a non-zero are removed (Section 4.4) and norms recomputed."""
    data = M.data.copy()
    data[np.abs(data) < tau] = 0.0
    return from_leaves(M.n, M.bs, M.bi, M.bj, data)


def morton(bi, bj) -> np.ndarray:
    """Morton code of leaf (row, col): bits interleaved, the row bit above the
    column bit (the order in which quadtree leaves are enumerated)."""
    code = np.zeros(len(bi), dtype=np.uint64)
    r = np.asarray(bi, dtype=np.uint64)
    c = np.asarray(bj, dtype=np.uint64)
    for b in range(16):
        code |= ((r >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
        code |= ((c >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
    return code


def truncate_error_controlled(M: LeafMatrix, tau: float) -> LeafMatrix:
    """Error-controlled rule (tau is an error budget; Section 1 cites this
    kind of truncation): visit the leaves by ascending squared norm (equal
    norms in Morton order), add their squared norms one by one, and drop every
    leaf whose running sum stays <= tau^2; so ||M - M~||_F <= tau and no more
    leaves can be dropped within the budget."""
    order = np.lexsort((morton(M.bi, M.bj), M.sq))
    run = np.cumsum(M.sq[order])
    k = int(np.sum(run <= tau * tau))
    keep = np.ones(M.m, dtype=bool)
    keep[order[:k]] = False
    return LeafMatrix(M.n, M.bs, M.bi[keep], M.bj[keep], M.data[keep], M.sq[keep])


def truncate(M: LeafMatrix, tau: float, rule: str = "block") -> LeafMatrix:
    if rule == "error":
        return truncate_error_controlled(M, tau)
    return truncate_block(M, tau) if rule == "block" else truncate_element(M, tau)


def _sort_ijk(ikj: np.ndarray) -> np.ndarray:
    if len(ikj) == 0:
        return ikj.reshape(0, 3)
    order = np.lexsort((ikj[:, 1], ikj[:, 2], ikj[:, 0]))  # by i, then j, then k
    return ikj[order]


def kept_flat(A: LeafMatrix, B: LeafMatrix, tau: float, mode: int) -> np.ndarray:
    """Kept leaf triples (i,k,j), flat: all non-null pairs passing the test."""
    assert A.n == B.n and A.bs == B.bs
    lib = _load()
    ob = np.argsort(B.bi, kind="stable")
    bbi, bbj, bsq = (np.ascontiguousarray(B.bi[ob]), np.ascontiguousarray(B.bj[ob]),
                     np.ascontiguousarray(B.sq[ob]))
    args = (A.m, _p(A.bi, ctypes.c_int32), _p(A.bj, ctypes.c_int32), _p(A.sq),
            B.m, _p(bbi, ctypes.c_int32), _p(bbj, ctypes.c_int32), _p(bsq), 1 << A.L, float(tau), int(mode))
    cnt = lib.orc_kept_flat(*args, None)
    out = np.empty((cnt, 3), np.int32)
    lib.orc_kept_flat(*args, _p(out, ctypes.c_int32))
    return _sort_ijk(out)


def kept_recursive(A: LeafMatrix, B: LeafMatrix, tau: float, mode: int) -> np.ndarray:
    """Kept leaf triples by literal recursion of Algorithm 1 over the quadtree."""
    assert A.n == B.n and A.bs == B.bs
    lib = _load()
    if A.m == 0 or B.m == 0:
        return np.zeros((0, 3), np.int32)
    _, ga = tree_norms(A)
    _, gb = tree_norms(B)
    cnt = lib.orc_kept_recursive(A.L, _p(ga), _p(gb), float(tau), int(mode), None)
    out = np.empty((cnt, 3), np.int32)
    lib.orc_kept_recursive(A.L, _p(ga), _p(gb), float(tau), int(mode), _p(out, ctypes.c_int32))
    return _sort_ijk(out)


def _index_of(M: LeafMatrix, rows, cols) -> np.ndarray:
    side = 1 << M.L
    keys = M.keys()
    order = np.argsort(keys, kind="stable")
    want = np.asarray(rows, np.int64) * side + np.asarray(cols, np.int64)
    pos = np.searchsorted(keys[order], want)
    pos = np.minimum(pos, len(order) - 1)
    idx = order[pos]
    assert np.all(keys[idx] == want), "triple refers to a null leaf"
    return idx.astype(np.int64)


def product(A: LeafMatrix, B: LeafMatrix, ikj: np.ndarray) -> LeafMatrix:
    """C leaves from a kept-triple list sorted by (i, j, k): C_ij = sum_k A_ik B_kj.

    Every (i,j) with at least one kept triple is a leaf of C (the output
    quadtree is built in advance from the kept set, Section 4.4)."""
    ikj = _sort_ijk(np.asarray(ikj, np.int32).reshape(-1, 3))
    bs = A.bs
    if len(ikj) == 0:
        return LeafMatrix(A.n, bs, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros((0, bs, bs)))
    i, k, j = ikj[:, 0], ikj[:, 1], ikj[:, 2]
    start = np.concatenate([[True], (i[1:] != i[:-1]) | (j[1:] != j[:-1])])
    gstart = np.flatnonzero(start)
    cptr = np.concatenate([gstart, [len(ikj)]]).astype(np.int64)
    pa = _index_of(A, i, k)
    pb = _index_of(B, k, j)
    nc = len(gstart)
    cdata = np.empty((nc, bs, bs), np.float64)
    _load().orc_leaf_products(bs, _p(A.data), _p(B.data), nc, _p(cptr, ctypes.c_int64),
                              _p(pa, ctypes.c_int64), _p(pb, ctypes.c_int64), _p(cdata))
    return LeafMatrix(A.n, bs, i[gstart], j[gstart], cdata)


def multiply(A: LeafMatrix, B: LeafMatrix, tau: float, mode: int, rule: str = "block"):
    """Approximate product with one of the paper's three methods.

    truncate: C~ = A~ B~ (Theorem 1; inputs truncated, every pair multiplied)
    spamm:    C- = SpAMM(A, B, tau) (Algorithm 1 / Theorem 2)
    combined: C^ = SpAMM(A~, B~, tau), same tau for both steps (Theorem 3)
    Returns (C, kept triples)."""
    if mode in (TRUNCATE, COMBINED):
        A = truncate(A, tau, rule)
        B = truncate(B, tau, rule)
    ikj = kept_flat(A, B, tau, mode)
    return product(A, B, ikj), ikj


def exact(A: LeafMatrix, B: LeafMatrix) -> LeafMatrix:
    """The exact product AB over every pair of non-null leaves."""
    return product(A, B, kept_flat(A, B, 0.0, TRUNCATE))


def error(X: LeafMatrix, Y: LeafMatrix) -> float:
    """||X - Y||_F, a merged walk over the two leaf sets (a leaf missing on one
    side counts as zero)."""
    assert X.bs == Y.bs
    side = 1 << max(X.L, Y.L)
    kx = X.bi.astype(np.int64) * side + X.bj
    ky = Y.bi.astype(np.int64) * side + Y.bj
    common, ix, iy = np.intersect1d(kx, ky, assume_unique=True, return_indices=True)
    lib = _load()
    total = 0.0
    for a, b in zip(ix, iy):
        total += lib.orc_leaf_diff_sumsq(X.bs, _p(np.ascontiguousarray(X.data[a])),
                                         _p(np.ascontiguousarray(Y.data[b])))
    onlyx = np.setdiff1d(np.arange(X.m), ix)
    onlyy = np.setdiff1d(np.arange(Y.m), iy)
    total += float(np.sum(X.sq[onlyx])) + float(np.sum(Y.sq[onlyy]))
    return float(np.sqrt(total))


def skipped_bound(A: LeafMatrix, B: LeafMatrix, tau: float, mode: int, rule: str = "block") -> float:
    """sqrt(sum_ij beta_ij^2), beta_ij = sum over the skipped products of
    ||A_ik|| ||B_kj|| (original norms); for the element rule the truncated
    but kept products add ||A - A~|| ||B|| + ||A~|| ||B - B~||.

    By the triangle inequality and submultiplicativity of the Frobenius norm,
    ||AB - C||_F <= this bound (up to rounding)."""
    cand = kept_flat(A, B, 0.0, TRUNCATE)
    if mode in (TRUNCATE, COMBINED):
        At, Bt = truncate(A, tau, rule), truncate(B, tau, rule)
    else:
        At, Bt = A, B
    kept = kept_flat(At, Bt, tau, mode)
    side = 1 << A.L
    ck = (cand[:, 0].astype(np.int64) * side + cand[:, 2]) * side + cand[:, 1]
    kk = (kept[:, 0].astype(np.int64) * side + kept[:, 2]) * side + kept[:, 1]
    is_kept = np.isin(ck, kk)
    na = np.sqrt(A.sq[_index_of(A, cand[:, 0], cand[:, 1])])
    nb = np.sqrt(B.sq[_index_of(B, cand[:, 1], cand[:, 2])])
    term = np.where(is_kept, 0.0, na * nb)
    if rule == "element" and mode in (TRUNCATE, COMBINED) and np.any(is_kept):
        kc = cand[is_kept]
        ia, ib = _index_of(A, kc[:, 0], kc[:, 1]), _index_of(B, kc[:, 1], kc[:, 2])
        ita, itb = _index_of(At, kc[:, 0], kc[:, 1]), _index_of(Bt, kc[:, 1], kc[:, 2])
        da = np.sqrt(leaf_sqnorms(A.data[ia] - At.data[ita]))
        db = np.sqrt(leaf_sqnorms(B.data[ib] - Bt.data[itb]))
        term[is_kept] = da * nb[is_kept] + np.sqrt(At.sq[ita]) * db
    cij = cand[:, 0].astype(np.int64) * side + cand[:, 2]
    _, inv = np.unique(cij, return_inverse=True)
    beta = np.bincount(inv, weights=term)
    return float(np.sqrt(np.sum(beta * beta)))
