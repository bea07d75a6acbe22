"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library.

Only input generation lives here: matrices with exponential decay
|a_ij| <= c exp(-alpha d(i,j)) (Definition 1 of the paper) on the 1-D index
line (the model problem of Section 5.3) or on a 3-D unit lattice in Morton
order (the stand-in for the water-cluster overlap matrices of Section 5.4).
The element rule is in ``decaygen.h``; this module builds the host copy of it
and wraps it with ctypes.  Nothing here computes norms, thresholds or products.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None

KIND_1D = 0
KIND_3D = 1
LAW_EXPONENTIAL = 0
LAW_ALGEBRAIC = 1


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("kind", ctypes.c_int32), ("law", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("c", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


@dataclass(frozen=True)
class DecayParams:
    """One synthetic decay matrix: a_ij = c u_ij exp(-alpha d(i,j)) (law 0) or
    c u_ij / (1 + d(i,j))^alpha for integer alpha (law 1); |a| < cutoff -> 0."""
    n: int
    kind: int = KIND_3D
    alpha: float = 1.0
    seed: int = 1
    c: float = 1.0
    cutoff: float = 1e-16
    law: int = 0

    def as_c(self) -> _Params:
        return _Params(self.n, self.kind, self.law, self.alpha, self.c, self.cutoff, self.seed)


def build(force: bool = False) -> str:
    """Compile libsynth.so (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "synth_host.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "decaygen.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lib.synth_fill_dense.argtypes = [P, dp]
        lib.synth_fill_leaves.argtypes = [P, ctypes.c_int32, ctypes.c_int64, ip, ip, dp]
        lib.synth_exp_nonpos_host.argtypes = [ctypes.c_double]
        lib.synth_exp_nonpos_host.restype = ctypes.c_double
        lib.synth_uniform_host.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
        lib.synth_uniform_host.restype = ctypes.c_double
        lib.synth_distance_host.argtypes = [P, ctypes.c_int64, ctypes.c_int64]
        lib.synth_distance_host.restype = ctypes.c_double
        lib.synth_lattice_point_host.argtypes = [ctypes.c_int64, ip]
        lib.synth_leaf_bound_host.argtypes = [P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]
        lib.synth_leaf_bound_host.restype = ctypes.c_double
        lib.synth_leaf_bounds_row.argtypes = [P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.POINTER(ctypes.c_int64), dp]
        lib.synth_block_sparse.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                           ip, ip, dp]
        lib.synth_block_sparse.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def dense(p: DecayParams) -> np.ndarray:
    """The full n x n matrix (small n only)."""
    out = np.empty((p.n, p.n), dtype=np.float64)
    cp = p.as_c()
    _load().synth_fill_dense(ctypes.byref(cp), _ptr(out, ctypes.c_double))
    return out


def leaves(p: DecayParams, bs: int, bi, bj) -> np.ndarray:
    """Leaf blocks (len, bs, bs): rows bi*bs.., cols bj*bs.., zero past n."""
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    out = np.empty((len(bi), bs, bs), dtype=np.float64)
    cp = p.as_c()
    _load().synth_fill_leaves(ctypes.byref(cp), bs, len(bi), _ptr(bi, ctypes.c_int32),
                              _ptr(bj, ctypes.c_int32), _ptr(out, ctypes.c_double))
    return out


def exp_nonpos(x: float) -> float:
    return _load().synth_exp_nonpos_host(float(x))


def uniform(seed: int, i: int, j: int) -> float:
    return _load().synth_uniform_host(seed, i, j)


def distance(p: DecayParams, i: int, j: int) -> float:
    cp = p.as_c()
    return _load().synth_distance_host(ctypes.byref(cp), i, j)


def leaf_bound(p: DecayParams, bs: int, bi: int, bj: int) -> float:
    """Upper bound of |a_ij| over leaf (bi, bj)."""
    cp = p.as_c()
    return _load().synth_leaf_bound_host(ctypes.byref(cp), bs, bi, bj)


def leaf_bounds_row(p: DecayParams, bs: int, bi: int, bj) -> np.ndarray:
    """leaf_bound(p, bs, bi, bj[q]) for every q, in one call."""
    bj = np.ascontiguousarray(bj, dtype=np.int64)
    out = np.empty(len(bj), dtype=np.float64)
    cp = p.as_c()
    _load().synth_leaf_bounds_row(ctypes.byref(cp), bs, int(bi), len(bj), _ptr(bj, ctypes.c_int64),
                                  _ptr(out, ctypes.c_double))
    return out


def lattice_point(i: int):
    xyz = np.zeros(3, dtype=np.int32)
    _load().synth_lattice_point_host(i, _ptr(xyz, ctypes.c_int32))
    return tuple(int(v) for v in xyz)


def spectral_bound(p: DecayParams) -> float:
    """An upper bound of ||A||_2 for the matrices of `p`: the largest absolute
    row sum (Gershgorin) is at most |c| sum_j f(d(i, j)) over lattice points j,
    f the decay factor.  Exponential law: over all integer offsets (1-D: the
    closed form coth(alpha/2); 3-D: offsets within radius 48/alpha, the rest
    below 1e-12 relative).  Algebraic law: over the offsets that fit the
    matrix (|k| < n in 1-D; within the bounding box of the n lattice points in
    3-D).  Enlarged by 1e-9 relative."""
    a = float(p.alpha)
    if p.law == LAW_ALGEBRAIC:
        k = max(1, int(a))
        if p.kind == KIND_1D:
            off = np.arange(-(p.n - 1), p.n, dtype=np.float64)
            s = float(np.sum((1.0 + np.abs(off)) ** -k))
        else:
            i = np.arange(p.n, dtype=np.uint64)
            box = []
            for ax in range(3):  # bounding box of the points (Morton order, x first)
                v = np.zeros(p.n, dtype=np.uint64)
                for bit in range(21):
                    v |= ((i >> np.uint64(3 * bit + ax)) & np.uint64(1)) << np.uint64(bit)
                box.append(int(v.max()) + 1)
            r = [np.arange(-(m - 1), m, dtype=np.float64) for m in box]
            d = np.sqrt(r[0][:, None, None] ** 2 + r[1][None, :, None] ** 2 + r[2][None, None, :] ** 2)
            s = float(np.sum((1.0 + d) ** -k))
    elif p.kind == KIND_1D:
        s = 1.0 + 2.0 * math.exp(-a) / (1.0 - math.exp(-a))
    else:
        R = int(math.ceil(48.0 / a))
        r = np.arange(-R, R + 1, dtype=np.float64)
        d2 = r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2
        s = float(np.sum(np.exp(-a * np.sqrt(d2))))
    return abs(p.c) * s * (1.0 + 1e-9)


def block_sparse(n: int, bs: int, fill: float, seed: int = 1):
    """Random block-sparse n x n matrix (Section 5.2's leaf-library benchmark):
    each bs x bs block non-zero with probability `fill`, elements U[-1, 1)
    (zero past row / column n).
    Returns (bi, bj, data) with data of shape (count, bs, bs)."""
    lib = _load()
    cnt = lib.synth_block_sparse(n, bs, float(fill), seed, None, None, None)
    bi = np.empty(cnt, np.int32)
    bj = np.empty(cnt, np.int32)
    data = np.empty((cnt, bs, bs), np.float64)
    if cnt:
        lib.synth_block_sparse(n, bs, float(fill), seed, _ptr(bi, ctypes.c_int32), _ptr(bj, ctypes.c_int32),
                               _ptr(data, ctypes.c_double))
    return bi, bj, data


def sublattice_parity(n: int) -> np.ndarray:
    """(x + y + z) mod 2 of the 3-D lattice points 0..n-1 (Morton order, x in
    bit 0, y in bit 1, z in bit 2 of each coordinate triple): int8 array."""
    i = np.arange(n, dtype=np.int64)
    return ((i ^ (i >> 1) ^ (i >> 2)) & 1).astype(np.int8)


def onsite_blocks(n: int, bs: int, delta: float):
    """Diagonal on-site term of a two-sublattice insulator on the 3-D lattice:
    -delta on the points with x + y + z even, +delta on the odd ones.  Added
    to a decay matrix V of norm below delta it opens a gap around 0 in the
    spectrum, so the projector onto the negative eigenvalues (the density
    matrix at half filling) decays exponentially, as for the insulating
    systems the paper's purification application treats.
    Returns (bi, bj, data) of the ceil(n / bs) diagonal leaves, and the count
    of -delta points (the number of occupied states)."""
    par = sublattice_parity(n)
    nb = -(-n // bs)
    data = np.zeros((nb, bs, bs))
    diag = np.zeros(nb * bs)
    diag[:n] = np.where(par == 0, -delta, delta)
    r = np.arange(bs)
    data[:, r, r] = diag.reshape(nb, bs)
    idx = np.arange(nb, dtype=np.int32)
    return idx, idx.copy(), data, int(np.count_nonzero(par == 0))


# The synthetic workloads (sizes and decay of the paper's model problem and
# of the large chemical systems it stands in for).
def model_1d(n=2048, alpha=0.05, seed=1) -> DecayParams:
    return DecayParams(n=n, kind=KIND_1D, alpha=alpha, seed=seed)


def lattice_3d(n=65536, alpha=1.0, seed=1) -> DecayParams:
    return DecayParams(n=n, kind=KIND_3D, alpha=alpha, seed=seed)


def algebraic_3d(n=65536, p=4, seed=1) -> DecayParams:
    """3-D lattice with algebraic decay |a_ij| <= (1 + d)^-p."""
    return DecayParams(n=n, kind=KIND_3D, alpha=float(p), seed=seed, law=LAW_ALGEBRAIC)
