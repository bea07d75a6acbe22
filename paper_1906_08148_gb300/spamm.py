"""ctypes binding of libspamm (include/spamm.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python
objects (numpy arrays for host memory, torch CUDA tensors for device memory)
to pointers and sizes, calls the C entry point of the same name and turns a
non-OK status into SpammError.  PyTorch provides device memory and streams:
a Context can run on a torch CUDA stream and allocate through torch's caching
allocator.  There is no CPU fallback: if libspamm.so is missing the import of
the library fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libspamm.so")

OK, E_INVALID_ARG, E_SHAPE, E_NONFINITE, E_OOM, E_CUDA, E_TIMEOUT, E_BUSY, E_CAPACITY, E_UNSUPPORTED = range(10)
MODE_TRUNCATE, MODE_SPAMM, MODE_COMBINED = 0, 1, 2
MODES = {"truncate": MODE_TRUNCATE, "spamm": MODE_SPAMM, "combined": MODE_COMBINED}
TRUNC_BLOCK_FROB, TRUNC_ELEMENT, TRUNC_ERROR_CONTROL = 0, 1, 2
RULES = {"block": TRUNC_BLOCK_FROB, "element": TRUNC_ELEMENT, "error": TRUNC_ERROR_CONTROL}
PREC_FP64, PREC_BF16_SPLIT, PREC_FP16_SCALED, PREC_BF16_SPLIT4 = 0, 1, 2, 3
PRECS = {"fp64": PREC_FP64, "bf16_split": PREC_BF16_SPLIT, "fp16_scaled": PREC_FP16_SCALED,
         "bf16_split4": PREC_BF16_SPLIT4}
MAX_LEVELS = 17

# every entry point of include/spamm.h
ENTRY_POINTS = (
    "spamm_create", "spamm_destroy", "spamm_set_stream", "spamm_set_allocator", "spamm_sync", "spamm_last_error",
    "spamm_from_dense", "spamm_from_blocks", "spamm_from_coo", "spamm_generate", "spamm_truncate", "spamm_release",
    "spamm_multiply", "spamm_kept_tasks", "spamm_frob_norm", "spamm_error", "spamm_mat_info", "spamm_to_dense",
    "spamm_to_blocks", "spamm_gather_leaves", "spamm_level_norms", "spamm_leaf_sqnorms_noalloc",
    "spamm_plan_create", "spamm_plan_info", "spamm_execute", "spamm_plan_release", "spamm_set_gemm_sms",
    "spamm_set_exec_graph", "spamm_set_claim_order", "spamm_add", "spamm_identity", "spamm_trace", "spamm_check_timeout_path", "spamm_trim",
    "spamm_set_symmetric", "spamm_job_begin", "spamm_job_info", "spamm_run", "spamm_job_finish",
    "spamm_job_release", "spamm_exec_graph_info",
)
NOALLOC_MAX_LEAVES = 1 << 24


class SpammError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libspamm status {status}: {message}")
        self.status = status


class GenParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("kind", ctypes.c_int32), ("law", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("c", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int64 * MAX_LEVELS), ("n_kept_level", ctypes.c_int64 * MAX_LEVELS),
                ("n_kept", ctypes.c_int64), ("n_borderline", ctypes.c_int64), ("n_c_leaves", ctypes.c_int64),
                ("n_a_leaves", ctypes.c_int64), ("n_b_leaves", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("bs", ctypes.c_int32), ("kept_flops", ctypes.c_double), ("ms_truncate", ctypes.c_double),
                ("ms_tasks", ctypes.c_double), ("ms_gemm", ctypes.c_double), ("ms_cnorm", ctypes.c_double),
                ("n_launches", ctypes.c_int64), ("ms_prep", ctypes.c_double), ("n_steps", ctypes.c_int64),
                ("executed_flops", ctypes.c_double), ("terms_shared", ctypes.c_int64)]

    def as_dict(self) -> dict:
        L = self.levels
        return {"n_candidates": list(self.n_candidates[1:L + 1]), "n_kept_level": list(self.n_kept_level[1:L + 1]),
                "n_kept": self.n_kept, "n_borderline": self.n_borderline, "n_c_leaves": self.n_c_leaves,
                "n_a_leaves": self.n_a_leaves, "n_b_leaves": self.n_b_leaves, "levels": L, "bs": self.bs,
                "kept_flops": self.kept_flops, "ms_truncate": self.ms_truncate, "ms_tasks": self.ms_tasks,
                "ms_gemm": self.ms_gemm, "ms_cnorm": self.ms_cnorm, "n_launches": self.n_launches,
                "ms_prep": self.ms_prep, "n_steps": self.n_steps, "executed_flops": self.executed_flops,
                "terms_shared": self.terms_shared}


_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_lib = None


def load(path: str = LIB_PATH):
    """Load libspamm.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libspamm.so not found at {path}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    L = ctypes.CDLL(path)
    vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    pi32, pi64, pf64, pu32 = (ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint32))
    sig = {
        "spamm_create": [ctypes.c_int, vp, ctypes.POINTER(vp)],
        "spamm_destroy": [vp],
        "spamm_set_stream": [vp, vp],
        "spamm_set_allocator": [vp, _ALLOC_T, _FREE_T, vp],
        "spamm_sync": [vp],
        "spamm_trim": [vp],
        "spamm_from_dense": [vp, i64, vp, i64, ctypes.c_int, ctypes.c_int, f64, ctypes.c_int, ctypes.POINTER(vp)],
        "spamm_from_blocks": [vp, i64, ctypes.c_int, i64, vp, vp, vp, ctypes.c_int, f64, ctypes.c_int,
                              ctypes.POINTER(vp)],
        "spamm_from_coo": [vp, i64, i64, vp, vp, vp, ctypes.c_int, ctypes.c_int, f64, ctypes.c_int,
                           ctypes.POINTER(vp)],
        "spamm_generate": [vp, ctypes.POINTER(GenParams), ctypes.c_int, f64, ctypes.c_int, ctypes.POINTER(vp)],
        "spamm_truncate": [vp, vp, f64, ctypes.c_int, ctypes.POINTER(vp)],
        "spamm_release": [vp],
        "spamm_multiply": [vp, vp, vp, f64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(Stats)],
        "spamm_kept_tasks": [vp, vp, vp, f64, ctypes.c_int, vp, i64, pi64],
        "spamm_frob_norm": [vp, vp, pf64],
        "spamm_error": [vp, vp, vp, pf64],
        "spamm_mat_info": [vp, pi64, pi32, pi32, pi64],
        "spamm_set_symmetric": [vp, ctypes.c_int],
        "spamm_job_begin": [vp, vp, ctypes.POINTER(vp)],
        "spamm_job_info": [vp, pi64, pi64, pf64, pf64],
        "spamm_run": [vp, i64, ctypes.POINTER(vp), pf64, pi64, pf64],
        "spamm_job_finish": [vp, vp, ctypes.POINTER(vp), ctypes.POINTER(Stats)],
        "spamm_job_release": [vp],
        "spamm_exec_graph_info": [vp, pi64, pi64],
        "spamm_to_dense": [vp, vp, vp, i64, ctypes.c_int],
        "spamm_to_blocks": [vp, vp, vp, vp, vp, vp, i64, ctypes.c_int],
        "spamm_level_norms": [vp, vp, ctypes.c_int, vp, vp, i64, pi64],
        "spamm_gather_leaves": [vp, vp, i64, vp, vp, vp, vp, ctypes.c_int],
        "spamm_leaf_sqnorms_noalloc": [vp, i64, ctypes.c_int, vp, vp, vp],
        "spamm_plan_create": [vp, vp, vp, f64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
        "spamm_plan_info": [vp, pi64, pi64, pi64, pi64],
        "spamm_execute": [vp, i64, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(Stats)],
        "spamm_plan_release": [vp],
        "spamm_set_gemm_sms": [vp, ctypes.c_int],
        "spamm_set_exec_graph": [vp, ctypes.c_int],
        "spamm_set_claim_order": [vp, ctypes.c_int],
        "spamm_add": [vp, f64, vp, f64, vp, ctypes.POINTER(vp)],
        "spamm_identity": [vp, i64, ctypes.c_int, ctypes.POINTER(vp)],
        "spamm_trace": [vp, vp, pf64],
        "spamm_check_timeout_path": [vp, i64],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.spamm_last_error.argtypes = [vp]
    L.spamm_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(ctx_handle, status: int):
    if status != OK:
        msg = load().spamm_last_error(ctx_handle).decode() if ctx_handle else ""
        raise SpammError(status, msg)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        assert x.is_contiguous(), "tensor must be contiguous"
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), 0, a


class Context:
    """A libspamm context on one CUDA device and stream (spamm_create)."""

    def __init__(self, device: int = 0, stream=None, torch_allocator: bool = False):
        self._lib = load()
        s = stream.cuda_stream if (stream is not None and hasattr(stream, "cuda_stream")) else stream
        h = ctypes.c_void_p()
        st = self._lib.spamm_create(device, ctypes.c_void_p(s or 0), ctypes.byref(h))
        if st != OK:
            raise SpammError(st, "spamm_create failed")
        self.handle = h
        self.device = device
        self._callbacks = None
        if torch_allocator:
            spamm_set_allocator(self, "torch")

    def close(self):
        if self.handle:
            _check(self.handle, self._lib.spamm_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Matrix:
    """An immutable quadtree matrix handle (released on close or garbage collection)."""

    def __init__(self, ctx: Context, handle: ctypes.c_void_p):
        self.ctx = ctx
        self.handle = handle

    def info(self) -> dict:
        n, bs, L, m = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(self.ctx.handle, load().spamm_mat_info(self.handle, ctypes.byref(n), ctypes.byref(bs),
                                                      ctypes.byref(L), ctypes.byref(m)))
        return {"n": n.value, "bs": bs.value, "levels": L.value, "nleaves": m.value}

    def set_symmetric(self, symmetric: bool = True):
        """spamm_set_symmetric: mark (or unmark) the matrix as equal to its transpose."""
        _check(self.ctx.handle, load().spamm_set_symmetric(self.handle, int(bool(symmetric))))

    def close(self):
        if self.handle:
            load().spamm_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _new(ctx, fn, *args) -> Matrix:
    out = ctypes.c_void_p()
    _check(ctx.handle, fn(ctx.handle, *args, ctypes.byref(out)))
    return Matrix(ctx, out)


def spamm_set_allocator(ctx: Context, which: Optional[str] = "torch"):
    """Route the library's device allocations through torch's caching allocator (or back to cudaMallocAsync)."""
    lib = load()
    if which is None:
        _check(ctx.handle, lib.spamm_set_allocator(ctx.handle, _ALLOC_T(), _FREE_T(), None))
        ctx._callbacks = None
        return
    import torch

    dev = ctx.device

    def _alloc(nbytes, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, torch.cuda.current_stream(dev))
        except Exception:
            return None

    def _free(p, _user):
        torch.cuda.caching_allocator_delete(p)

    cbs = (_ALLOC_T(_alloc), _FREE_T(_free))
    _check(ctx.handle, lib.spamm_set_allocator(ctx.handle, cbs[0], cbs[1], None))
    ctx._callbacks = cbs


def spamm_sync(ctx: Context):
    _check(ctx.handle, load().spamm_sync(ctx.handle))


def spamm_trim(ctx: Context):
    """Return the device memory the stream-ordered pool keeps cached to the driver (spamm_trim)."""
    _check(ctx.handle, load().spamm_trim(ctx.handle))


def spamm_from_dense(ctx: Context, a, bs: int, tau: float = 0.0, rule: str = "block") -> Matrix:
    n = a.shape[0]
    p, dev, keep = _ptr(a, np.float64)
    lda = a.stride(0) if _is_torch(a) else n
    return _new(ctx, load().spamm_from_dense, n, p, lda, dev, bs, float(tau), RULES[rule])


def spamm_from_blocks(ctx: Context, n: int, bs: int, bi, bj, payload, tau: float = 0.0, rule: str = "block") -> Matrix:
    pbi, dev, k1 = _ptr(bi, np.int32)
    pbj, _, k2 = _ptr(bj, np.int32)
    pp, _, k3 = _ptr(payload, np.float64)
    return _new(ctx, load().spamm_from_blocks, n, bs, len(bi), pbi, pbj, pp, dev, float(tau), RULES[rule])


def spamm_from_coo(ctx: Context, n: int, row, col, val, bs: int, tau: float = 0.0, rule: str = "block") -> Matrix:
    pr, dev, k1 = _ptr(row, np.int64)
    pc, _, k2 = _ptr(col, np.int64)
    pv, _, k3 = _ptr(val, np.float64)
    return _new(ctx, load().spamm_from_coo, n, len(row), pr, pc, pv, dev, bs, float(tau), RULES[rule])


def spamm_generate(ctx: Context, params, bs: int, tau: float = 0.0, rule: str = "block") -> Matrix:
    """params: any object with n, kind, alpha, c, cutoff, seed (e.g. synth.DecayParams)."""
    gp = GenParams(int(params.n), int(params.kind), int(getattr(params, "law", 0)), float(params.alpha),
                   float(params.c), float(params.cutoff), int(params.seed))
    return _new(ctx, load().spamm_generate, ctypes.byref(gp), bs, float(tau), RULES[rule])


def spamm_truncate(ctx: Context, m: Matrix, tau: float, rule: str = "block") -> Matrix:
    return _new(ctx, load().spamm_truncate, m.handle, float(tau), RULES[rule])


def spamm_release(m: Matrix):
    m.close()


def spamm_multiply(ctx: Context, A: Matrix, B: Matrix, tau: float, mode: str = "spamm", prec: str = "fp64",
                   stats: bool = False):
    out = ctypes.c_void_p()
    st = Stats()
    _check(ctx.handle, load().spamm_multiply(ctx.handle, A.handle, B.handle, float(tau), MODES[mode], PRECS[prec],
                                             ctypes.byref(out), ctypes.byref(st)))
    C = Matrix(ctx, out)
    return (C, st.as_dict()) if stats else C


def spamm_kept_tasks(ctx: Context, A: Matrix, B: Matrix, tau: float, mode: str = "spamm") -> np.ndarray:
    lib = load()
    cnt = ctypes.c_int64()
    st = lib.spamm_kept_tasks(ctx.handle, A.handle, B.handle, float(tau), MODES[mode], None, 0, ctypes.byref(cnt))
    if st not in (OK, E_CAPACITY):
        _check(ctx.handle, st)
    out = np.empty((cnt.value, 3), np.int32)
    if cnt.value:
        _check(ctx.handle, lib.spamm_kept_tasks(ctx.handle, A.handle, B.handle, float(tau), MODES[mode],
                                                out.ctypes.data_as(ctypes.c_void_p), cnt.value, ctypes.byref(cnt)))
    return out


def spamm_frob_norm(ctx: Context, m: Matrix) -> float:
    v = ctypes.c_double()
    _check(ctx.handle, load().spamm_frob_norm(ctx.handle, m.handle, ctypes.byref(v)))
    return v.value


def spamm_error(ctx: Context, X: Matrix, Y: Matrix) -> float:
    v = ctypes.c_double()
    _check(ctx.handle, load().spamm_error(ctx.handle, X.handle, Y.handle, ctypes.byref(v)))
    return v.value


def spamm_to_dense(ctx: Context, m: Matrix, out=None):
    n = m.info()["n"]
    if out is None:
        out = np.empty((n, n), np.float64)
    p, dev, keep = _ptr(out, np.float64)
    ld = out.stride(0) if _is_torch(out) else n
    if not _is_torch(out):
        assert out.flags["C_CONTIGUOUS"] and out.dtype == np.float64
        p = out.ctypes.data_as(ctypes.c_void_p)
    _check(ctx.handle, load().spamm_to_dense(ctx.handle, m.handle, p, ld, dev))
    return out


def spamm_to_blocks(ctx: Context, m: Matrix, payload: bool = True, out=None):
    """(bi, bj, payload (m, bs, bs) or None, sq) on the host, leaves in Morton order.

    `out` may supply preallocated host arrays (bi, bj, payload, sq), e.g. pinned."""
    info = m.info()
    nl, bs = info["nleaves"], info["bs"]
    if out is not None:
        bi, bj, pay, sq = out
        assert len(bi) >= nl and len(bj) >= nl and len(sq) >= nl and (pay is None or len(pay) >= nl)
        payload = pay is not None
    else:
        bi = np.empty(nl, np.int32)
        bj = np.empty(nl, np.int32)
        sq = np.empty(nl, np.float64)
        pay = np.empty((nl, bs, bs), np.float64) if payload else None
    vp = ctypes.c_void_p
    _check(ctx.handle, load().spamm_to_blocks(
        ctx.handle, m.handle, bi.ctypes.data_as(vp), bj.ctypes.data_as(vp),
        pay.ctypes.data_as(vp) if payload else None, sq.ctypes.data_as(vp), nl, 0))
    return bi, bj, pay, sq


def spamm_level_norms(ctx: Context, m: Matrix, level: int):
    """(codes uint32, squared norms) of one quadtree level, Morton order."""
    lib = load()
    cnt = ctypes.c_int64()
    st = lib.spamm_level_norms(ctx.handle, m.handle, level, None, None, 0, ctypes.byref(cnt))
    if st not in (OK, E_CAPACITY):
        _check(ctx.handle, st)
    codes = np.empty(cnt.value, np.uint32)
    sq = np.empty(cnt.value, np.float64)
    if cnt.value:
        vp = ctypes.c_void_p
        _check(ctx.handle, lib.spamm_level_norms(ctx.handle, m.handle, level, codes.ctypes.data_as(vp),
                                                 sq.ctypes.data_as(vp), cnt.value, ctypes.byref(cnt)))
    return codes, sq


def spamm_gather_leaves(ctx: Context, m: Matrix, bi, bj):
    """(payload (nq, bs, bs), found (nq,)) for the leaves at (bi[q], bj[q]), host arrays."""
    bs = m.info()["bs"]
    bi = np.ascontiguousarray(bi, np.int32)
    bj = np.ascontiguousarray(bj, np.int32)
    out = np.empty((len(bi), bs, bs), np.float64)
    found = np.empty(len(bi), np.int32)
    vp = ctypes.c_void_p
    _check(ctx.handle, load().spamm_gather_leaves(ctx.handle, m.handle, len(bi), bi.ctypes.data_as(vp),
                                                  bj.ctypes.data_as(vp), out.ctypes.data_as(vp),
                                                  found.ctypes.data_as(vp), 0))
    return out, found.astype(bool)


def spamm_leaf_sqnorms_noalloc(payload, nleaves: int, bs: int, sq_out, total_out, stream=None) -> int:
    """Allocation-free leaf norms: raw device pointers (ints) or CUDA tensors in,
    the C status code out (OK = 0).  See include/spamm.h.

    Tensors must be contiguous CUDA float64 tensors holding at least
    nleaves * bs * bs (payload), nleaves (sq_out) and 1 (total_out) elements;
    anything else raises ValueError before the library is called.  Raw
    pointers are passed through unchecked (the library refuses misaligned ones)."""
    need = {"payload": int(nleaves) * int(bs) * int(bs), "sq_out": int(nleaves), "total_out": 1}

    def addr(name, x):
        if x is None:
            return None
        if _is_torch(x):
            if not x.is_cuda or str(x.dtype) != "torch.float64":
                raise ValueError(f"{name} must be a CUDA float64 tensor")
            if not x.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
            if x.numel() < need[name]:
                raise ValueError(f"{name} holds {x.numel()} elements, fewer than {need[name]}")
            return ctypes.c_void_p(x.data_ptr())
        return ctypes.c_void_p(int(x))
    s = stream.cuda_stream if (stream is not None and hasattr(stream, "cuda_stream")) else stream
    return load().spamm_leaf_sqnorms_noalloc(addr("payload", payload), int(nleaves), int(bs),
                                              addr("sq_out", sq_out), addr("total_out", total_out),
                                              ctypes.c_void_p(s or 0))


class Plan:
    """First phase of a multiplication (spamm_plan_create): truncation, task list, operand terms."""

    def __init__(self, ctx: Context, handle: ctypes.c_void_p):
        self.ctx = ctx
        self.handle = handle

    def info(self) -> dict:
        k, c, pb, eb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self.ctx.handle, load().spamm_plan_info(self.handle, ctypes.byref(k), ctypes.byref(c),
                                                       ctypes.byref(pb), ctypes.byref(eb)))
        return {"n_kept": k.value, "n_c_leaves": c.value, "plan_bytes": pb.value, "exec_bytes": eb.value}

    def close(self):
        if self.handle:
            load().spamm_plan_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spamm_plan_create(ctx: Context, A: Matrix, B: Matrix, tau: float, mode: str = "spamm",
                      prec: str = "fp64") -> Plan:
    out = ctypes.c_void_p()
    _check(ctx.handle, load().spamm_plan_create(ctx.handle, A.handle, B.handle, float(tau), MODES[mode],
                                                PRECS[prec], ctypes.byref(out)))
    return Plan(ctx, out)


def spamm_plan_info(plan: Plan) -> dict:
    return plan.info()


def spamm_plan_release(plan: Plan):
    plan.close()


def spamm_execute(ctx: Context, plans, stats: bool = False):
    """Run the leaf products of all plans in one persistent launch; returns the outputs (and stats)."""
    n = len(plans)
    arr = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    outs = (ctypes.c_void_p * n)()
    sts = (Stats * n)()
    _check(ctx.handle, load().spamm_execute(ctx.handle, n, arr, outs, sts))
    Cs = [Matrix(ctx, ctypes.c_void_p(outs[i])) for i in range(n)]
    return (Cs, [s.as_dict() for s in sts]) if stats else Cs


class Job:
    """The execute phase of a plan in slices (spamm_job_begin): its units run in spamm_run calls."""

    def __init__(self, ctx: Context, handle: ctypes.c_void_p, plan: "Plan"):
        self.ctx = ctx
        self.handle = handle
        self.plan = plan  # the plan must outlive the job

    def info(self) -> dict:
        u, d, w, wd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(self.ctx.handle, load().spamm_job_info(self.handle, ctypes.byref(u), ctypes.byref(d),
                                                      ctypes.byref(w), ctypes.byref(wd)))
        return {"units": u.value, "units_done": d.value, "work": w.value, "work_done": wd.value}

    def close(self):
        if self.handle:
            load().spamm_job_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spamm_job_begin(ctx: Context, plan: "Plan") -> Job:
    out = ctypes.c_void_p()
    _check(ctx.handle, load().spamm_job_begin(ctx.handle, plan.handle, ctypes.byref(out)))
    return Job(ctx, out, plan)


def spamm_run(ctx: Context, jobs, work_budget):
    """One launch over the next units of every job (work_budget: one number or one per job);
    returns (units run per job, ms of the launch)."""
    n = len(jobs)
    arr = (ctypes.c_void_p * n)(*[j.handle for j in jobs])
    wb = [float(work_budget)] * n if np.isscalar(work_budget) else [float(w) for w in work_budget]
    budget = (ctypes.c_double * n)(*wb)
    ran = (ctypes.c_int64 * n)()
    ms = ctypes.c_double()
    _check(ctx.handle, load().spamm_run(ctx.handle, n, arr, budget, ran, ctypes.byref(ms)))
    return [int(x) for x in ran], ms.value


def spamm_job_finish(ctx: Context, job: Job, stats: bool = False):
    out = ctypes.c_void_p()
    st = Stats()
    _check(ctx.handle, load().spamm_job_finish(ctx.handle, job.handle, ctypes.byref(out), ctypes.byref(st)))
    C = Matrix(ctx, out)
    return (C, st.as_dict()) if stats else C


def spamm_exec_graph_info(ctx: Context) -> dict:
    i, u = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx.handle, load().spamm_exec_graph_info(ctx.handle, ctypes.byref(i), ctypes.byref(u)))
    return {"instantiations": i.value, "updates": u.value}


def spamm_set_gemm_sms(ctx: Context, nsms: int):
    _check(ctx.handle, load().spamm_set_gemm_sms(ctx.handle, int(nsms)))


def spamm_add(ctx: Context, alpha: float, X: Matrix, beta: float, Y: Matrix) -> Matrix:
    """alpha X + beta Y (union of the leaf sets, exact-zero leaves dropped)."""
    return _new(ctx, load().spamm_add, float(alpha), X.handle, float(beta), Y.handle)


def spamm_identity(ctx: Context, n: int, bs: int) -> Matrix:
    return _new(ctx, load().spamm_identity, int(n), int(bs))


def spamm_trace(ctx: Context, X: Matrix) -> float:
    v = ctypes.c_double()
    _check(ctx.handle, load().spamm_trace(ctx.handle, X.handle, ctypes.byref(v)))
    return v.value


def spamm_check_timeout_path(ctx: Context, wait_ns: int = 50_000_000) -> int:
    """Run the device-timeout diagnostic; returns the raw status (E_TIMEOUT expected)."""
    return int(load().spamm_check_timeout_path(ctx.handle, int(wait_ns)))


ORDERS = {"auto": 0, "morton": 1, "longest": 2}


def spamm_set_claim_order(ctx: Context, order: str):
    """spamm_set_claim_order: the work units' claiming order of the plans
    created afterwards on ctx ("auto", "morton" or "longest")."""
    _check(ctx.handle, load().spamm_set_claim_order(ctx.handle, ORDERS[order]))


def spamm_set_exec_graph(ctx: Context, enable: bool):
    _check(ctx.handle, load().spamm_set_exec_graph(ctx.handle, 1 if enable else 0))
