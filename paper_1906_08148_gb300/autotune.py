"""Choice of precision form and leaf size per multiply request, and the
work rate that sizes each launch of the served stream.

A request is described by (n, alpha, tau): the size, the decay rate of its
inputs and the threshold.  The candidates are the library's forms: FP64 leaf
products with 32 x 32, 64 x 64 or 128 x 128 leaves, and the tensor-core
forms (BF16 3-slice and 4-slice error-free splits, FP16 with per-leaf
scaling) with 64 x 64 or 128 x 128 leaves.

`calibrate` measures the candidates on synthetic decay inputs at a grid of
(n, alpha, tau) points: the time of plan + execute, and for each tensor form
its arithmetic error ||C_form - C_ref||_F, where C_ref is the 4-slice split
at the same tau and leaf size (its own arithmetic error, about 4e-10 of
||C||, is far below every other form's and is measured against FP64 where
FP64 is timed), next to the method's truncation error, estimated as
||C_ref(tau) - C_ref(tau / 100)||_F (the error of C at tau against a product
a hundred times more accurate; no exact product is formed, so the grid
reaches the largest served sizes).  FP64 is timed where its expected time is
short and otherwise estimated from its measured rate (kept products per
second).  A form is admissible at a point when its arithmetic error does not
exceed the truncation error there (the error of the result is then still
dominated by the method's own approximation); the fastest admissible
candidate wins.  Each candidate's measured work rate (kept products per ms
for FP64, quad steps per ms for the tensor forms) is kept too: the server
sizes its launches from it (the slice schedule).

The tile schedule is calibrated too: for the winner at each point the leaf
products run once with the work units claimed in Morton order and once
longest first (spamm_set_claim_order), and the faster order (GEMM time) is
part of the choice.

`choose` maps a request to the winner of the nearest calibrated point
(distance in log2 n, alpha, log10 tau).  It depends only on the request and
the table, so a request gets the same form and leaf size alone or in a mix.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import dataclass
from typing import Iterable, List, Optional, Sequence

CANDIDATES = (("fp64", 32), ("fp64", 64), ("fp64", 128), ("bf16_split", 64), ("bf16_split", 128),
              ("bf16_split4", 64), ("bf16_split4", 128), ("fp16_scaled", 64), ("fp16_scaled", 128))
FP64_TIMED_MAX_S = 3.0  # FP64 is timed where it is expected to take less than this
TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


@dataclass(frozen=True)
class Choice:
    prec: str
    bs: int
    order: str = "auto"   # claiming order of the leaf-product units (spamm_set_claim_order)


@dataclass
class Point:
    n: int
    alpha: float
    tau: float
    choice: Choice
    ms: dict          # candidate "prec/bs" -> milliseconds (measured, or estimated for long FP64 runs)
    arith_err: dict   # tensor candidate -> ||C_form - C_ref||_F
    trunc_err: float  # ||AB - C||_F estimate, or a dict per leaf size
    rate: dict = None       # candidate -> work per ms (kept products or quad steps)
    estimated: tuple = ()   # candidates whose ms is estimated from a rate
    order_ms: dict = None   # claiming order -> GEMM ms of the winner (empty: not measured)

    def trunc(self, bs: int) -> float:
        return self.trunc_err.get(str(bs), math.inf) if isinstance(self.trunc_err, dict) else self.trunc_err

    def key(self):
        return (math.log2(self.n), self.alpha, math.log10(self.tau))


def _name(prec: str, bs: int) -> str:
    return f"{prec}/{bs}"


def decide(ms: dict, arith_err: dict, trunc_err) -> Choice:
    """Fastest candidate whose arithmetic error is within the truncation error
    (trunc_err: one number, or a dict by leaf size)."""
    best = None
    for prec, bs in CANDIDATES:
        k = _name(prec, bs)
        if k not in ms:
            continue
        t = trunc_err.get(str(bs), math.inf) if isinstance(trunc_err, dict) else trunc_err
        if prec != "fp64" and not (arith_err.get(k, math.inf) <= t):
            continue
        if best is None or ms[k] < ms[best]:
            best = k
    if best is None:
        return Choice("fp64", 64)
    p, b = best.split("/")
    return Choice(p, int(b))


class Autotuner:
    def __init__(self, points: Optional[Sequence[Point]] = None, path: str = TABLE_PATH):
        if points is None:
            points = load(path) if os.path.exists(path) else []
        self.points: List[Point] = list(points)

    def choose(self, n: int, alpha: float, tau: float, bs: Optional[int] = None) -> Choice:
        """Form and leaf size for a request (bs given: inputs already built with
        that leaf size, only the form is chosen).  FP64 with 64 x 64 leaves (or
        the given bs) without a table or for exact products (tau = 0)."""
        default = Choice("fp64", bs or 64)
        if not self.points or tau <= 0.0:
            return default
        q = (math.log2(max(n, 1)), alpha, math.log10(tau))

        def dist(p: Point):
            k = p.key()
            return sum((a - b) ** 2 for a, b in zip(q, k)), k  # ties: the smaller key, deterministic

        p = min(self.points, key=dist)
        if bs is None:
            return p.choice
        ms = {k: v for k, v in p.ms.items() if int(k.split("/")[1]) == bs}
        if not ms:
            return default
        c = decide(ms, p.arith_err, p.trunc_err)
        return p.choice if (c.prec, c.bs) == (p.choice.prec, p.choice.bs) else c

    def rate(self, prec: str, bs: int) -> Optional[float]:
        """Median measured work rate (per ms) of a candidate over the table, or None."""
        v = sorted(p.rate[_name(prec, bs)] for p in self.points if p.rate and _name(prec, bs) in p.rate)
        return v[len(v) // 2] if v else None


def load(path: str = TABLE_PATH) -> List[Point]:
    d = json.load(open(path))
    return [Point(p["n"], p["alpha"], p["tau"],
                  Choice(p["choice"]["prec"], p["choice"]["bs"], p["choice"].get("order", "auto")), p["ms"],
                  p["arith_err"], p["trunc_err"], p.get("rate"), tuple(p.get("estimated", ())), p.get("order_ms"))
            for p in d["points"]]


def save(points: Iterable[Point], path: str = TABLE_PATH, meta: Optional[dict] = None):
    out = {"meta": meta or {}, "points": [
        {"n": p.n, "alpha": p.alpha, "tau": p.tau,
         "choice": {"prec": p.choice.prec, "bs": p.choice.bs, "order": p.choice.order},
         "ms": p.ms, "arith_err": p.arith_err, "trunc_err": p.trunc_err, "rate": p.rate,
         "estimated": list(p.estimated), "order_ms": p.order_ms} for p in points]}
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def calibrate(S, ctx, grid: Iterable[tuple], repeats: int = 2, mode: str = "combined",
              log=None) -> List[Point]:
    """Measure the candidates at each (n, alpha, tau) of `grid` on the 3-D
    lattice generator (seeds 1 and 2).  S: the libspamm binding module."""
    import synth
    pts = []
    fp64_rate = {}  # leaf size -> measured kept products per second
    for n, alpha, tau in grid:
        pa, pb = synth.lattice_3d(n, alpha=alpha, seed=1), synth.lattice_3d(n, alpha=alpha, seed=2)
        ms, arith, trunc, rate, est = {}, {}, {}, {}, []
        try:
            _measure_point(S, ctx, pa, pb, tau, mode, repeats, fp64_rate, ms, arith, trunc, rate, est)
        except S.SpammError as e:
            if e.status != S.E_OOM:
                raise
            if log:
                log(f"{n} {alpha} {tau}: does not fit ({e})")
            continue
        arith = {k: v for k, v in arith.items() if not k.startswith("fp64")}
        # the reference's error against itself is 0: use its measured error against FP64 where known
        for bs in {b for _, b in CANDIDATES if _ != "fp64"}:
            k = _name("bf16_split4", bs)
            if k + ":vs_fp64" in arith:
                arith[k] = arith[k + ":vs_fp64"]
        ch = decide(ms, arith, trunc)
        order_ms = {}
        if _name(ch.prec, ch.bs) not in est:
            try:
                order_ms = _measure_order(S, ctx, pa, pb, tau, mode, ch, repeats)
            except S.SpammError as e:
                if e.status != S.E_OOM:
                    raise
        if order_ms:
            ch = Choice(ch.prec, ch.bs, min(order_ms, key=order_ms.get))
        pt = Point(n, alpha, tau, ch, ms, arith, trunc, rate, tuple(est), order_ms)
        pts.append(pt)
        if log:
            log(pt)
    return pts


def _measure_point(S, ctx, pa, pb, tau, mode, repeats, fp64_rate, ms, arith, trunc, rate, est):
    """Every candidate at one grid point (inputs truncated while generated at
    tau / 100, exact for the combined method at tau and at tau / 100).  A leaf
    size whose inputs or products do not fit leaves its candidates out (the
    others are still measured); every handle is released on the way out."""
    for bs in sorted({b for _, b in CANDIDATES}):
        try:
            _measure_bs(S, ctx, pa, pb, tau, mode, repeats, fp64_rate, ms, arith, trunc, rate, est, bs)
        except S.SpammError as e:
            if e.status != S.E_OOM:
                raise
            for prec, b in CANDIDATES:
                if b == bs:
                    ms.pop(_name(prec, bs), None)
                    arith.pop(_name(prec, bs), None)
            trunc.pop(str(bs), None)
            S.spamm_trim(ctx)
    if not ms or not any(k.split("/")[0] != "fp64" for k in ms):
        # no tensor form measured (their reference products do not fit): the
        # point would only say that FP64 fits, so it is left out
        raise S.SpammError(S.E_OOM, "no tensor-form candidate fits")


def _measure_bs(S, ctx, pa, pb, tau, mode, repeats, fp64_rate, ms, arith, trunc, rate, est, bs):
    held = []

    def keep(h):
        held.append(h)
        return h

    def drop(h):
        held.remove(h)
        h.close()

    try:
        GA = keep(S.spamm_generate(ctx, pa, bs, tau / 100.0))
        GB = keep(S.spamm_generate(ctx, pb, bs, tau / 100.0))
        tensor = [p for p, b in CANDIDATES if b == bs and p != "fp64"]
        ref = None
        if tensor:
            ref, _ = S.spamm_multiply(ctx, GA, GB, tau, mode, "bf16_split4", stats=True)
            keep(ref)
            fine = keep(S.spamm_multiply(ctx, GA, GB, tau / 100.0, mode, "bf16_split4"))
            trunc[str(bs)] = S.spamm_error(ctx, fine, ref)
            drop(fine)
        for prec, cbs in CANDIDATES:
            if cbs != bs:
                continue
            k = _name(prec, bs)
            if prec == "fp64" and bs in fp64_rate:
                plan = keep(S.spamm_plan_create(ctx, GA, GB, tau, mode, "fp64"))
                nk = plan.info()["n_kept"]
                drop(plan)
                if nk / fp64_rate[bs] > FP64_TIMED_MAX_S:
                    ms[k] = 1e3 * nk / fp64_rate[bs]  # too long to time here: estimated from its rate
                    est.append(k)
                    continue
            times, st, C = [], None, None
            for _ in range(repeats + 1):  # the first run warms up
                if C is not None:
                    drop(C)
                t0 = time.perf_counter()
                C, st = S.spamm_multiply(ctx, GA, GB, tau, mode, prec, stats=True)
                times.append(time.perf_counter() - t0)
                keep(C)
                if prec == "fp64" and times[-1] > FP64_TIMED_MAX_S:
                    break
            tm = sorted(times[1:])[len(times[1:]) // 2] if len(times) > 1 else times[0]
            ms[k] = 1e3 * tm
            rate[k] = st["n_steps"] / st["ms_gemm"] if st["ms_gemm"] > 0 else None
            if prec == "fp64":
                fp64_rate[bs] = st["n_kept"] / max(tm, 1e-9)
            if ref is not None:
                arith[k] = S.spamm_error(ctx, ref, C) if prec != "fp64" else 0.0
                if prec == "fp64":  # the reference's own error, where FP64 ran
                    arith[_name("bf16_split4", bs) + ":vs_fp64"] = S.spamm_error(ctx, C, ref)
            drop(C)
    finally:
        for h in reversed(held):
            h.close()


def _measure_order(S, ctx, pa, pb, tau, mode, ch: Choice, repeats) -> dict:
    """GEMM milliseconds of the chosen form with its units claimed in Morton
    order and longest first (median of `repeats` after one untimed run)."""
    out = {}
    GA = S.spamm_generate(ctx, pa, ch.bs, tau / 100.0)
    GB = S.spamm_generate(ctx, pb, ch.bs, tau / 100.0)
    try:
        for order in ("morton", "longest"):
            S.spamm_set_claim_order(ctx, order)
            t = []
            for _ in range(repeats + 1):
                C, st = S.spamm_multiply(ctx, GA, GB, tau, mode, ch.prec, stats=True)
                C.close()
                t.append(st["ms_gemm"])
            v = sorted(t[1:])
            out[order] = v[len(v) // 2]
    finally:
        S.spamm_set_claim_order(ctx, "auto")
        GA.close()
        GB.close()
    return out


if __name__ == "__main__":
    # Calibration run on a GPU: writes tuned.json beside this file.
    import argparse
    import sys

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[4096, 16384, 65536, 131072])
    ap.add_argument("--alpha", type=float, nargs="+", default=[0.6, 1.2])
    ap.add_argument("--tau", type=float, nargs="+", default=[1e-4, 1e-6, 1e-8])
    ap.add_argument("--repeats", type=int, default=2)
    ap.add_argument("--out", default=TABLE_PATH)
    a = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_1906_08148_gb300 import spamm as S
    c = S.Context(0)
    grid = [(n, al, t) for n in a.n for al in a.alpha for t in a.tau]
    def log(p):
        if isinstance(p, str):
            print(p, flush=True)
            return
        print(p.n, p.alpha, p.tau, p.choice, {k: round(v, 2) for k, v in p.ms.items()},
              {k: "%.2e" % v for k, v in p.arith_err.items()}, p.trunc_err, p.order_ms, flush=True)

    pts = calibrate(S, c, grid, repeats=a.repeats, log=log)
    save(pts, a.out, meta={"workload": "3-D lattice decay, seeds 1 and 2, combined method",
                           "candidates": [list(x) for x in CANDIDATES], "repeats": a.repeats,
                           "truncation_error": "||C_ref(tau) - C_ref(tau/100)||_F, C_ref the 4-slice split",
                           "fp64_timed_max_s": FP64_TIMED_MAX_S})
