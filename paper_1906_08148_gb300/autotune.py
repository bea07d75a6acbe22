"""Choice of precision form and leaf size per multiply request.

A request is described by (n, alpha, tau): the size, the decay rate of its
inputs and the threshold.  The candidates are the library's forms: FP64 leaf
products with 32 x 32, 64 x 64 or 128 x 128 leaves, and the tensor-core
forms (BF16 three-term split, FP16 with per-leaf scaling) with 64 x 64
leaves.

`calibrate` measures every candidate on synthetic decay inputs at a grid of
(n, alpha, tau) points: the time of plan + execute, and for each tensor form
its arithmetic error against the FP64 product at the same tau next to the
truncation error of the method itself (against the exact FP64 product).  A
form is admissible at a point when its arithmetic error does not exceed the
truncation error there (the error of the result is then still dominated by
the method's own approximation); the fastest admissible candidate wins.

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

CANDIDATES = (("fp64", 32), ("fp64", 64), ("fp64", 128), ("bf16_split", 64), ("fp16_scaled", 64))
TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


@dataclass(frozen=True)
class Choice:
    prec: str
    bs: int


@dataclass
class Point:
    n: int
    alpha: float
    tau: float
    choice: Choice
    ms: dict          # candidate "prec/bs" -> measured milliseconds
    arith_err: dict   # tensor candidate -> ||C_form - C_fp64||_F
    trunc_err: float  # ||AB - C_fp64||_F

    def key(self):
        return (math.log2(self.n), self.alpha, math.log10(self.tau))


def _name(prec: str, bs: int) -> str:
    return f"{prec}/{bs}"


def decide(ms: dict, arith_err: dict, trunc_err: float) -> Choice:
    """Fastest candidate whose arithmetic error is within the truncation error."""
    best = None
    for prec, bs in CANDIDATES:
        k = _name(prec, bs)
        if k not in ms:
            continue
        if prec != "fp64" and not (arith_err.get(k, math.inf) <= trunc_err):
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
        return decide(ms, p.arith_err, p.trunc_err) if ms else default


def load(path: str = TABLE_PATH) -> List[Point]:
    d = json.load(open(path))
    return [Point(p["n"], p["alpha"], p["tau"], Choice(p["choice"]["prec"], p["choice"]["bs"]), p["ms"],
                  p["arith_err"], p["trunc_err"]) for p in d["points"]]


def save(points: Iterable[Point], path: str = TABLE_PATH, meta: Optional[dict] = None):
    out = {"meta": meta or {}, "points": [
        {"n": p.n, "alpha": p.alpha, "tau": p.tau, "choice": {"prec": p.choice.prec, "bs": p.choice.bs},
         "ms": p.ms, "arith_err": p.arith_err, "trunc_err": p.trunc_err} for p in points]}
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def calibrate(S, ctx, grid: Iterable[tuple], repeats: int = 3, mode: str = "combined") -> List[Point]:
    """Measure every candidate at each (n, alpha, tau) of `grid` on the 3-D
    lattice generator (seeds 1 and 2).  S: the libspamm binding module."""
    import synth
    pts = []
    for n, alpha, tau in grid:
        pa, pb = synth.lattice_3d(n, alpha=alpha, seed=1), synth.lattice_3d(n, alpha=alpha, seed=2)
        ms, res = {}, {}
        for bs in sorted({b for _, b in CANDIDATES}):
            GA, GB = S.spamm_generate(ctx, pa, bs), S.spamm_generate(ctx, pb, bs)
            for prec, cbs in CANDIDATES:
                if cbs != bs:
                    continue
                times = []
                for _ in range(repeats + 1):  # the first run warms up
                    t0 = time.perf_counter()
                    C = S.spamm_multiply(ctx, GA, GB, tau, mode, prec)
                    times.append(time.perf_counter() - t0)
                    if len(times) <= repeats:
                        C.close()
                ms[_name(prec, bs)] = 1e3 * sorted(times[1:])[len(times[1:]) // 2]
                if bs == 64:
                    res[prec] = C
                else:
                    C.close()
            if bs == 64:
                X = S.spamm_multiply(ctx, GA, GB, 0.0, "spamm", "fp64")
                trunc = S.spamm_error(ctx, X, res["fp64"])
                arith = {_name(p, 64): S.spamm_error(ctx, res["fp64"], res[p]) for p in res if p != "fp64"}
                X.close()
                for C in res.values():
                    C.close()
            GA.close()
            GB.close()
        pts.append(Point(n, alpha, tau, decide(ms, arith, trunc), ms, arith, trunc))
    return pts


if __name__ == "__main__":
    # Calibration run on a GPU: writes tuned.json beside this file.
    import argparse
    import sys

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[4096, 16384])
    ap.add_argument("--alpha", type=float, nargs="+", default=[0.6, 0.9, 1.2])
    ap.add_argument("--tau", type=float, nargs="+", default=[1e-4, 1e-6, 1e-8])
    ap.add_argument("--repeats", type=int, default=2)
    ap.add_argument("--out", default=TABLE_PATH)
    a = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_1906_08148_gb300 import spamm as S
    c = S.Context(0)
    grid = [(n, al, t) for n in a.n for al in a.alpha for t in a.tau]
    pts = calibrate(S, c, grid, repeats=a.repeats)
    save(pts, a.out, meta={"workload": "3-D lattice decay, seeds 1 and 2, combined method",
                           "candidates": [list(x) for x in CANDIDATES], "repeats": a.repeats})
    for p in pts:
        print(p.n, p.alpha, p.tau, p.choice, {k: round(v, 2) for k, v in p.ms.items()},
              {k: "%.2e" % v for k, v in p.arith_err.items()}, "%.2e" % p.trunc_err)
