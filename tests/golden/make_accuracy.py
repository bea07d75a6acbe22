"""Writes tests/golden/accuracy.json: the approximation error ||AB - C||_F of
the benchmark workloads, per method and tau, estimated by the CPU oracle
(oracle.sampled.error_estimate: stratified samples of output leaves, each
leaf of AB exact over every non-null k of the untruncated inputs, each leaf
of C the method's own; 95 % normal-approximation interval).  The benchmark
reads this table to pick, for a target sigma, the largest tau of the grid
whose error meets it (the equal-accuracy comparison of Section 5.3).

Only oracle/ and synth/ are used: no value here comes from the GPU path.
Usage: python tests/golden/make_accuracy.py [--samples 256] [--only NAME]"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import sampled  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "accuracy.json")

# name -> (n, alpha, seeds of A and B (equal: X times X), bs, modes, taus)
WORKLOADS = {
    "lattice65536": (65536, 1.0, (1, 2), 64, ("combined", "spamm", "truncate"), (1e-4, 1e-6, 1e-8)),
    "lattice262144_square": (262144, 0.8, (1, 1), 64, ("combined",), (1e-5, 1e-7)),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=256)
    ap.add_argument("--only", default=None)
    a = ap.parse_args()
    table = json.load(open(OUT)) if os.path.exists(OUT) else {}
    table["source"] = ("tests/golden/make_accuracy.py: oracle.sampled.error_estimate, stratified output-leaf "
                       "samples, exact leaves of AB over all non-null k, 95 % interval (Section 5.3 compares "
                       "methods at equal ||AB - C||_F)")
    for name, (n, alpha, seeds, bs, modes, taus) in WORKLOADS.items():
        if a.only and name != a.only:
            continue
        pa = synth.lattice_3d(n, alpha=alpha, seed=seeds[0])
        pb = synth.lattice_3d(n, alpha=alpha, seed=seeds[1])
        w = table.setdefault("workloads", {}).setdefault(name, {"n": n, "alpha": alpha, "seeds": list(seeds),
                                                                 "bs": bs, "errors": {}})
        for mode in modes:
            for tau in taus:
                t0 = time.perf_counter()
                r = sampled.error_estimate(pa, pb, bs, tau, oracle.MODES[mode], samples=a.samples, seed=0)
                w["errors"]["%s %g" % (mode, tau)] = {
                    "mode": mode, "tau": tau, "estimate": r["estimate"], "low": r["low"], "high": r["high"],
                    "exact_norm": r["exact_norm"], "samples": r["samples"],
                    "seconds": round(time.perf_counter() - t0, 1), "threads": oracle.num_threads()}
                json.dump(table, open(OUT, "w"), indent=1)
                print(name, mode, tau, r["estimate"], r["low"], r["high"], flush=True)


if __name__ == "__main__":
    main()
