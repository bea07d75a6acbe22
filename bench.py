#!/usr/bin/env python
"""Benchmark: kept-block GFLOP/s of approximate C ~ AB on one GB300.

Workload (default): the 3-D lattice decay problem, n = 65536 indices on a
64 x 32 x 32 unit lattice in Morton order, a_ij = u_ij exp(-1.0 d), u_ij ~
U[-1,1) symmetric, A != B from seeds 1 and 2, 64 x 64 leaves, Hybrid
(combined) method at tau = 1e-6, FP64 leaf products.  One step is one pass
of the whole hot path from device-resident inputs (leaves and norms, which
the paper treats as given): input truncation, task-list build, batched leaf
products with the C-leaf norm epilogue, C quadtree norms, ||C||_F read-back.

Metric: kept-block GFLOP/s = 2 bs^3 N_kept / t (the paper's flop count,
Section 5.3); mults/s = N_kept / t is reported beside it.  Inputs are 2 x
27.7 GB, far larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]

--impl reference times the CPU oracle (the only reference implementation
this method has) on a bounded window of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_BYTES = 129 << 20  # GB300 L2 (for the flush rule)
FP64_PEAK_GFLOPS = 1258.6  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (DFMA probe: 1208)
CONFIGS = {
    "lattice65536": dict(n=65536, kind=1, alpha=1.0, bs=64, seeds=(1, 2),
                         desc="3-D lattice 64x32x32 Morton, alpha=1.0, A!=B seeds 1,2, 64x64 leaves"),
    "lattice262144": dict(n=262144, kind=1, alpha=0.8, bs=64, seeds=(1, 1),
                          desc="3-D lattice 64x64x64 Morton, alpha=0.8, X times X (A = B, seed 1), 64x64 leaves, "
                               "inputs truncated while generated (precision-form configuration)"),
    "lattice16384": dict(n=16384, kind=1, alpha=1.0, bs=64, seeds=(1, 2),
                         desc="3-D lattice 32x32x16 Morton, alpha=1.0, A!=B seeds 1,2, 64x64 leaves (profiling size)"),
    "model2048": dict(n=2048, kind=0, alpha=0.05, bs=32, seeds=(1, 1),
                      desc="1-D decay n=2048, alpha=0.05, A=B seed 1, 32x32 leaves"),
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--latency-repeats", type=int, default=50,
                    help="p50/p99 latency over at least this many warm multiplies: the timed steps, then "
                         "untimed-for-throughput repeats up to this count")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="lattice65536", choices=sorted(CONFIGS))
    ap.add_argument("--mode", default="combined", choices=["truncate", "spamm", "combined"])
    ap.add_argument("--tau", type=float, default=None,
                    help="default: chosen for --sigma from the accuracy table (equal-accuracy headline), else 1e-6")
    ap.add_argument("--prec", default=None, choices=["fp64", "bf16_split", "bf16_split4", "fp16_scaled", "auto"],
                    help="default: the fastest form whose arithmetic error stays below the truncation error "
                         "(equal-accuracy headline), else fp64; auto: the autotuner's choice per request "
                         "(served stream only)")
    ap.add_argument("--sigma", type=float, default=1e-4,
                    help="target ||AB - C||_F of the equal-accuracy headline")
    ap.add_argument("--pc-taus", type=float, nargs="+", default=[1e-5, 1e-7],
                    help="taus of the precision-form configuration (--config lattice262144)")
    ap.add_argument("--pc-samples", type=int, default=256,
                    help="output leaves compared between each form and FP64 (precision-form configuration)")
    ap.add_argument("--pc-no-fp64", action="store_true", help="precision-form configuration without the FP64 runs")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve", action="store_true", help="served-stream benchmark instead of the single workload")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-inputs", type=int, default=12)
    ap.add_argument("--serve-nmax", type=int, default=131072)
    ap.add_argument("--serve-batch", type=int, default=32)
    ap.add_argument("--serve-alpha", type=float, nargs=2, default=[0.6, 1.2])
    ap.add_argument("--serve-input-frac", type=float, default=0.3,
                    help="fraction of the free device memory the resident inputs may hold")
    ap.add_argument("--serve-fp64-prefix", type=int, default=32,
                    help="first requests of the stream also served all-FP64 for comparison (0: skip)")
    ap.add_argument("--serve-slice-ms", type=float, default=25.0,
                    help="target duration of one launch of the served stream (continuous batching slices)")
    ap.add_argument("--no-forms", action="store_true", help="skip the tensor-form comparison in the bench line")
    ap.add_argument("--form-steps", type=int, default=5)
    ap.add_argument("--model-problem", action="store_true", help="the paper's 1-D model problem sweep")
    ap.add_argument("--sweep", action="store_true", help="the three methods at equal accuracy on --config")
    ap.add_argument("--sweep-taus", type=float, nargs="+", default=[1e-4, 1e-6, 1e-8])
    ap.add_argument("--sigmas", type=float, nargs="+", default=[1e-2, 1e-4, 1e-6])
    ap.add_argument("--sweep-precs", nargs="+", default=["fp64", "bf16_split", "bf16_split4", "fp16_scaled"])
    ap.add_argument("--block-sparse", action="store_true", help="random block-sparse sweep over fill-in")
    ap.add_argument("--bsp-n", type=int, default=2048)
    ap.add_argument("--bsp-bs", type=int, nargs="+", default=[32, 64, 128, 256])
    ap.add_argument("--bsp-fills", type=float, nargs="+", default=[0.05, 0.1, 0.2, 0.3, 0.5, 0.7, 0.9])
    ap.add_argument("--bsp-repeats", type=int, default=20)
    ap.add_argument("--chain", action="store_true", help="repeated squaring chain")
    ap.add_argument("--chain-n", type=int, default=262144)
    ap.add_argument("--chain-alpha", type=float, default=1.0)
    ap.add_argument("--chain-tau", type=float, default=1e-6)
    ap.add_argument("--chain-steps", type=int, default=20)
    ap.add_argument("--chain-precs", nargs="+", default=["fp64", "fp16_scaled"])
    ap.add_argument("--sp2", action="store_true", help="SP2 purification chain (gapped two-sublattice insulator)")
    ap.add_argument("--sp2-n", type=int, nargs="+", default=[1048576, 524288, 262144, 131072],
                    help="lattice sizes, tried from the largest: the chain runs at the largest one admitted")
    ap.add_argument("--sp2-alpha", type=float, default=1.0)
    ap.add_argument("--sp2-delta", type=float, default=6.0, help="on-site term +-delta (opens the gap)")
    ap.add_argument("--sp2-tau", type=float, default=1e-6)
    ap.add_argument("--sp2-iters", type=int, default=20)
    ap.add_argument("--sp2-tol", type=float, default=0.0)
    ap.add_argument("--sp2-fp64-iters", type=int, default=None,
                    help="iterations of the FP64 chain (default: as many as the tensor forms run)")
    ap.add_argument("--sp2-probe-every", type=int, default=5)
    ap.add_argument("--sp2-probe-rows", type=int, default=4)
    ap.add_argument("--sp2-budget", type=float, default=0.9, help="fraction of free device memory admitted")
    ap.add_argument("--sp2-force", action="store_true", help="run every size without the footprint estimate")
    ap.add_argument("--passes", action="store_true",
                    help="bandwidth of the norm pass and the task-list pass on the bench workload")
    ap.add_argument("--mp-n", type=int, default=40000)
    ap.add_argument("--mp-bs", type=int, nargs="+", default=[64])
    ap.add_argument("--mp-sigma", type=float, default=1e-6)
    ap.add_argument("--mp-tau-lo", type=int, default=4, help="largest tau = 10^-lo")
    ap.add_argument("--mp-tau-hi", type=int, default=12, help="smallest tau = 10^-hi")
    return ap.parse_args()


# ----------------------------------------------------- equal-accuracy choice
ACCURACY = os.path.join(ROOT, "tests", "golden", "accuracy.json")
TC_FORMS = ("fp16_scaled", "bf16_split", "bf16_split4")


def accuracy_entry(workload, mode, tau):
    """The oracle's sampled ||AB - C||_F (estimate and 95 % interval) for a
    workload, method and tau, from the committed table; None if absent."""
    if not os.path.exists(ACCURACY):
        return None
    w = json.load(open(ACCURACY)).get("workloads", {}).get(workload)
    if not w:
        return None
    return w["errors"].get("%s %g" % (mode, tau))


def tau_for_sigma(workload, mode, sigma, taus=(1e-4, 1e-6, 1e-8)):
    """Largest tau of the grid whose error (upper end of its interval) meets
    sigma: the paper's rule for comparing methods at equal accuracy (Section
    5.3)."""
    for t in sorted(taus, reverse=True):
        e = accuracy_entry(workload, mode, t)
        if e is not None and e["high"] <= sigma:
            return t
    return None


def resolve_defaults(args):
    """No --prec, no --tau and no other mode on a workload the accuracy table
    covers: the equal-accuracy headline (tau from --sigma, the form chosen on
    the GPU).  Otherwise tau defaults to 1e-6 and the form to FP64."""
    special = any((args.serve, args.sweep, args.model_problem, args.block_sparse, args.chain, args.sp2,
                   args.passes))
    args.headline = (not special and args.prec is None and args.tau is None
                     and tau_for_sigma(args.config, args.mode, args.sigma) is not None)
    if args.headline:
        args.tau = tau_for_sigma(args.config, args.mode, args.sigma)
    if args.tau is None:
        args.tau = 1e-6
    if args.prec is None and not args.headline:
        args.prec = "fp64"


def equal_accuracy_choice(S, ctx, GA, GB, args, stream, torch):
    """At the tau chosen for sigma, the FP64 product and every tensor-core
    form, each timed once with CUDA events (after an untimed run of the form):
    a form is admissible if its arithmetic error ||C_form - C_fp64||_F stays
    below the lower end of the method's truncation-error interval and the two
    together stay within sigma.  The fastest admissible form is chosen (FP64
    if none is)."""
    trunc = accuracy_entry(args.config, args.mode, args.tau)

    def timed(prec):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        C, st = S.spamm_multiply(ctx, GA, GB, args.tau, args.mode, prec, stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return C, st, {"ms_per_step": ms, "kept_gflops": st["kept_flops"] / ms / 1e6,
                       "mults_per_s": st["n_kept"] / ms * 1e3, "ms_gemm": st["ms_gemm"]}

    ref, st_ref, fp64 = timed("fp64")
    forms = {"fp64": dict(fp64, arith_error=0.0, admissible=trunc["high"] <= args.sigma)}
    for prec in TC_FORMS:
        S.spamm_multiply(ctx, GA, GB, args.tau, args.mode, prec).close()
        C, st, rec = timed(prec)
        arith = S.spamm_error(ctx, ref, C)
        C.close()
        rec.update(arith_error=arith, admissible=bool(arith <= trunc["low"] and trunc["high"] + arith <= args.sigma))
        forms[prec] = rec
    ref.close()
    ok = [p for p in TC_FORMS if forms[p]["admissible"]]
    chosen = min(ok, key=lambda p: forms[p]["ms_per_step"]) if ok else "fp64"
    return chosen, {"sigma": args.sigma, "tau": args.tau, "method": args.mode, "truncation_error": trunc,
                    "forms": forms, "chosen": chosen,
                    "rule": "largest tau of {1e-4, 1e-6, 1e-8} whose sampled ||AB - C||_F (95 % upper end) meets "
                            "sigma; a tensor form is admissible if ||C_form - C_fp64||_F is below the lower end "
                            "of that error's interval and the two add up to at most sigma; the fastest admissible "
                            "form is timed"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle
def oracle_window(cfg, mode, tau, target_s):
    """Oracle inputs for a window of C leaves sized for about target_s seconds."""
    import oracle
    from oracle import sampled
    import synth
    pa = synth.DecayParams(n=cfg["n"], kind=cfg["kind"], alpha=cfg["alpha"], seed=cfg["seeds"][0])
    pb = synth.DecayParams(n=cfg["n"], kind=cfg["kind"], alpha=cfg["alpha"], seed=cfg["seeds"][1])
    bs = cfg["bs"]
    nb = -(-cfg["n"] // bs)
    w = min(8, nb)
    while True:
        A, B = sampled.window_inputs(pa, pb, bs, range(w), range(w))
        t0 = time.perf_counter()
        C, ikj = sampled.window_product(A, B, tau, oracle.MODES[mode])
        dt = time.perf_counter() - t0
        if dt >= 0.25 * target_s or w >= nb:
            return A, B, w, dt, len(ikj)
        grow = (target_s / max(dt, 1e-3)) ** 0.5
        w = min(nb, max(w + 1, int(w * min(grow, 4.0))))


def cpu_baseline(cfg, mode, tau, target_s):
    import oracle
    from oracle import sampled
    A, B, w, _, _ = oracle_window(cfg, mode, tau, target_s)
    t0 = time.perf_counter()
    C, ikj = sampled.window_product(A, B, tau, oracle.MODES[mode])
    dt = time.perf_counter() - t0
    flops = 2.0 * cfg["bs"] ** 3 * len(ikj)
    return {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"C leaves (i,j) in block rows/cols [0,{w}) of the same workload: {len(ikj)} kept leaf "
                      f"products ({flops / 1e9:.1f} GFLOP) in {dt:.1f} s"}


def run_reference(args, cfg):
    """--impl reference: the CPU oracle, each step a bounded window of the workload."""
    import oracle
    from oracle import sampled
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    A, B, w, _, _ = oracle_window(cfg, args.mode, args.tau, per_step)
    for _ in range(args.warmup):
        sampled.window_product(A, B, args.tau, oracle.MODES[args.mode])
    flops, t = 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        C, ikj = sampled.window_product(A, B, args.tau, oracle.MODES[args.mode])
        t += time.perf_counter() - t0
        flops += 2.0 * cfg["bs"] ** 3 * len(ikj)
    value = flops / t / 1e9
    line = {"metric": "kept-block GFLOP/s", "value": value, "unit": "GFLOP/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.config, "desc": cfg["desc"], "method": args.mode, "tau": args.tau,
                       "precision": "fp64", "bs": cfg["bs"]},
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"C leaves in block rows/cols [0,{w}) per step"},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- served stream
def run_served(args):
    """Continuous batching: a Poisson stream of combined-method requests on
    resident 3-D lattice matrices (n log-uniform in [4096, --serve-nmax],
    alpha uniform in --serve-alpha, tau from {1e-4, 1e-6, 1e-8}), first all at
    once (saturated capacity), then at 0.9 x that rate; p50/p99 latency from
    arrival to completion.  --prec auto: each request's precision form and
    leaf size from the autotuner (a function of its n, alpha and tau only),
    with the tuner's measured work rates as the server's first slice sizes;
    otherwise every request in --prec with 64 x 64 leaves.  The input pairs
    are generated in order until they hold --serve-input-frac of the free
    device memory; a pair that does not fit is left out and requests are
    drawn from the resident ones (reported).  The first --serve-fp64-prefix
    requests of the stream also run all at once in the chosen forms and in
    FP64 (64 x 64 leaves): requests/s and latency of both."""
    import math
    import random

    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm as S
    from paper_1906_08148_gb300.autotune import CANDIDATES, Autotuner, Choice
    from paper_1906_08148_gb300.serving import Request, Server

    rng = random.Random(7)
    data = S.Context(0)
    taus = [1e-4, 1e-6, 1e-8]
    tuner = Autotuner() if args.prec == "auto" else None
    guess = None
    if tuner:
        guess = {f"{p}/{b}": tuner.rate(p, b) for p, b in CANDIDATES if tuner.rate(p, b)}
    specs = []
    for i in range(args.serve_inputs):
        n = int(2 ** rng.uniform(math.log2(4096), math.log2(args.serve_nmax))) // 64 * 64
        alpha = rng.uniform(args.serve_alpha[0], args.serve_alpha[1])
        specs.append((n, alpha))
    inputs, dropped = {}, []
    free0, _ = torch.cuda.mem_get_info()
    input_budget = args.serve_input_frac * free0

    def held():
        return sum(m.info()["nleaves"] * 8 * m.info()["bs"] ** 2 for pair in inputs.values() for m in pair)

    def make(i, bs):
        # inputs truncated at the smallest tau of the stream while generating
        # (exact for the combined method: the block rule is per leaf)
        n, alpha = specs[i]
        A = B = None
        try:
            A = S.spamm_generate(data, synth.lattice_3d(n, alpha=alpha, seed=2 * i + 1), bs, min(taus))
            B = S.spamm_generate(data, synth.lattice_3d(n, alpha=alpha, seed=2 * i + 2), bs, min(taus))
        except S.SpammError as e:
            if e.status != S.E_OOM:
                raise
        pair = (A, B)
        if B is None or held() + sum(m.info()["nleaves"] * 8 * bs * bs for m in pair) > input_budget:
            for m in pair:
                if m is not None:
                    m.close()
            return None
        return pair

    def choice(i, tau):
        n, alpha = specs[i]
        return tuner.choose(n, alpha, tau) if tuner else Choice(args.prec, 64)

    # resident inputs: every leaf size the stream's requests on input i ask for
    live = []
    for i in range(len(specs)):
        need = sorted({choice(i, t).bs for t in taus} | ({64} if args.serve_fp64_prefix else set()))
        got = {}
        for bs in need:
            pair = make(i, bs)
            if pair is None:
                break
            got[bs] = pair
        if len(got) == len(need):
            inputs.update({(i, bs): pr for bs, pr in got.items()})
            live.append(i)
        else:
            for pr in got.values():
                for m in pr:
                    m.close()
            dropped.append({"n": specs[i][0], "alpha": specs[i][1], "why": "inputs above the resident-input budget"})
    if not live:
        print(json.dumps({"metric": "requests/s (served stream)", "unavailable": "no input pair fits"}), flush=True)
        return

    def stream(rate, forced=None, count=None):
        reqs, t = [], 0.0
        r2 = random.Random(11)
        for _ in range(count or args.serve_requests):
            if rate:
                t += r2.expovariate(rate)
            i = live[r2.randrange(len(live))]
            tau = r2.choice(taus)
            ch = Choice(forced, 64) if forced else choice(i, tau)
            A, B = inputs[(i, ch.bs)]
            reqs.append(Request(A, B, tau=tau, mode="combined", prec=ch.prec, order=ch.order, arrival=t))
        return reqs

    def serve(reqs):
        srv = Server(max_batch=args.serve_batch, exec_sms=144, slice_ms=args.serve_slice_ms, rate_guess=guess,
                     keep_results=False)
        srv.start()
        ids = [srv.submit(r) for r in reqs]
        for i in ids:
            srv.wait(i, timeout=7200)
        srv.stop()
        out = srv.summary()
        for r in reqs:
            if r.result is not None:
                r.result.close()
                r.result = None
        return out

    first = stream(0.0)
    torch.cuda.synchronize()
    forms = {}
    for r in first:
        k = f"{r.prec}/{r.A.info()['bs']}"
        forms[k] = forms.get(k, 0) + 1
    del first
    serve(stream(0.0, count=min(8, args.serve_requests)))  # warm-up
    sat = serve(stream(0.0))
    cap = sat["requests_per_s"]
    load = serve(stream(0.9 * cap))
    prefix = None
    if args.serve_fp64_prefix:
        k = min(args.serve_fp64_prefix, args.serve_requests)
        prefix = {"requests": k, "arrivals": "all at t = 0 (the stream's first requests)",
                  "chosen_forms": serve(stream(0.0, count=k)), "fp64": serve(stream(0.0, forced="fp64", count=k))}
    line = {"metric": "requests/s (served stream)", "value": load["requests_per_s"], "unit": "req/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": compute_dtype(args.prec), "data": "synthetic",
            "config": {"workload": "served_stream", "requests": args.serve_requests, "inputs": args.serve_inputs,
                       "resident_inputs": [{"n": specs[i][0], "alpha": specs[i][1]} for i in live],
                       "dropped_inputs": dropped, "n_range": [4096, args.serve_nmax],
                       "alpha": list(args.serve_alpha), "tau": taus, "method": "combined", "forms": forms,
                       "arrivals": "Poisson at 0.9 x saturated capacity", "slice_ms": args.serve_slice_ms,
                       "rate_guess": guess},
            "saturated": sat, "loaded": load, "p50_s": load["p50_s"], "p99_s": load["p99_s"],
            "kept_gflops": load["kept_gflops"], "prefix_vs_fp64": prefix}
    print(json.dumps(line), flush=True)


# ------------------------------------------------ methods at equal accuracy
def tau_sweep(S, ctx, GA, GB, taus, sigmas, precs=("fp64",)):
    """The paper's comparison of the three methods (Section 5.3): multiply with
    each method over a tau grid, measure ||AB - C||_F against the exact product
    (tau = 0, no truncation, FP64), and for each target accuracy sigma take,
    per method (and precision form), the largest tau whose error is <= sigma.
    Times are wall time of the synchronous multiply (truncation + task list +
    operand prep + leaf products + C norms)."""
    X, xs = S.spamm_multiply(ctx, GA, GB, 0.0, "spamm", "fp64", stats=True)
    exact = {"n_kept": xs["n_kept"], "frob": S.spamm_frob_norm(ctx, X), "ms_gemm": xs["ms_gemm"]}
    rows = {}
    for prec in precs:
        S.spamm_multiply(ctx, GA, GB, max(taus), "spamm", prec).close()  # first launch of this form, untimed
        for mode in ("truncate", "spamm", "combined"):
            key = mode if prec == "fp64" else f"{mode}/{prec}"
            rows[key] = []
            for tau in taus:
                t0 = time.perf_counter()
                C, st = S.spamm_multiply(ctx, GA, GB, tau, mode, prec, stats=True)
                ms = 1e3 * (time.perf_counter() - t0)
                err = S.spamm_error(ctx, X, C)
                rows[key].append({"tau": tau, "n_kept": st["n_kept"], "error": err, "ms": ms,
                                  "ms_gemm": st["ms_gemm"], "gflops": st["kept_flops"] / ms / 1e6,
                                  "mults_per_s": st["n_kept"] / ms * 1e3})
                C.close()
    X.close()
    chosen = {}
    for sigma in sigmas:
        pick = {}
        for key, rs in rows.items():
            ok = [r for r in rs if r["error"] <= sigma]
            pick[key] = max(ok, key=lambda r: r["tau"]) if ok else None
        base = pick.get("truncate")
        chosen["%g" % sigma] = {
            m: (c and {"tau": c["tau"], "n_kept": c["n_kept"], "error": c["error"], "ms": c["ms"],
                       "gflops": c["gflops"], "mults_per_s": c["mults_per_s"],
                       "gemm_vs_truncmul": c["n_kept"] / base["n_kept"] if base else None,
                       "time_vs_truncmul": c["ms"] / base["ms"] if base else None})
            for m, c in pick.items()}
    return {"exact": exact, "chosen": chosen, "sweep": rows}


def run_sweep(args, cfg):
    """Equal-accuracy comparison on a bench workload (default: the 3-D lattice,
    tau in {1e-4, 1e-6, 1e-8}, sigma in {1e-2, 1e-4, 1e-6})."""
    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm as S

    ctx = S.Context(0)
    pa = synth.DecayParams(n=cfg["n"], kind=cfg["kind"], alpha=cfg["alpha"], seed=cfg["seeds"][0])
    pb = synth.DecayParams(n=cfg["n"], kind=cfg["kind"], alpha=cfg["alpha"], seed=cfg["seeds"][1])
    GA = S.spamm_generate(ctx, pa, cfg["bs"])
    GB = GA if pb == pa else S.spamm_generate(ctx, pb, cfg["bs"])
    res = tau_sweep(S, ctx, GA, GB, args.sweep_taus, args.sigmas, args.sweep_precs)
    print(json.dumps({"metric": "methods at equal accuracy", "unit": "ms", "data": "synthetic",
                      "config": {"workload": args.config, "desc": cfg["desc"], "bs": cfg["bs"],
                                 "taus": args.sweep_taus, "sigmas": args.sigmas, "precisions": args.sweep_precs},
                      **res}), flush=True)
    for m in {id(GA): GA, id(GB): GB}.values():
        m.close()


def run_model_problem(args):
    """The paper's single-node model problem (Section 5.3): a 1-D decay matrix,
    a_ij = u_ij exp(-0.005 |i-j|) (|a_ij| <= exp(-0.005 |i-j|)), elements below
    1e-16 set to zero, n = 40000, multiplied by itself with the three methods,
    tau = 1e-4 ... 1e-12, target accuracy sigma = 1e-6; per leaf size the
    chosen tau of each method and its leaf products (gemm calls) and time
    relative to Truncmul."""
    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm as S

    ctx = S.Context(0)
    p = synth.model_1d(args.mp_n, alpha=0.005, seed=1)
    taus = [10.0 ** -e for e in range(args.mp_tau_lo, args.mp_tau_hi + 1)]
    out = {"metric": "model problem: methods at equal accuracy", "unit": "ms", "data": "synthetic",
           "config": {"workload": "model_problem_1d", "n": args.mp_n, "alpha": 0.005, "cutoff": 1e-16,
                      "sigma": args.mp_sigma, "taus": taus, "precision": "fp64"}, "by_bs": {}}
    for bs in args.mp_bs:
        G = S.spamm_generate(ctx, p, bs)
        out["by_bs"][str(bs)] = tau_sweep(S, ctx, G, G, taus, [args.mp_sigma])
        G.close()
    print(json.dumps(out), flush=True)


# ------------------------------------------------ random block-sparse inputs
def run_block_sparse(args):
    """Section 5.2's leaf-library benchmark: two n x n matrices (n = 2048)
    whose non-zero blocks are placed uniformly at random with fill-in factor
    f, multiplied at tau = 0 (every non-null pair is a product; FP64).  Per
    (bs, f): kept-block GFLOP/s (2 bs^3 x products / time of the whole
    multiply), and the time of the quadtree task-list build (the predictor)
    relative to the leaf products, the ratio the paper reports as ~1e-4 on
    its CPU cluster."""
    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm as S

    ctx = S.Context(0)
    rows = []
    for bs in args.bsp_bs:
        for fill in args.bsp_fills:
            A = S.spamm_from_blocks(ctx, args.bsp_n, bs, *synth.block_sparse(args.bsp_n, bs, fill, seed=1))
            B = S.spamm_from_blocks(ctx, args.bsp_n, bs, *synth.block_sparse(args.bsp_n, bs, fill, seed=2))
            for _ in range(2):
                S.spamm_multiply(ctx, A, B, 0.0, "spamm", args.prec).close()
            ms, sts = [], []
            for _ in range(args.bsp_repeats):
                t0 = time.perf_counter()
                C, st = S.spamm_multiply(ctx, A, B, 0.0, "spamm", args.prec, stats=True)
                ms.append(1e3 * (time.perf_counter() - t0))
                sts.append(st)
                C.close()
            med = statistics.median(ms)
            tasks = statistics.median(s["ms_tasks"] for s in sts)
            gemm = statistics.median(s["ms_gemm"] for s in sts)
            rows.append({"bs": bs, "fill": fill, "a_blocks": A.info()["nleaves"], "n_kept": sts[0]["n_kept"],
                         "ms": med, "gflops": sts[0]["kept_flops"] / med / 1e6,
                         "gemm_gflops": sts[0]["kept_flops"] / gemm / 1e6, "ms_tasks": tasks, "ms_gemm": gemm,
                         "predictor_over_multiply": tasks / gemm})
            A.close()
            B.close()
    print(json.dumps({"metric": "random block-sparse multiply, tau = 0", "unit": "GFLOP/s", "data": "synthetic",
                      "config": {"workload": "block_sparse", "n": args.bsp_n, "precision": args.prec,
                                 "repeats": args.bsp_repeats, "timing": "median wall time of the synchronous call"},
                      "rows": rows}), flush=True)


# ------------------------------------------------------ purification chains
def run_chain(args):
    """Repeated squaring X <- X X with the state resident on the device (the
    purification-style chain): 3-D lattice decay matrix scaled by an upper
    bound of its spectral norm (so ||X0||_2 <= 1), combined method, 64 x 64
    leaves, `--chain-steps` squarings, FP64 leaves and a tensor-core form.
    Squaring a matrix of spectral radius < 1 drives it to 0, so the work per
    step shrinks as leaves fall below tau; that is reported, not hidden.
    Per form: total and per-step time, kept products and ||X||_F; and the
    relative difference of the two forms' final X."""
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1906_08148_gb300 import chain
    from paper_1906_08148_gb300 import spamm as S

    ctx = S.Context(0)
    p = synth.lattice_3d(args.chain_n, alpha=args.chain_alpha, seed=1)
    bound = synth.spectral_bound(p)
    ps = synth.DecayParams(n=p.n, kind=p.kind, alpha=p.alpha, seed=p.seed, c=1.0 / bound)
    out = {"metric": "purification-style squaring chain", "unit": "s", "data": "synthetic",
           "config": {"workload": "square_chain", "n": args.chain_n, "alpha": args.chain_alpha, "bs": 64,
                      "tau": args.chain_tau, "method": "combined", "steps": args.chain_steps,
                      "scale": "1 / spectral bound %.6g" % bound, "inputs": "generated with block truncation at tau"},
           "forms": {}}
    finals = {}
    for prec in args.chain_precs:
        X0 = S.spamm_generate(ctx, ps, 64, args.chain_tau)
        nl0 = X0.info()["nleaves"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, hist = chain.square_chain(ctx, X0, args.chain_steps, args.chain_tau, "combined", prec, keep_input=False)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        flops = sum(h["kept_flops"] for h in hist)
        out["forms"][prec] = {"seconds": secs, "x0_leaves": nl0, "kept_flops": flops,
                              "kept_gflops": flops / secs / 1e9, "steps": hist}
        finals[prec] = X
    if "fp64" in finals:
        ref = S.spamm_frob_norm(ctx, finals["fp64"])
        for prec, X in finals.items():
            if prec != "fp64":
                e = S.spamm_error(ctx, finals["fp64"], X)
                out["forms"][prec]["diff_vs_fp64"] = e / ref if ref > 0 else e
    for X in finals.values():
        X.close()
    print(json.dumps(out), flush=True)


SP2_GROWTH = 1.75  # state leaves of the converged projector / leaves of X0 (1.71 measured at n = 262144)
SP2_PEAK = 3.7     # peak device bytes / (state leaves x 8 bs^2) (3.6 measured at n = 262144, FP16 form)


def sp2_estimate(p, bs, delta, tau, rows=16, held=0):
    """Leaves of X0 = (bI - F) / (2b) before any allocation: the generator's
    leaves of block rows sampled evenly over the matrix whose norm / (2b)
    reaches tau, plus the diagonal leaf, scaled to all block rows; and the
    chain's estimated peak device footprint (the state grows by SP2_GROWTH
    towards the projector; a product holds the previous state, its
    untruncated square and, on the 2X - X^2 branch, the sum: SP2_PEAK times
    the state; `held` more states kept meanwhile)."""
    import numpy as np

    import synth
    b = delta + synth.spectral_bound(p)
    thr = 2.0 * b * tau
    nb = -(-p.n // bs)
    cols = np.arange(nb)
    counts = []
    for r in np.linspace(0, nb - 1, min(rows, nb)).astype(np.int64):
        bnd = synth.leaf_bounds_row(p, bs, int(r), cols)
        cand = cols[bs * bnd >= thr]
        d = synth.leaves(p, bs, np.full(len(cand), r), cand)
        nrm = np.sqrt(np.sum(d * d, axis=(1, 2)))
        counts.append(int(np.count_nonzero((nrm >= thr) | (cand == r))))
    leaves = float(np.mean(counts)) * nb
    peak = leaves * SP2_GROWTH * (SP2_PEAK + held) * 8 * bs * bs
    return {"x0_leaves_est": int(leaves), "peak_bytes_est": int(peak), "bound": b, "v_threshold": thr}


def sp2_probe_rows(S, ctx, X, X2, rows, tau, n, bs):
    """Block rows `rows` of the product X X three ways, all on the device:
    exact (every non-zero leaf pair, FP64), the method in FP64 (combined at
    tau) and the chain's own product X2.  Returns the sampled rows' squared
    norms: ||exact - method||^2, ||method - X2||^2, ||exact||^2."""
    import numpy as np
    bi, bj, _, _ = S.spamm_to_blocks(ctx, X, payload=False)
    sel = np.isin(bi, rows)
    pay, _ = S.spamm_gather_leaves(ctx, X, bi[sel], bj[sel])
    XR = S.spamm_from_blocks(ctx, n, bs, bi[sel], bj[sel], pay)
    E = S.spamm_multiply(ctx, XR, X, 0.0, "spamm", "fp64")
    M = S.spamm_multiply(ctx, XR, X, tau, "combined", "fp64")
    ei, ej, _, _ = S.spamm_to_blocks(ctx, E, payload=False)
    tp, found = S.spamm_gather_leaves(ctx, X2, ei, ej)
    TR = S.spamm_from_blocks(ctx, n, bs, ei[found], ej[found], tp[found])
    out = (S.spamm_error(ctx, E, M) ** 2, S.spamm_error(ctx, M, TR) ** 2, S.spamm_frob_norm(ctx, E) ** 2)
    for m in (XR, E, M, TR):
        m.close()
    return out


def run_sp2(args):
    """SP2 purification (second-order spectral projection) of a gapped
    two-sublattice insulator on the 3-D lattice: F = V + D, V the decay
    matrix (alpha, seed 1), D the on-site term -+delta by sublattice, n_occ =
    the -delta sites; X0 = (b I - F) / (2 b) with b = delta + the Gershgorin
    bound of V, then X <- X^2 or 2X - X^2 by the trace rule, every product an
    approximate multiply (combined method at tau), the state resident on the
    device.  The sizes of --sp2-n are tried from the largest: a size whose
    estimated footprint exceeds the free device memory is refused before
    anything is allocated (and one that runs out of memory is recorded), the
    chain runs at the largest admitted size.  Per form and iteration: branch,
    traces, ||X - X^2||_F, kept products and time, device memory in use;
    every --sp2-probe-every iterations the sampled-row errors of the product
    (method against exact, the form against the method in FP64).  FP64 runs
    --sp2-fp64-iters products, and the tensor form's product after as many
    iterations is compared with it."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1906_08148_gb300 import chain
    from paper_1906_08148_gb300 import spamm as S

    ctx = S.Context(0)
    bs = 64
    out = {"metric": "SP2 purification chain", "unit": "s", "data": "synthetic",
           "config": {"workload": "sp2_insulator", "alpha": args.sp2_alpha, "delta": args.sp2_delta, "bs": bs,
                      "tau": args.sp2_tau, "method": "combined", "iterations": args.sp2_iters,
                      "sizes_tried": sorted(args.sp2_n, reverse=True)},
           "admission": [], "forms": {}}
    free0, total = torch.cuda.mem_get_info()
    budget = args.sp2_budget * free0
    forms = sorted(args.chain_precs, key=lambda q: q != "fp64")  # FP64 first: the forms compare with it
    fp64_iters = args.sp2_iters if args.sp2_fp64_iters is None else args.sp2_fp64_iters
    out["config"]["fp64_iterations"] = fp64_iters
    for n in sorted(args.sp2_n, reverse=True):
        p = synth.lattice_3d(n, alpha=args.sp2_alpha, seed=1)
        # the FP64 chain's final state is kept while the tensor forms run, to compare with
        est = sp2_estimate(p, bs, args.sp2_delta, args.sp2_tau,
                           held=int("fp64" in forms and len(forms) > 1))
        rec = {"n": n, **est, "budget_bytes": int(budget)}
        if est["peak_bytes_est"] > budget and not args.sp2_force:
            rec["admission"] = "refused (estimated footprint above the free device memory)"
            out["admission"].append(rec)
            continue
        thr = est["v_threshold"]
        pv = synth.DecayParams(n=n, kind=p.kind, alpha=p.alpha, seed=p.seed)
        di, dj, dd, n_occ = synth.onsite_blocks(n, bs, args.sp2_delta)
        nb = -(-n // bs)
        rows = np.unique(np.linspace(nb // 8, nb - 1 - nb // 8, args.sp2_probe_rows).astype(np.int32))

        def start():
            """X0 = (b I - F) / (2 b), F = V + D; F itself is not kept."""
            V = S.spamm_generate(ctx, pv, bs, thr)
            D = S.spamm_from_blocks(ctx, n, bs, di, dj, dd)
            F = S.spamm_add(ctx, 1.0, V, 1.0, D)
            V.close()
            D.close()
            I = S.spamm_identity(ctx, n, bs)
            X0 = S.spamm_add(ctx, -0.5 / est["bound"], F, 0.5, I)
            F.close()
            I.close()
            return X0

        res, fp64_prod, fp64_final, fp64_hist = {}, None, None, None
        try:
            for prec in forms:
                iters = fp64_iters if prec == "fp64" else args.sp2_iters
                X0 = start()
                x0_leaves = X0.info()["nleaves"]
                used, keep, probe_s = [], {}, [0.0]

                def probe(it, X, X2, prec=prec, used=used, keep=keep, probe_s=probe_s):
                    torch.cuda.synchronize()
                    t_in = time.perf_counter()
                    f, _ = torch.cuda.mem_get_info()
                    used.append(total - f)
                    d = {"device_bytes_in_use": int(total - f), "x_leaves": X.info()["nleaves"],
                         "product_leaves": X2.info()["nleaves"]}
                    if prec != "fp64" and fp64_prod is not None and it == fp64_iters - 1 < args.sp2_iters - 1:
                        ref = S.spamm_frob_norm(ctx, fp64_prod)
                        d["product_diff_vs_fp64_chain"] = S.spamm_error(ctx, fp64_prod, X2) / ref
                    if prec == "fp64" and it == iters - 1 and iters < args.sp2_iters:
                        keep["prod"] = S.spamm_add(ctx, 1.0, X2, 0.0, X2)
                    if args.sp2_probe_every and (it % args.sp2_probe_every == 0 or it == iters - 1):
                        ea, ef, ex = sp2_probe_rows(S, ctx, X, X2, rows, args.sp2_tau, n, bs)
                        d["sampled_rows"] = rows.tolist()
                        d["sampled_error_vs_exact"] = float(np.sqrt(ea / ex))
                        d["sampled_form_vs_fp64_method"] = float(np.sqrt(ef / ex))
                    torch.cuda.synchronize()
                    probe_s[0] += time.perf_counter() - t_in
                    return d

                torch.cuda.synchronize()
                t0 = time.perf_counter()
                X, hist = chain.sp2(ctx, None, n_occ, est["bound"], args.sp2_tau, "combined", prec, iters,
                                    tol=args.sp2_tol, X0=X0, probe=probe)
                torch.cuda.synchronize()
                secs = time.perf_counter() - t0 - probe_s[0]
                flops = sum(h["kept_flops"] for h in hist)
                gemm_s = sum(h["ms_gemm"] for h in hist) / 1e3
                res[prec] = {"seconds": secs, "probe_seconds": probe_s[0], "iterations": len(hist),
                             "kept_flops": flops,
                             "kept_gflops_gemm": flops / gemm_s / 1e9 if gemm_s > 0 else None,
                             "final_trace": S.spamm_trace(ctx, X), "n_occ": n_occ, "x0_leaves": x0_leaves,
                             "final_leaves": X.info()["nleaves"], "peak_device_bytes_sampled": max(used),
                             "note": "seconds: the chain (products, adds, traces, ||X - X^2||_F), probes excluded",
                             "history": hist}
                if "prod" in keep:
                    fp64_prod = keep["prod"]
                if prec == "fp64":
                    fp64_final, fp64_hist = X, hist
                else:
                    if fp64_final is not None and len(fp64_hist) == len(hist):
                        res[prec]["final_diff_vs_fp64_chain"] = (S.spamm_error(ctx, fp64_final, X) /
                                                                 S.spamm_frob_norm(ctx, fp64_final))
                        res[prec]["same_branches_as_fp64"] = sum(
                            a["branch"] == b["branch"] for a, b in zip(hist, fp64_hist))
                    X.close()
        except S.SpammError as e:
            if e.status != S.E_OOM:
                raise
            rec["admission"] = "admitted; ran out of device memory (%s)" % str(e)[:160]
            rec["partial"] = {k: {kk: v[kk] for kk in ("seconds", "iterations")} for k, v in res.items()}
            out["admission"].append(rec)
            res = fp64_prod = fp64_final = fp64_hist = None
            gc.collect()
            S.spamm_trim(ctx)
            continue
        rec["admission"] = "admitted"
        out["admission"].append(rec)
        out["config"]["n"] = n
        out["config"]["n_occ"] = n_occ
        out["config"]["bound"] = est["bound"]
        out["forms"] = res
        for m in (fp64_prod, fp64_final):
            if m is not None:
                m.close()
        break
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------- multi-rank timing
def run_passes(args, cfg):
    """The two passes around the leaf GEMM, timed with CUDA events on the
    bench workload.  Kernel (a), the leaf norms, in its allocation-free form
    (the same per-leaf arithmetic) over as many random 64 x 64 leaves as the
    workload's truncated input has (far above L2; L2 written over before each
    run): bytes read and written / time.  Kernel (b), the task list, inside
    the multiply (FP16 form, whose leaf products are short): its algorithmic
    traffic per level, per kept parent pair its two node indices (8 B), both
    nodes' child-norm records (2 x 32 B) and child links (2 x 16 B), and 8 B
    per kept child written, over the task-list time the library reports."""
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm as S

    stream = torch.cuda.current_stream()
    ctx = S.Context(0, stream=stream)
    bs = cfg["bs"]
    GA = S.spamm_generate(ctx, synth.DecayParams(n=cfg["n"], kind=cfg["kind"], alpha=cfg["alpha"],
                                                 seed=cfg["seeds"][0]), bs)
    GB = S.spamm_generate(ctx, synth.DecayParams(n=cfg["n"], kind=cfg["kind"], alpha=cfg["alpha"],
                                                 seed=cfg["seeds"][1]), bs)
    tasks = []
    for _ in range(max(2, args.steps)):
        C, st = S.spamm_multiply(ctx, GA, GB, args.tau, args.mode, "fp16_scaled" if bs == 64 else "fp64", stats=True)
        C.close()
        tasks.append(st)
    st = tasks[-1]
    kept = [1] + list(st["n_kept_level"])  # the root pair, then every level's kept pairs
    task_bytes = 104.0 * sum(kept[:-1]) + 8.0 * sum(kept[1:])
    ms_tasks = statistics.median(s["ms_tasks"] for s in tasks[1:])
    nl = st["n_a_leaves"]
    pay = torch.rand(nl * bs * bs, dtype=torch.float64, device="cuda")
    sq = torch.empty(nl, dtype=torch.float64, device="cuda")
    tot = torch.empty(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ms = []
    for _ in range(max(4, args.steps)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if S.spamm_leaf_sqnorms_noalloc(pay, nl, bs, sq, tot, stream) != 0:
            raise RuntimeError("spamm_leaf_sqnorms_noalloc failed")
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    norm_ms = statistics.median(ms[1:])
    norm_bytes = nl * (bs * bs * 8 + 8)
    # the library's own norm pass (leaf_sqnorm_kernel) runs inside a build from
    # device-resident leaves; its time is read from the ncu launch list
    bi, bj, pay_h, _ = S.spamm_to_blocks(ctx, GA)
    dbi, dbj = torch.from_numpy(bi).cuda(), torch.from_numpy(bj).cuda()
    dpay = torch.from_numpy(pay_h).cuda()
    del pay_h
    for _ in range(2):
        S.spamm_from_blocks(ctx, cfg["n"], bs, dbi, dbj, dpay).close()
    torch.cuda.synchronize()
    del dbi, dbj, dpay
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    print(json.dumps({
        "metric": "pass bandwidth", "unit": "GB/s", "data": "synthetic",
        "config": {"workload": args.config, "method": args.mode, "tau": args.tau},
        "hbm_peak_gbs": hbm, "hbm_peak_source": "MEASURED_PEAKS.json" if "hbm_gbs" in peaks else "fallback",
        "norm_pass": {"kernel": "noalloc_sqnorm_kernel", "leaves": nl, "bytes": norm_bytes, "ms": norm_ms,
                      "gbs": norm_bytes / norm_ms / 1e6, "frac": norm_bytes / norm_ms / 1e6 / hbm},
        "task_pass": {"levels": st["levels"], "candidates": st["n_candidates"], "kept": st["n_kept_level"],
                      "bytes": task_bytes, "ms": ms_tasks, "gbs": task_bytes / ms_tasks / 1e6,
                      "frac": task_bytes / ms_tasks / 1e6 / hbm}}), flush=True)


def aggregate_ranks(ms_local, flops_local, kept_local, dist=None):
    """Whole-job numbers over independent replicas (one per GPU): the timed
    region is the slowest rank's, the work is every rank's.
    Returns (ms, GFLOP/s, mults/s)."""
    import torch
    ms, flops, kept = float(ms_local), float(flops_local), float(kept_local)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        w = torch.tensor([flops, kept], dtype=torch.float64)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
        ms, flops, kept = float(t[0]), float(w[0]), float(w[1])
    return ms, flops / (ms / 1e3) / 1e9, kept / (ms / 1e3)


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse_args()
    cfg = CONFIGS[args.config]
    resolve_defaults(args)
    if args.impl == "reference":
        return run_reference(args, cfg)
    if args.serve:
        return run_served(args)
    if args.prec == "auto":
        raise SystemExit("--prec auto applies to the served stream (--serve)")
    if args.model_problem:
        return run_model_problem(args)
    if args.sweep:
        return run_sweep(args, cfg)
    if args.block_sparse:
        return run_block_sparse(args)
    if args.chain:
        return run_chain(args)
    if args.sp2:
        return run_sp2(args)
    if args.passes:
        return run_passes(args, cfg)
    if args.config == "lattice262144":
        return run_precision_config(args, cfg)

    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = S.Context(local, stream=stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    pa = synth.DecayParams(n=cfg["n"], kind=cfg["kind"], alpha=cfg["alpha"], seed=cfg["seeds"][0])
    pb = synth.DecayParams(n=cfg["n"], kind=cfg["kind"], alpha=cfg["alpha"], seed=cfg["seeds"][1])
    bs = cfg["bs"]
    GA = S.spamm_generate(ctx, pa, bs)
    GB = GA if pb == pa else S.spamm_generate(ctx, pb, bs)
    choice = None
    if args.headline:
        args.prec, choice = equal_accuracy_choice(S, ctx, GA, GB, args, stream, torch)

    def step():
        C, st = S.spamm_multiply(ctx, GA, GB, args.tau, args.mode, args.prec, stats=True)
        nrm = S.spamm_frob_norm(ctx, C)
        C.close()
        return st, nrm

    # inputs smaller than twice the L2: write a 256 MB buffer before every step, outside its events
    in_bytes = (GA.info()["nleaves"] + (0 if GB is GA else GB.info()["nleaves"])) * bs * bs * 8
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if in_bytes < 2 * L2_BYTES else None
    for _ in range(args.warmup):
        st0, nrm0 = step()
    barrier()
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stats = []
    with ClockSampler(local) as clk:
        barrier()
        for k in range(args.steps):
            if flush is not None:
                flush.zero_()
            ev_a[k].record(stream)
            st, nrm = step()
            stats.append(st)
            ev_b[k].record(stream)
        barrier()
    per_step = sorted(ev_a[k].elapsed_time(ev_b[k]) for k in range(args.steps))
    # latency percentiles over at least --latency-repeats warm multiplies: the
    # timed steps plus further ones, each between its own events (not part of
    # the throughput above)
    lat = list(per_step)
    extra = max(0, args.latency_repeats - args.steps) if rank == 0 else 0
    if extra:
        ex_a = [torch.cuda.Event(enable_timing=True) for _ in range(extra)]
        ex_b = [torch.cuda.Event(enable_timing=True) for _ in range(extra)]
        for k in range(extra):
            if flush is not None:
                flush.zero_()
            ex_a[k].record(stream)
            step()
            ex_b[k].record(stream)
        torch.cuda.synchronize()
        lat += [ex_a[k].elapsed_time(ex_b[k]) for k in range(extra)]
    latency = latency_summary(lat)
    ms_total, value, mults = aggregate_ranks(sum(per_step), sum(s["kept_flops"] for s in stats),
                                             sum(s["n_kept"] for s in stats), dist)
    clocks = clk.summary()

    ms_gemm = statistics.mean(s["ms_gemm"] for s in stats)
    kept = stats[-1]["n_kept"]
    phases = {k: statistics.mean(s[k] for s in stats)
              for k in ("ms_truncate", "ms_tasks", "ms_prep", "ms_gemm", "ms_cnorm")}

    forms = None
    if not args.no_forms and rank == 0 and args.prec == "fp64" and bs == 64:  # tensor forms: 64 x 64 leaves
        forms = precision_forms(S, ctx, GA, GB, args, stream, torch)

    # last on the device: the end-to-end steps take the inputs over (copied to
    # pinned host buffers, their device copies released) and start from a
    # trimmed pool, so the earlier phases' cached blocks of other sizes do not
    # crowd the device when the end-to-end steps allocate
    e2e = None
    if not args.no_e2e and rank == 0:
        e2e = run_e2e(S, ctx, GA, GB, args, bs, torch, np)
        GA = GB = None

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline(cfg, args.mode, args.tau, args.cpu_seconds)

    if rank == 0:
        roof = roofline(args.prec, bs, kept, ms_gemm, statistics.mean(s["executed_flops"] for s in stats))
        in_gb = in_bytes / 1e9
        line = {
            "metric": "kept-block GFLOP/s", "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": compute_dtype(args.prec), "data": "synthetic",
            "config": {"workload": args.config, "desc": cfg["desc"], "n": cfg["n"], "bs": bs, "method": args.mode,
                       "tau": args.tau, "precision": args.prec,
                       "sigma": args.sigma if args.headline else None, "l2": ("inputs (%.1f GB of leaves) larger than L2" % in_gb) if flush is None
                       else "L2 flushed before every step (256 MB write, outside the step's events)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "mults_per_s": mults,
            "n_kept": kept, "n_steps": stats[-1]["n_steps"], "n_c_leaves": stats[-1]["n_c_leaves"], "n_borderline": stats[-1]["n_borderline"],
            "n_a_leaves": stats[-1]["n_a_leaves"], "n_b_leaves": stats[-1]["n_b_leaves"],
            "c_frob": nrm, "phase_ms": phases, "latency": latency, "roofline": roof,
            "gpu_launches": None, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu, "precision_forms": forms,
            "equal_accuracy": choice,
        }
        if choice is not None:
            fp = choice["forms"]["fp64"]
            choice["vs_fp64"] = {"kept_gflops": value / fp["kept_gflops"],
                                 "mults_per_s": mults / fp["mults_per_s"],
                                 "note": "this line's timed steps against one timed FP64 step at the same tau"}
        line["gpu_launches"] = int(sum(s["n_launches"] for s in stats))
        if forms:
            for f in forms.values():
                f["vs_fp64"] = f["kept_gflops"] / value if value else None
        print(json.dumps(line), flush=True)
    for m in {id(GA): GA, id(GB): GB}.values():
        if m is not None:
            m.close()
    if dist is not None:
        dist.destroy_process_group()


def run_precision_config(args, cfg):
    """The precision-form configuration: X times X for the 64^3 lattice
    (n = 262144, alpha = 0.8, X symmetric, 64 x 64 leaves), combined, at each
    tau of --pc-taus.  X is generated with the block rule applied while
    generating (the same leaves as truncating the full matrix, which would not
    fit).  Each tensor form: plan (one set of operand terms for both roles,
    X being symmetric), release X, execute: --warmup untimed and --steps timed
    executions (CUDA events), output leaves sampled for the comparison with
    FP64; the FP64 form then runs the same multiply once (timed), where it
    fits.  A step is the plan's phases (truncation, task list, operand terms,
    device-timed by the library) plus one execution.  A form is admissible at tau if its error against FP64 on the
    sampled leaves, scaled to the whole output, stays below the lower end of
    the oracle's sampled truncation error (tests/golden/accuracy.json).  The
    line's value is the fastest admissible form at the smallest tau."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm as S

    stream = torch.cuda.current_stream()
    ctx = S.Context(0, stream=stream)
    p = synth.DecayParams(n=cfg["n"], kind=cfg["kind"], alpha=cfg["alpha"], seed=cfg["seeds"][0])
    bs, nb = cfg["bs"], cfg["n"] // cfg["bs"]
    rng = np.random.default_rng(3)
    # sampled output leaves: the diagonal band and scattered positions near it
    ii = rng.integers(0, nb, args.pc_samples)
    jj = np.clip(ii + rng.integers(-40, 41, args.pc_samples), 0, nb - 1)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    per_tau = {}
    with ClockSampler(0) as clk:
        for tau in args.pc_taus:
            trunc = accuracy_entry("lattice262144_square", "combined", tau)
            rec = {"truncation_error": trunc, "forms": {}}
            samples = {}
            for prec in TC_FORMS + (() if args.pc_no_fp64 else ("fp64",)):
                X = S.spamm_generate(ctx, p, bs, tau)
                nx = X.info()["nleaves"]
                try:
                    plan = S.spamm_plan_create(ctx, X, X, tau, "combined", prec)
                except S.SpammError as e:
                    X.close()
                    rec["forms"][prec] = {"admission": "refused: %s" % e}
                    continue
                if prec != "fp64":
                    X.close()  # the plan keeps the operand terms only
                info = plan.info()
                out = {"x_leaves": nx, "plan_gb": info["plan_bytes"] / 1e9, "exec_gb": info["exec_bytes"] / 1e9}
                try:
                    steps = 1 if prec == "fp64" else args.steps
                    for _ in range(0 if prec == "fp64" else args.warmup):
                        (C,) = S.spamm_execute(ctx, [plan])
                        C.close()
                    ms, st = [], None
                    for _ in range(steps):
                        e0, e1 = ev(), ev()
                        e0.record(stream)
                        (C,), (st,) = S.spamm_execute(ctx, [plan], stats=True)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        ms.append(e0.elapsed_time(e1))
                        last = C
                        if len(ms) < steps:
                            C.close()
                    samples[prec], found = S.spamm_gather_leaves(ctx, last, ii, jj)
                    samples[prec] = np.where(found[:, None, None], samples[prec], 0.0)
                    cn = S.spamm_frob_norm(ctx, last)
                    last.close()
                except S.SpammError as e:
                    out["admission"] = "refused at execution: %s" % e
                    rec["forms"][prec] = out
                    plan.close()
                    if prec == "fp64":
                        X.close()
                    continue
                plan.close()
                if prec == "fp64":
                    X.close()
                # a step: the plan's phases (truncation, task list, operand terms; device-timed by the
                # library when the plan was made) plus one execution (CUDA events)
                msx = st["ms_truncate"] + st["ms_tasks"] + st["ms_prep"] + statistics.median(ms)
                out.update({"admission": "ran", "ms_per_step": msx, "ms_execute": statistics.median(ms),
                            "ms_gemm": st["ms_gemm"], "ms_truncate": st["ms_truncate"],
                            "ms_prep": st["ms_prep"], "ms_tasks": st["ms_tasks"], "n_kept": st["n_kept"],
                            "n_steps": st["n_steps"], "n_c_leaves": st["n_c_leaves"],
                            "terms_shared": st["terms_shared"], "c_frob": cn,
                            "kept_gflops": st["kept_flops"] / msx / 1e6, "mults_per_s": st["n_kept"] / msx * 1e3,
                            "roofline": roofline(prec, bs, st["n_kept"], st["ms_gemm"], st["executed_flops"])})
                rec["forms"][prec] = out
            ref = samples.get("fp64")
            for prec, f in rec["forms"].items():
                if prec == "fp64" or prec not in samples or ref is None:
                    continue
                num = float(np.sqrt(np.sum((samples[prec] - ref) ** 2)))
                den = float(np.sqrt(np.sum(ref ** 2)))
                rel = num / den if den > 0 else 0.0
                arith = rel * rec["forms"]["fp64"]["c_frob"]
                f["arith_rel_sampled"] = rel
                f["arith_error_est"] = arith
                f["admissible"] = bool(trunc is not None and arith <= trunc["low"])
            per_tau["%g" % tau] = rec
    tau0 = "%g" % min(args.pc_taus)
    forms0 = per_tau[tau0]["forms"]
    ok = [k for k, f in forms0.items() if k != "fp64" and f.get("admissible")]
    chosen = min(ok, key=lambda k: forms0[k]["ms_per_step"]) if ok else (
        "fp64" if forms0.get("fp64", {}).get("admission") == "ran" else None)
    ch = forms0.get(chosen, {}) if chosen else {}
    fp = forms0.get("fp64", {})
    cpu = None if args.no_cpu else cpu_baseline(cfg, "combined", min(args.pc_taus), args.cpu_seconds)
    line = {"metric": "kept-block GFLOP/s", "value": ch.get("kept_gflops"), "unit": "GFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ch.get("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": compute_dtype(chosen), "data": "synthetic",
            "config": {"workload": "lattice262144", "desc": cfg["desc"], "n": cfg["n"], "bs": bs,
                       "method": "combined", "tau": min(args.pc_taus), "precision": chosen,
                       "l2": "inputs far larger than L2", "parallelism": "single"},
            "mults_per_s": ch.get("mults_per_s"), "roofline": ch.get("roofline"),
            "vs_fp64": ({"kept_gflops": ch["kept_gflops"] / fp["kept_gflops"]}
                        if chosen and chosen != "fp64" and fp.get("admission") == "ran" else None),
            "per_tau": per_tau, "clocks": clk.summary(), "cpu_baseline": cpu,
            "e2e": None, "e2e_note": "not run for this configuration (host staging of 100-250 GB per step)",
            "gpu_launches": None}
    print(json.dumps(line), flush=True)


def precision_forms(S, ctx, GA, GB, args, stream, torch):
    """The same multiply in the tensor-core forms, after the timed FP64 steps:
    kept-block GFLOP/s over `--form-steps` steps (CUDA events on the bench
    stream) and the form's deviation from the FP64 product of the same tau,
    ||C_form - C_fp64||_F / ||C_fp64||_F (the method's own truncation error
    at this tau, against the exact product, is what --sweep measures)."""
    ref = S.spamm_multiply(ctx, GA, GB, args.tau, args.mode, "fp64")
    nref = S.spamm_frob_norm(ctx, ref)
    out = {}
    for prec in ("bf16_split", "bf16_split4", "fp16_scaled"):
        C = S.spamm_multiply(ctx, GA, GB, args.tau, args.mode, prec)  # untimed first run of the form
        dev = S.spamm_error(ctx, ref, C) / nref
        C.close()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flops, gemm = 0.0, 0.0
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.form_steps):
            C, st = S.spamm_multiply(ctx, GA, GB, args.tau, args.mode, prec, stats=True)
            C.close()
            flops += st["kept_flops"]
            gemm += st["ms_gemm"]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.form_steps
        out[prec] = {"kept_gflops": flops / args.form_steps / ms / 1e6, "ms_per_step": ms,
                     "ms_gemm": gemm / args.form_steps, "rel_dev_vs_fp64": dev,
                     "vs_fp64": None}
    ref.close()
    return out


def roofline(prec, bs, kept, ms_gemm, executed_flops):
    """Roofline entry for the dominant kernel (the leaf GEMM), from the
    CUDA-event duration of its launch inside the timed steps.  executed_flops:
    what the kernel runs (tensor forms: every term product of every quad step
    over the full 128 x 128 x 64 tile, counted by the library)."""
    import json as _json
    algo = 2.0 * bs ** 3 * kept
    secs = ms_gemm / 1e3
    if prec == "fp64":
        achieved = algo / secs / 1e9
        kernel = f"gemm_fp64_kernel<{bs}>"
        return {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": achieved / FP64_PEAK_GFLOPS, "traffic": load_traffic(kernel, kept),
                "peak_source": "FP64 DFMA units x clock (derived; no FP64 entry in MEASURED_PEAKS.json)"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = _json.load(open(path)) if os.path.exists(path) else {}
    measured = "bf16_tflops_sustained" in peaks
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    achieved = algo / secs / 1e12
    executed = executed_flops / secs / 1e12
    kernel = "gemm_quad_kernel<%s>" % prec
    return {"kernel": kernel, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "executed": executed, "executed_frac": executed / peak,
            "traffic": load_traffic(kernel, kept),
            "peak_source": ("bf16 dense sustained, of measured (MEASURED_PEAKS.json)" if measured else
                            "bf16 dense sustained, of fallback (1.7 PFLOP/s; MEASURED_PEAKS.json absent)")
                           + "; fp16 dense has the same nominal rate"}


def load_traffic(kernel, kept):
    """DRAM bytes per GEMM launch: the committed ncu capture's bytes per kept leaf
    product times this launch's products; None once the kernel source has
    changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(kernel)
    if not d:
        return None
    src = open(os.path.join(ROOT, d["source"]), "rb").read()
    if hashlib.sha256(src).hexdigest()[:16] != d["source_sha256_16"]:
        return None
    return d["dram_bytes_per_product"] * kept


def compute_dtype(prec) -> str:
    """The arithmetic type a form's leaf products compute in (the form itself is
    named in the line's config): FP64 leaves "f64", the BF16 slice splits "bf16",
    the scaled FP16 form "f16"; the autotuned mix of the served stream "mixed"."""
    return {"fp64": "f64", "bf16_split": "bf16", "bf16_split4": "bf16", "fp16_scaled": "f16"}.get(prec, "mixed")


def latency_summary(ms) -> dict:
    """p50 and p99 (nearest rank) of per-multiply times in ms."""
    v = sorted(ms)
    return {"p50_ms": v[(len(v) - 1) // 2], "p99_ms": v[min(len(v) - 1, int(math.ceil(0.99 * len(v))) - 1)],
            "steps": len(v)}


def host_available_bytes() -> int:
    """MemAvailable of /proc/meminfo in bytes (0 where it cannot be read)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def run_e2e(S, ctx, GA, GB, args, bs, torch, np):
    """Same metric through the public API from host buffers: H2D of both
    inputs' leaves, multiply, D2H of every C leaf, all inside the timed region.
    GA and GB are copied to pinned host buffers and released here (the steps
    build their own device copies); the device pool is trimmed once before
    the untimed first step."""
    ia, ib = GA.info(), GB.info()
    e = bs * bs

    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()

    # The first large pinned block of a busy process can stream over the host
    # link well below its rate (measured: 0.2-0.7 s for a first 27.6 GB input
    # against 0.138 s for every later block of that size; a standalone process
    # shows full rate for its first block; cause not found).  One block the
    # size of an input's payload is pinned first and held, unused, when the
    # host has room for it, so that both inputs stream at the link's rate.
    reserve_bytes = ia["nleaves"] * e * 8
    reserve = None
    if 4 * reserve_bytes < host_available_bytes():
        reserve = pinned((ia["nleaves"], bs, bs), torch.float64)

    hA = (pinned(ia["nleaves"], torch.int32), pinned(ia["nleaves"], torch.int32),
          pinned((ia["nleaves"], bs, bs), torch.float64), pinned(ia["nleaves"], torch.float64))
    S.spamm_to_blocks(ctx, GA, out=hA)
    if GB is GA:
        hB = hA
    else:
        hB = (pinned(ib["nleaves"], torch.int32), pinned(ib["nleaves"], torch.int32),
              pinned((ib["nleaves"], bs, bs), torch.float64), pinned(ib["nleaves"], torch.float64))
        S.spamm_to_blocks(ctx, GB, out=hB)
    for m in {id(GA): GA, id(GB): GB}.values():
        m.close()
    S.spamm_trim(ctx)
    hC = None
    times, flops, h2d, d2h = [], 0.0, 0, 0
    phase = {"from_blocks_s": 0.0, "multiply_s": 0.0, "to_blocks_s": 0.0}
    per_step = []
    n = ia["n"]
    for it in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A = S.spamm_from_blocks(ctx, n, bs, hA[0], hA[1], hA[2])
        torch.cuda.synchronize()
        ta = time.perf_counter()
        B = A if hB is hA else S.spamm_from_blocks(ctx, n, bs, hB[0], hB[1], hB[2])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        C, st = S.spamm_multiply(ctx, A, B, args.tau, args.mode, args.prec, stats=True)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        nc = C.info()["nleaves"]
        if hC is None or len(hC[0]) < nc:
            hC = (pinned(nc, torch.int32), pinned(nc, torch.int32), pinned((nc, bs, bs), torch.float64),
                  pinned(nc, torch.float64))
            if it > 0:
                raise RuntimeError("C size changed between steps")
        if it == 0:
            # first pass sizes the pinned C buffer; time the next ones
            S.spamm_to_blocks(ctx, C, out=hC)
            for m in (C, A, B):
                m.close()
            continue
        S.spamm_to_blocks(ctx, C, out=hC)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        times.append(t3 - t0)
        for k, v in zip(phase, (t1 - t0, t2 - t1, t3 - t2)):
            phase[k] += v
        per_step.append({"from_blocks_A_s": ta - t0, "from_blocks_B_s": t1 - ta, "multiply_s": t2 - t1,
                         "to_blocks_s": t3 - t2})
        flops += st["kept_flops"]
        h2d = hA[2].nbytes + 8 * len(hA[0]) + (0 if hB is hA else hB[2].nbytes + 8 * len(hB[0]))
        d2h = 8 * nc * e + 16 * nc
        for m in {id(C): C, id(A): A, id(B): B}.values():
            m.close()
    held = reserve_bytes if reserve is not None else 0
    del reserve
    return {"value": flops / sum(times) / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": len(times), "ms_per_step": 1e3 * sum(times) / len(times),
            "host_reserve_bytes": held,
            "phases_s_per_step": {k: v / len(times) for k, v in phase.items()}, "per_step": per_step}


if __name__ == "__main__":
    main()
