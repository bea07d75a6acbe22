"""Continuous-batching request loop over the C ABI.

Requests (A, B, tau, mode, precision) arrive at any time and are served by
two host threads, each with its own libspamm context and CUDA stream:

* the planner takes arrived requests in order and creates their plans
  (truncation, quadtree descent, operand terms: spamm_plan_create).  Device
  memory is charged to the budget when planning starts (an estimate from the
  inputs' leaf counts), then corrected to the plan's footprint (plan + output
  bytes, spamm_plan_info); the planner waits while the charged bytes would
  exceed the budget, and a request whose footprint exceeds the whole budget
  is refused, not crashed;
* the executor runs the leaf products in slices (spamm_job_begin /
  spamm_run / spamm_job_finish): every planned request becomes a job at once,
  and each iteration is ONE persistent launch over the next units of every
  running job of one precision form and leaf size, sized so the launch takes
  about `slice_ms` (a work rate per form is measured as it goes).  Requests
  that arrive while others run therefore join the very next launches of their
  form: their units run in the same kernels as those of the requests already
  on the GPU, and a short request finishes without waiting for a long one.
  Forms take turns, one launch each.

While a launch executes, the planner keeps planning new arrivals on its own
stream; the executor's launches are kept off a few SMs (spamm_set_gemm_sms)
so those kernels can run beside them.  Each output is bit-identical to
multiplying the same request alone (every output leaf is computed whole by
one unit, its products in ascending k).

The device work goes through a backend object (the real binding by default)
so the scheduling logic can be exercised without a GPU.
"""
from __future__ import annotations

import collections
import statistics
import threading
import time
from dataclasses import dataclass, field
from typing import Any, Optional

# operand-term bytes per input leaf of the tensor forms (64 x 64 leaves)
TERM_BYTES = {"fp64": 0, "fp16_scaled": 16384, "bf16_split": 24576, "bf16_split4": 32768}
# first guesses of the work rate per millisecond (kept leaf products for FP64,
# quad steps for the tensor forms), replaced by measurements as launches run
RATE_GUESS = {"fp64": 2400.0, "fp16_scaled": 160000.0, "bf16_split": 90000.0, "bf16_split4": 53000.0}


@dataclass
class Request:
    A: Any
    B: Any
    tau: float
    mode: str = "combined"
    prec: str = "bf16_split4"
    order: str = "auto"      # claiming order of its leaf-product units (spamm_set_claim_order)
    rid: int = -1
    arrival: float = 0.0     # seconds since the server started (when it may be served)
    # filled in by the server
    state: str = "pending"   # pending, planned, running, done, cancelled, refused, failed
    plan: Any = None
    job: Any = None
    footprint: int = 0       # bytes charged to the device budget
    t_planned: float = 0.0
    t_start: float = 0.0     # first launch that ran some of its units
    t_done: float = 0.0
    launches: int = 0
    result: Any = None
    stats: dict = field(default_factory=dict)
    error: str = ""

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class SpammBackend:
    """The real device work through libspamm: plan, sliced execution, release."""

    def __init__(self, device: int = 0, exec_sms: Optional[int] = None):
        import torch

        from . import spamm as S
        self.S = S
        torch.cuda.set_device(device)
        self.plan_stream = torch.cuda.Stream(device)
        self.exec_stream = torch.cuda.Stream(device)
        self.plan_ctx = S.Context(device, stream=self.plan_stream)
        self.exec_ctx = S.Context(device, stream=self.exec_stream)
        if exec_sms:
            S.spamm_set_gemm_sms(self.exec_ctx, exec_sms)
        free, _ = torch.cuda.mem_get_info(device)
        self.free_bytes = free
        self.sms = exec_sms or torch.cuda.get_device_properties(device).multi_processor_count

    def estimate(self, req: Request) -> int:
        """Bytes to charge before planning: the operand terms and an output as
        large as both inputs."""
        ia, ib = req.A.info(), req.B.info()
        leaves = ia["nleaves"] + (0 if req.B is req.A else ib["nleaves"])
        return int(leaves * (TERM_BYTES.get(req.prec, 0) + 8 * ia["bs"] ** 2))

    def plan(self, req: Request):
        self.S.spamm_set_claim_order(self.plan_ctx, req.order)  # the planner thread is the context's only user
        p = self.S.spamm_plan_create(self.plan_ctx, req.A, req.B, req.tau, req.mode, req.prec)
        info = p.info()
        info["bs"] = req.A.info()["bs"]
        return p, int(info["plan_bytes"] + info["exec_bytes"]), info

    def begin(self, plan):
        return self.S.spamm_job_begin(self.exec_ctx, plan)

    def work(self, job):
        i = job.info()
        return i["work"], i["work_done"]

    def units(self, job):
        i = job.info()
        return i["units"], i["units_done"]

    def slots(self, prec: str, bs) -> int:
        """Work units one launch runs side by side: the FP64 kernel holds three
        CTAs per SM, the tensor-core kernel one."""
        return (3 if prec == "fp64" else 1) * self.sms

    def run(self, jobs, budgets) -> float:
        _, ms = self.S.spamm_run(self.exec_ctx, jobs, budgets)
        return ms

    def finish(self, job):
        return self.S.spamm_job_finish(self.exec_ctx, job, stats=True)

    def release_job(self, job):
        job.close()

    def release(self, plan):
        plan.close()


class Server:
    def __init__(self, backend=None, hbm_budget: Optional[int] = None, max_batch: int = 64, device: int = 0,
                 exec_sms: Optional[int] = None, slice_ms: float = 25.0, rate_guess: Optional[dict] = None,
                 keep_results: bool = True):
        self.backend = backend if backend is not None else SpammBackend(device, exec_sms)
        if hbm_budget is None:
            hbm_budget = int(0.8 * getattr(self.backend, "free_bytes", 1 << 40))
        self.budget = int(hbm_budget)
        self.max_batch = max_batch
        self.slice_ms = float(slice_ms)
        self.keep_results = keep_results  # False: a product is released once its statistics are taken
        self.in_use = 0            # bytes charged: requests being planned, planned and running
        self.peak_in_use = 0
        self.requests = {}
        self._arrivals = collections.deque()   # submitted, not yet planned (by arrival time)
        self._planned = collections.deque()    # planned, not yet handed to the executor
        self._lock = threading.Condition()
        self._next = 0
        self._stop = False
        self._t0 = None
        self._rate = {}            # (form, leaf size) -> measured work per ms
        self._rate_guess = dict(RATE_GUESS, **(rate_guess or {}))
        self.batches = []          # (jobs in the launch, ms of the launch) per launch
        self._threads = []

    # ------------------------------------------------------------ client API
    def now(self) -> float:
        return time.perf_counter() - self._t0 if self._t0 is not None else 0.0

    def submit(self, req: Request) -> int:
        with self._lock:
            req.rid = self._next
            self._next += 1
            self.requests[req.rid] = req
            self._arrivals.append(req)
            self._lock.notify_all()
        return req.rid

    def poll(self, rid: int) -> bool:
        return self.requests[rid].state in ("done", "cancelled", "refused", "failed")

    def wait(self, rid: int, timeout: Optional[float] = None) -> Request:
        end = None if timeout is None else time.perf_counter() + timeout
        with self._lock:
            while not self.poll(rid):
                left = None if end is None else end - time.perf_counter()
                if left is not None and left <= 0:
                    raise TimeoutError(f"request {rid} not done")
                self._lock.wait(left)
        return self.requests[rid]

    def cancel(self, rid: int) -> bool:
        """Cancel a request that has not been handed to the executor."""
        with self._lock:
            r = self.requests[rid]
            if r.state in ("pending", "planned"):
                if r in self._arrivals:
                    self._arrivals.remove(r)
                if r in self._planned:
                    self._planned.remove(r)
                    self.backend.release(r.plan)
                    r.plan = None
                    self._charge(-r.footprint)
                r.state = "cancelled"
                r.t_done = self.now()
                self._lock.notify_all()
                return True
            return False

    def start(self):
        self._t0 = time.perf_counter()
        self._threads = [threading.Thread(target=self._planner, daemon=True),
                         threading.Thread(target=self._executor, daemon=True)]
        for t in self._threads:
            t.start()

    def stop(self, timeout: float = 60.0):
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        for t in self._threads:
            t.join(timeout)

    # --------------------------------------------------------------- workers
    def _charge(self, nbytes: int):
        """Under the lock."""
        self.in_use += nbytes
        self.peak_in_use = max(self.peak_in_use, self.in_use)

    def _planner(self):
        while True:
            with self._lock:
                while not self._stop and not self._ready_arrival():
                    self._lock.wait(self._time_to_next_arrival())
                if self._stop:
                    return
                req = self._arrivals[0]
                est = int(self.backend.estimate(req))
                # wait for memory; a request estimated above the whole budget is
                # planned alone and uncharged, to learn whether it is to be refused
                while not self._stop and self.in_use > 0 and self.in_use + est > self.budget:
                    self._lock.wait(0.05)
                if self._stop:
                    return
                self._arrivals.popleft()
                if est > self.budget:
                    est = 0
                self._charge(est)
            try:
                plan, foot, info = self.backend.plan(req)
            except Exception as e:  # a failed request must not stop the server
                with self._lock:
                    self._charge(-est)
                    req.state, req.error, req.t_done = "failed", str(e), self.now()
                    self._lock.notify_all()
                continue
            with self._lock:
                self._charge(-est)
                if req.state == "cancelled":
                    self.backend.release(plan)
                    self._lock.notify_all()
                    continue
                req.plan, req.t_planned = plan, self.now()
                req.stats["n_kept"] = info.get("n_kept", 0)
                req.stats["bs"] = info.get("bs")
                if foot > self.budget:
                    req.state, req.error, req.t_done = "refused", "footprint exceeds the device budget", self.now()
                    self.backend.release(plan)
                    req.plan = None
                else:
                    req.footprint = foot
                    self._charge(foot)
                    req.state = "planned"
                    self._planned.append(req)
                self._lock.notify_all()

    def _ready_arrival(self) -> bool:
        return bool(self._arrivals) and self._arrivals[0].arrival <= self.now()

    def _time_to_next_arrival(self):
        if not self._arrivals:
            return None
        return max(1e-4, self._arrivals[0].arrival - self.now())

    @staticmethod
    def _key(r: Request):
        return (r.prec, r.stats.get("bs"))

    def _first_rate(self, prec: str, bs) -> float:
        """Work rate before any launch of a form and leaf size was measured:
        the given guess for "prec/bs" or "prec"; an FP64 unit (a leaf
        product) scales with bs^3, a tensor-form unit (a 128 x 128 x 64 quad
        step) does not."""
        bs = bs or 64
        if f"{prec}/{bs}" in self._rate_guess:
            return self._rate_guess[f"{prec}/{bs}"]
        base = self._rate_guess.get(prec, 2400.0)
        return base * (64.0 / bs) ** 3 if prec == "fp64" else base

    def _budgets(self, key, group, rate: float):
        """Work each job of the launch may run: its share of the slice at the
        measured rate, but at least enough units that the launch fills every
        CTA slot (a unit is one output leaf or quad and runs on one CTA: FP64
        units of long rows take tens of milliseconds, so a slice of a few of
        them would leave most of the device idle)."""
        share = max(1.0, rate * self.slice_ms / len(group))
        slots = getattr(self.backend, "slots", None)
        units = getattr(self.backend, "units", None)
        if slots is None or units is None:
            return [share] * len(group)
        per_job = -(-slots(*key) // len(group))
        out = []
        for r in group:
            total, done = self.backend.work(r.job)
            nu, nd = units(r.job)
            left = max(1, nu - nd)
            out.append(max(share, per_job * (total - done) / left))
        return out

    def _complete(self, r: Request, C, st: dict, err: Optional[str]):
        if C is not None and not self.keep_results:
            C.close()
            C = None
        with self._lock:
            self._charge(-r.footprint)
            r.result, r.t_done = C, self.now()
            r.stats.update(st or {})
            r.state, r.error = ("failed", err) if err else ("done", "")
            self._lock.notify_all()

    def _executor(self):
        active = []   # running requests, in the order they were admitted
        turn = 0
        while True:
            with self._lock:
                while not self._stop and not self._planned and not active:
                    self._lock.wait(0.05)
                if self._stop and not self._planned and not active:
                    return
                new = list(self._planned)
                self._planned.clear()
                for r in new:
                    r.state = "running"
            for r in new:
                try:
                    r.job = self.backend.begin(r.plan)
                    active.append(r)
                except Exception as e:
                    self.backend.release(r.plan)
                    r.plan = None
                    self._complete(r, None, {}, str(e))
            if not active:
                continue
            keys = []
            for r in active:
                if self._key(r) not in keys:
                    keys.append(self._key(r))
            key = keys[turn % len(keys)]
            turn += 1
            group = [r for r in active if self._key(r) == key][:self.max_batch]
            rate = self._rate.get(key, self._first_rate(*key))
            budgets = self._budgets(key, group, rate)
            before = [self.backend.work(r.job)[1] for r in group]
            t_launch = self.now()
            try:
                ms = self.backend.run([r.job for r in group], budgets)
                err = None
            except Exception as e:
                ms, err = 0.0, str(e)
            if err is not None:
                for r in group:
                    active.remove(r)
                    self.backend.release_job(r.job)
                    self.backend.release(r.plan)
                    r.job = r.plan = None
                    self._complete(r, None, {}, err)
                continue
            done_work = 0.0
            for r, w0 in zip(group, before):
                total, w1 = self.backend.work(r.job)
                done_work += w1 - w0
                if r.launches == 0:
                    r.t_start = t_launch
                r.launches += 1
            if ms > 0 and done_work > 0:
                self._rate[key] = 0.5 * rate + 0.5 * done_work / ms
            self.batches.append((len(group), ms))
            for r in group:
                total, w = self.backend.work(r.job)
                if w < total:
                    continue
                try:
                    C, st = self.backend.finish(r.job)
                    err = None
                except Exception as e:
                    C, st, err = None, {}, str(e)
                active.remove(r)
                self.backend.release_job(r.job)
                self.backend.release(r.plan)
                r.job = r.plan = None
                self._complete(r, C, st, err)

    # ----------------------------------------------------------------- report
    def summary(self) -> dict:
        done = [r for r in self.requests.values() if r.state == "done"]
        lat = sorted(r.latency for r in done)
        span = max((r.t_done for r in done), default=0.0) - min((r.arrival for r in done), default=0.0)

        def pct(p):
            if not lat:
                return None
            return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]

        flops = sum(r.stats.get("kept_flops", 0.0) for r in done)
        return {"requests": len(self.requests), "done": len(done),
                "refused": sum(r.state == "refused" for r in self.requests.values()),
                "failed": sum(r.state == "failed" for r in self.requests.values()),
                "p50_s": pct(50), "p99_s": pct(99), "mean_s": statistics.mean(lat) if lat else None,
                "span_s": span, "requests_per_s": len(done) / span if span > 0 else None,
                "kept_gflops": flops / span / 1e9 if span > 0 else None,
                "launches": len(self.batches), "mean_jobs_per_launch": statistics.mean(b for b, _ in self.batches)
                if self.batches else None, "peak_in_use_bytes": self.peak_in_use, "budget_bytes": self.budget,
                "slice_ms": self.slice_ms}
