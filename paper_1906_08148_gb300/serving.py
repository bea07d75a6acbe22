"""Continuous-batching request loop over the C ABI.

Requests (A, B, tau, mode, precision) arrive at any time and are served by
two host threads, each with its own libspamm context and CUDA stream:

* the planner takes arrived requests in order and creates their plans
  (truncation, quadtree descent, operand terms: spamm_plan_create);
* the executor admits planned requests while their device-memory footprint
  (plan + output, from spamm_plan_info) fits the budget, and runs every
  admitted request's leaf products in ONE persistent launch (spamm_execute);
  it then releases their plans and completes them.

While a batch executes, the planner keeps planning new arrivals on its own
stream; the executor's launch is kept off a few SMs (spamm_set_gemm_sms) so
those kernels can run beside it.  A request larger than the whole budget is
refused, not crashed.  Each output is bit-identical to multiplying the same
request alone (one owner per output leaf, fixed k order).

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


@dataclass
class Request:
    A: Any
    B: Any
    tau: float
    mode: str = "combined"
    prec: str = "bf16_split"
    rid: int = -1
    arrival: float = 0.0     # seconds since the server started (when it may be served)
    # filled in by the server
    state: str = "pending"   # pending, planned, running, done, cancelled, refused, failed
    plan: Any = None
    footprint: int = 0
    t_planned: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    result: Any = None
    stats: dict = field(default_factory=dict)
    error: str = ""

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class SpammBackend:
    """The real device work: plan / execute / release through libspamm."""

    def __init__(self, device: int = 0, exec_sms: Optional[int] = None, graph: bool = False):
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
        if graph:  # each batch's execute phase as one captured CUDA graph
            S.spamm_set_exec_graph(self.exec_ctx, True)
        free, _ = torch.cuda.mem_get_info(device)
        self.free_bytes = free

    def plan(self, req: Request):
        p = self.S.spamm_plan_create(self.plan_ctx, req.A, req.B, req.tau, req.mode, req.prec)
        info = p.info()
        info["bs"] = req.A.info()["bs"]
        return p, int(info["plan_bytes"] + info["exec_bytes"]), info

    def execute(self, plans):
        Cs, st = self.S.spamm_execute(self.exec_ctx, plans, stats=True)
        return Cs, st

    def release(self, plan):
        plan.close()


class Server:
    def __init__(self, backend=None, hbm_budget: Optional[int] = None, max_batch: int = 64, device: int = 0,
                 exec_sms: Optional[int] = None, graph: bool = False):
        self.backend = backend if backend is not None else SpammBackend(device, exec_sms, graph)
        if hbm_budget is None:
            hbm_budget = int(0.8 * getattr(self.backend, "free_bytes", 1 << 40))
        self.budget = int(hbm_budget)
        self.max_batch = max_batch
        self.in_use = 0            # bytes of admitted, unfinished requests
        self.peak_in_use = 0
        self.requests = {}
        self._arrivals = collections.deque()   # submitted, not yet planned (by arrival time)
        self._planned = collections.deque()    # planned, waiting for admission
        self._lock = threading.Condition()
        self._next = 0
        self._stop = False
        self._t0 = None
        self.batches = []          # (number of requests, ms of the launch) per executed batch
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
        """Cancel a request that has not started executing."""
        with self._lock:
            r = self.requests[rid]
            if r.state in ("pending", "planned"):
                if r in self._arrivals:
                    self._arrivals.remove(r)
                if r in self._planned:
                    self._planned.remove(r)
                    self.backend.release(r.plan)
                    r.plan = None
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
    def _planner(self):
        while True:
            with self._lock:
                while not self._stop and not self._ready_arrival():
                    self._lock.wait(self._time_to_next_arrival())
                if self._stop:
                    return
                req = self._arrivals.popleft()
            try:
                plan, foot, info = self.backend.plan(req)
            except Exception as e:  # a failed request must not stop the server
                with self._lock:
                    req.state, req.error, req.t_done = "failed", str(e), self.now()
                    self._lock.notify_all()
                continue
            with self._lock:
                if req.state == "cancelled":
                    self.backend.release(plan)
                    continue
                req.plan, req.footprint, req.t_planned = plan, foot, self.now()
                req.stats["n_kept"] = info.get("n_kept", 0)
                req.stats["bs"] = info.get("bs")
                if foot > self.budget:
                    req.state, req.error, req.t_done = "refused", "footprint exceeds the device budget", self.now()
                    self.backend.release(plan)
                    req.plan = None
                else:
                    req.state = "planned"
                    self._planned.append(req)
                self._lock.notify_all()

    def _ready_arrival(self) -> bool:
        return bool(self._arrivals) and self._arrivals[0].arrival <= self.now()

    def _time_to_next_arrival(self):
        if not self._arrivals:
            return None
        return max(1e-4, self._arrivals[0].arrival - self.now())

    def _admit(self):
        """Planned requests of the oldest one's kind (precision form, leaf size),
        in order, while their footprint fits the budget."""
        batch = []
        key = None
        for r in list(self._planned):
            if len(batch) >= self.max_batch:
                break
            k = (r.prec, r.stats.get("bs"))
            if key is None:
                key = k
            elif k != key:
                continue
            if self.in_use + r.footprint > self.budget and (batch or self.in_use > 0):
                break
            self._planned.remove(r)
            self.in_use += r.footprint
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            r.state, r.t_start = "running", self.now()
            batch.append(r)
        return batch

    def _executor(self):
        while True:
            with self._lock:
                while not self._stop and not self._planned:
                    self._lock.wait(0.05)
                if self._stop and not self._planned:
                    return
                batch = self._admit()
            if not batch:
                continue
            t0 = time.perf_counter()
            try:
                outs, stats = self.backend.execute([r.plan for r in batch])
                err = None
            except Exception as e:
                outs, stats, err = [None] * len(batch), [{}] * len(batch), str(e)
            ms = 1e3 * (time.perf_counter() - t0)
            for r in batch:
                self.backend.release(r.plan)
                r.plan = None
            with self._lock:
                self.batches.append((len(batch), ms))
                for r, C, st in zip(batch, outs, stats):
                    self.in_use -= r.footprint
                    r.result, r.t_done = C, self.now()
                    r.stats.update(st)
                    r.state, r.error = ("failed", err) if err else ("done", "")
                self._lock.notify_all()

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
                "batches": len(self.batches), "mean_batch": statistics.mean(b for b, _ in self.batches)
                if self.batches else None, "peak_in_use_bytes": self.peak_in_use, "budget_bytes": self.budget}
