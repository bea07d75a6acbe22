"""Scheduling logic of the serving loop, with a fake device backend (CPU)."""
import random
import threading
import time

from paper_1906_08148_gb300.serving import Request, Server


class FakeBackend:
    """Plans take 2 ms, a batch takes 5 ms + 1 ms per request; footprints are given."""

    def __init__(self, fail_on=None):
        self.server = None
        self.max_seen = 0
        self.batches = []
        self.released = []
        self.fail_on = fail_on
        self.lock = threading.Lock()

    def plan(self, req):
        time.sleep(0.002)
        return ("plan", req.rid), int(req.A), {"n_kept": 10}

    def execute(self, plans):
        with self.lock:
            self.max_seen = max(self.max_seen, self.server.in_use)
            self.batches.append(len(plans))
        if self.fail_on is not None and any(p[1] == self.fail_on for p in plans):
            raise RuntimeError("device error")
        time.sleep(0.005 + 0.001 * len(plans))
        return [("C", p[1]) for p in plans], [{"kept_flops": 1e9} for _ in plans]

    def release(self, plan):
        with self.lock:
            self.released.append(plan)


def _serve(reqs, budget, **kw):
    fb = kw.pop("backend", None) or FakeBackend()
    srv = Server(backend=fb, hbm_budget=budget, **kw)
    fb.server = srv
    srv.start()
    ids = [srv.submit(r) for r in reqs]
    for i in ids:
        srv.wait(i, timeout=30)
    srv.stop()
    return srv, fb, ids


def test_all_requests_complete_with_latency_percentiles():
    rng = random.Random(0)
    t, reqs = 0.0, []
    for _ in range(60):
        t += rng.expovariate(400.0)
        reqs.append(Request(A=100, B=None, tau=1e-6, arrival=t))
    srv, fb, ids = _serve(reqs, budget=10_000)
    s = srv.summary()
    assert s["done"] == 60 and s["failed"] == 0 and s["refused"] == 0
    assert 0 < s["p50_s"] <= s["p99_s"]
    assert s["batches"] < 60 and s["mean_batch"] > 1.0   # arrivals during a batch are batched together
    assert all(srv.requests[i].result == ("C", i) for i in ids)
    assert len(fb.released) == 60


def test_admission_never_exceeds_the_budget_and_refuses_oversized():
    reqs = [Request(A=300 + 50 * (i % 4), B=None, tau=1e-6, arrival=0.0) for i in range(30)]
    reqs.append(Request(A=5000, B=None, tau=1e-6, arrival=0.0))
    srv, fb, ids = _serve(reqs, budget=1000)
    assert fb.max_seen <= 1000
    assert srv.peak_in_use <= 1000
    assert srv.requests[ids[-1]].state == "refused"
    assert srv.summary()["done"] == 30
    assert srv.in_use == 0


def test_cancel_before_execution():
    fb = FakeBackend()
    srv = Server(backend=fb, hbm_budget=10_000)
    fb.server = srv
    r_late = Request(A=10, B=None, tau=1e-6, arrival=5.0)
    srv.start()
    rid = srv.submit(r_late)
    assert srv.cancel(rid)
    assert srv.wait(rid, timeout=5).state == "cancelled"
    srv.stop()
    assert fb.batches == []


def test_device_failure_fails_its_batch_and_server_continues():
    fb = FakeBackend(fail_on=3)
    reqs = [Request(A=10, B=None, tau=1e-6, arrival=0.01 * i) for i in range(8)]
    srv, _, ids = _serve(reqs, budget=10_000, backend=fb)
    states = [srv.requests[i].state for i in ids]
    assert states.count("failed") >= 1 and states.count("done") >= 1
    assert srv.requests[3].state == "failed"
    assert srv.in_use == 0


def test_requests_wait_for_their_arrival_time():
    reqs = [Request(A=10, B=None, tau=1e-6, arrival=0.15)]
    srv, _, ids = _serve(reqs, budget=100)
    r = srv.requests[ids[0]]
    assert r.t_planned >= 0.15 and r.latency > 0
