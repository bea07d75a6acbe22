"""Scheduling logic of the serving loop, with a fake device backend (CPU):
plans take 2 ms, a launch takes 1 ms plus 0.1 ms per unit of work it runs;
footprints (A) and work (B) are given per request."""
import random
import threading
import time

from paper_1906_08148_gb300.serving import Request, Server

SLOW = {"fp64": 50.0}  # first guess of the work rate per ms for these fake requests


class FakeBackend:
    def __init__(self, fail_on=None):
        self.server = None
        self.max_seen = 0
        self.launches = []
        self.released = []
        self.released_jobs = 0
        self.fail_on = fail_on
        self.lock = threading.Lock()

    def estimate(self, req):
        return int(req.A)

    def plan(self, req):
        time.sleep(0.002)
        return ("plan", req.rid, int(req.B or 10)), int(req.A), {"n_kept": 10, "bs": 64}

    def begin(self, plan):
        return {"rid": plan[1], "work": plan[2], "done": 0}

    def work(self, job):
        return job["work"], job["done"]

    def run(self, jobs, budgets):
        with self.lock:
            self.max_seen = max(self.max_seen, self.server.in_use)
            self.launches.append(sorted(j["rid"] for j in jobs))
        if self.fail_on is not None and any(j["rid"] == self.fail_on for j in jobs):
            raise RuntimeError("device error")
        took = 0
        for j, b in zip(jobs, budgets):
            t = min(j["work"] - j["done"], max(1, int(b)))
            j["done"] += t
            took += t
        ms = 1.0 + 0.1 * took
        time.sleep(ms / 1e3)
        return ms

    def finish(self, job):
        return ("C", job["rid"]), {"kept_flops": 1e9}

    def release_job(self, job):
        with self.lock:
            self.released_jobs += 1

    def release(self, plan):
        with self.lock:
            self.released.append(plan)


def _serve(reqs, budget, **kw):
    fb = kw.pop("backend", None) or FakeBackend()
    srv = Server(backend=fb, hbm_budget=budget, rate_guess=SLOW, **kw)
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
        reqs.append(Request(A=100, B=rng.randint(5, 40), tau=1e-6, prec="fp64", arrival=t))
    srv, fb, ids = _serve(reqs, budget=10_000)
    s = srv.summary()
    assert s["done"] == 60 and s["failed"] == 0 and s["refused"] == 0
    assert 0 < s["p50_s"] <= s["p99_s"]
    assert s["mean_jobs_per_launch"] > 1.0   # requests that arrive while others run share launches
    assert all(srv.requests[i].result == ("C", i) for i in ids)
    assert len(fb.released) == 60 and fb.released_jobs == 60
    assert srv.in_use == 0


def test_a_request_arriving_mid_way_joins_and_finishes_first():
    """A short request that arrives while a long one runs is admitted at the
    next launch boundary, shares launches with it, and completes before it."""
    long = Request(A=10, B=3000, tau=1e-6, prec="fp64", arrival=0.0)
    short = Request(A=10, B=20, tau=1e-6, prec="fp64", arrival=0.05)
    srv, fb, (il, ish) = _serve([long, short], budget=1000, slice_ms=5.0)
    L, Sh = srv.requests[il], srv.requests[ish]
    assert L.state == Sh.state == "done"
    assert Sh.t_start < L.t_done and Sh.t_done < L.t_done
    assert L.launches > 3
    assert any(launch == [il, ish] for launch in fb.launches)  # one launch ran units of both


def test_charged_memory_never_exceeds_the_budget_and_oversized_is_refused():
    reqs = [Request(A=300 + 50 * (i % 4), B=15, tau=1e-6, prec="fp64", arrival=0.0) for i in range(30)]
    reqs.append(Request(A=5000, B=15, tau=1e-6, prec="fp64", arrival=0.0))
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
    assert fb.launches == []
    assert srv.in_use == 0


def test_device_failure_fails_its_launch_and_server_continues():
    fb = FakeBackend(fail_on=3)
    reqs = [Request(A=10, B=10, tau=1e-6, prec="fp64", arrival=0.01 * i) for i in range(8)]
    srv, _, ids = _serve(reqs, budget=10_000, backend=fb)
    states = [srv.requests[i].state for i in ids]
    assert states.count("failed") >= 1 and states.count("done") >= 1
    assert srv.requests[3].state == "failed"
    assert srv.in_use == 0


def test_forms_take_turns():
    """Two forms: launches alternate, so a request of the second form does not
    wait for the first form's long request."""
    long = Request(A=10, B=3000, tau=1e-6, prec="fp64", arrival=0.0)
    other = Request(A=10, B=20, tau=1e-6, prec="fp16_scaled", arrival=0.05)
    srv, fb, (il, io) = _serve([long, other], budget=1000, slice_ms=5.0)
    assert srv.requests[io].t_done < srv.requests[il].t_done


def test_requests_wait_for_their_arrival_time():
    reqs = [Request(A=10, B=None, tau=1e-6, arrival=0.15)]
    srv, _, ids = _serve(reqs, budget=100)
    r = srv.requests[ids[0]]
    assert r.t_planned >= 0.15 and r.latency > 0


def test_results_released_on_completion_when_not_kept():
    closed = []

    class Result:
        def __init__(self, rid):
            self.rid = rid

        def close(self):
            closed.append(self.rid)

    class Releasing(FakeBackend):
        def finish(self, job):
            return Result(job["rid"]), {"kept_flops": 1e9}

    reqs = [Request(A=100, B=20, tau=1e-6, prec="fp64", arrival=0.0) for _ in range(6)]
    srv, fb, ids = _serve(reqs, 10_000, backend=Releasing(), keep_results=False)
    assert sorted(closed) == sorted(ids)
    assert all(srv.requests[i].state == "done" and srv.requests[i].result is None for i in ids)
    assert srv.summary()["done"] == 6


def test_launch_budgets_fill_every_slot():
    """With long units (fake FP64 rows of 100 work each) and a small rate, a
    launch still covers enough units to occupy every CTA slot."""
    class Slotted(FakeBackend):
        def __init__(self):
            super().__init__()
            self.budgets = []

        def plan(self, req):
            return ("plan", req.rid, 2000), int(req.A), {"n_kept": 10, "bs": 64}

        def begin(self, plan):
            return {"rid": plan[1], "work": plan[2], "done": 0, "units": 20}

        def units(self, job):
            return job["units"], job["done"] * job["units"] // job["work"]

        def slots(self, prec, bs):
            return 8

        def run(self, jobs, budgets):
            self.budgets.append(list(budgets))
            return super().run(jobs, budgets)

    fb = Slotted()
    reqs = [Request(A=100, B=None, tau=1e-6, prec="fp64", arrival=0.0) for _ in range(2)]
    srv, fb, ids = _serve(reqs, 10_000, backend=fb)
    assert all(srv.requests[i].state == "done" for i in ids)
    # 8 slots over the launch's jobs: each job's budget covers >= 4 of its 100-work units
    first = fb.budgets[0]
    assert all(b >= 4 * 100 for b in first)
