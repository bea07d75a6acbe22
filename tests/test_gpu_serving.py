"""Continuous batching on the GPU: requests of different sizes, tau and
precision forms arrive while others execute; every served result equals the
same multiplication run alone (bit for bit)."""
import random

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm
    return spamm


def test_served_results_equal_alone(S):
    from paper_1906_08148_gb300.serving import Request, Server
    data = S.Context(0)
    rng = random.Random(7)
    pool = []
    for n, alpha in ((4096, 0.9), (8192, 1.0), (2048, 0.7), (16384, 1.1)):
        A = S.spamm_generate(data, synth.lattice_3d(n, alpha=alpha, seed=1), 64)
        B = S.spamm_generate(data, synth.lattice_3d(n, alpha=alpha, seed=2), 64)
        pool.append((A, B))
    reqs, t = [], 0.0
    for i in range(24):
        t += rng.expovariate(200.0)
        A, B = pool[rng.randrange(len(pool))]
        reqs.append(Request(A, B, tau=rng.choice([1e-4, 1e-6, 1e-8]), mode=rng.choice(["combined", "spamm"]),
                            prec=rng.choice(["bf16_split", "bf16_split4", "fp16_scaled", "fp64"]), arrival=t))
    srv = Server(max_batch=8, exec_sms=136, slice_ms=10.0)
    srv.start()
    ids = [srv.submit(r) for r in reqs]
    for i in ids:
        srv.wait(i, timeout=300)
    srv.stop()
    s = srv.summary()
    assert s["done"] == len(reqs), [(r.state, r.error) for r in srv.requests.values()]
    assert s["p50_s"] is not None and s["p99_s"] >= s["p50_s"]
    assert s["peak_in_use_bytes"] <= s["budget_bytes"]
    for i in ids:
        r = srv.requests[i]
        alone = S.spamm_multiply(data, r.A, r.B, r.tau, r.mode, r.prec)
        a = S.spamm_to_blocks(data, alone)
        b = S.spamm_to_blocks(data, r.result)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), (r.rid, r.prec, r.tau)
    print("serving summary", s)


def test_request_arriving_during_a_long_fp64_request_finishes_first(S):
    """Continuous batching: a long FP64 request (n = 16384, tau = 1e-8) starts
    alone; a short one (n = 4096) arrives while it runs, joins its next
    launches and completes before it.  Both outputs equal the same
    multiplications run alone, bit for bit."""
    from paper_1906_08148_gb300.serving import Request, Server
    data = S.Context(0)
    A = S.spamm_generate(data, synth.lattice_3d(16384, alpha=0.9, seed=1), 64)
    B = S.spamm_generate(data, synth.lattice_3d(16384, alpha=0.9, seed=2), 64)
    a = S.spamm_generate(data, synth.lattice_3d(4096, alpha=0.9, seed=3), 64)
    b = S.spamm_generate(data, synth.lattice_3d(4096, alpha=0.9, seed=4), 64)
    long = Request(A, B, tau=1e-8, mode="combined", prec="fp64", arrival=0.0)
    short = Request(a, b, tau=1e-6, mode="combined", prec="fp64", arrival=0.3)
    other = Request(a, b, tau=1e-6, mode="spamm", prec="fp16_scaled", arrival=0.4)
    srv = Server(exec_sms=136, slice_ms=20.0)
    srv.start()
    ids = [srv.submit(r) for r in (long, short, other)]
    for i in ids:
        srv.wait(i, timeout=600)
    srv.stop()
    L, Sh, O = (srv.requests[i] for i in ids)
    assert L.state == Sh.state == O.state == "done", [(r.state, r.error) for r in (L, Sh, O)]
    print(f"long: {L.launches} launches, done at {L.t_done:.2f} s; short: started {Sh.t_start:.2f} s, "
          f"done {Sh.t_done:.2f} s; fp16: done {O.t_done:.2f} s")
    assert Sh.t_start < L.t_done and Sh.t_done < L.t_done and O.t_done < L.t_done
    assert L.launches > 5
    for r in (L, Sh, O):
        alone = S.spamm_multiply(data, r.A, r.B, r.tau, r.mode, r.prec)
        x, y = S.spamm_to_blocks(data, alone), S.spamm_to_blocks(data, r.result)
        for u, v in zip(x, y):
            assert np.array_equal(u, v)
