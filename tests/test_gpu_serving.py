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


@pytest.mark.parametrize("graph", [False, True])
def test_served_results_equal_alone(S, graph):
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
                            prec=rng.choice(["bf16_split", "fp16_scaled", "fp64"]), arrival=t))
    srv = Server(max_batch=8, exec_sms=136, graph=graph)
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
    print("serving summary", "graph" if graph else "eager", s)
