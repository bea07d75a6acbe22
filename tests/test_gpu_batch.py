"""Two-phase, batched multiplication: plans of different sizes, tau and methods
run in one persistent launch; every output is bit-identical to the same
plan executed alone and matches the oracle."""
import numpy as np
import pytest

import oracle
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


@pytest.fixture(scope="module")
def ctx(S):
    return S.Context(0)


REQUESTS = [(4096, 0.9, 1e-6, "combined"), (2048, 0.7, 1e-4, "spamm"), (8192, 1.1, 1e-8, "truncate"),
            (1000, 0.8, 1e-5, "combined"), (4096, 0.6, 1e-6, "spamm")]


def _inputs(S, ctx, n, alpha, bs):
    GA = S.spamm_generate(ctx, synth.lattice_3d(n, alpha=alpha, seed=1), bs)
    GB = S.spamm_generate(ctx, synth.lattice_3d(n, alpha=alpha, seed=2), bs)
    return GA, GB


@pytest.mark.parametrize("prec,bs", [("fp64", 64), ("fp64", 32), ("bf16_split", 64), ("fp16_scaled", 64)])
def test_batch_equals_alone_bitwise(S, ctx, prec, bs):
    plans, alone, inputs = [], [], []
    for n, alpha, tau, mode in REQUESTS:
        GA, GB = _inputs(S, ctx, n, alpha, bs)
        inputs.append((GA, GB))
        p = S.spamm_plan_create(ctx, GA, GB, tau, mode, prec)
        plans.append(p)
        alone.append(S.spamm_to_blocks(ctx, S.spamm_execute(ctx, [p])[0]))
    Cs, st = S.spamm_execute(ctx, plans, stats=True)
    for r, C in enumerate(Cs):
        got = S.spamm_to_blocks(ctx, C)
        for a, b in zip(alone[r], got):
            assert np.array_equal(a, b), (prec, r)
        assert st[r]["n_kept"] == plans[r].info()["n_kept"]
    # the plans are reusable and independent of their inputs' handles
    for GA, GB in inputs:
        GA.close()
        GB.close()
    again = S.spamm_execute(ctx, plans[::-1])[::-1]
    for r, C in enumerate(again):
        assert np.array_equal(S.spamm_to_blocks(ctx, C)[2], alone[r][2])


def test_batch_matches_oracle_fp64(S, ctx):
    plans, refs = [], []
    for n, alpha, tau, mode in REQUESTS[:3]:
        pa, pb = synth.lattice_3d(n, alpha=alpha, seed=1), synth.lattice_3d(n, alpha=alpha, seed=2)
        GA, GB = S.spamm_generate(ctx, pa, 64), S.spamm_generate(ctx, pb, 64)
        plans.append(S.spamm_plan_create(ctx, GA, GB, tau, mode, "fp64"))
        ref, _ = oracle.multiply(oracle.from_dense(synth.dense(pa), 64), oracle.from_dense(synth.dense(pb), 64),
                                 tau, oracle.MODES[mode])
        refs.append(ref)
    for C, ref in zip(S.spamm_execute(ctx, plans), refs):
        D = S.spamm_to_dense(ctx, C)
        R = oracle.to_dense(ref)
        assert np.linalg.norm(D - R) <= 1e-12 * np.linalg.norm(R)


def test_batch_rejects_mixed_forms_and_reports_footprint(S, ctx):
    GA, GB = _inputs(S, ctx, 2048, 0.8, 64)
    p1 = S.spamm_plan_create(ctx, GA, GB, 1e-6, "spamm", "fp64")
    p2 = S.spamm_plan_create(ctx, GA, GB, 1e-6, "spamm", "bf16_split")
    with pytest.raises(S.SpammError) as e:
        S.spamm_execute(ctx, [p1, p2])
    assert e.value.status == S.E_INVALID_ARG
    info = p2.info()
    assert info["plan_bytes"] > 0 and info["exec_bytes"] >= info["n_c_leaves"] * 64 * 64 * 8
    C, st = S.spamm_multiply(ctx, GA, GB, 1e-6, "spamm", "bf16_split", stats=True)
    assert st["n_kept"] == info["n_kept"] and st["ms_prep"] > 0


def test_gemm_sm_limit_keeps_results(S, ctx):
    GA, GB = _inputs(S, ctx, 4096, 0.8, 64)
    ref = S.spamm_to_blocks(ctx, S.spamm_multiply(ctx, GA, GB, 1e-6, "combined", "bf16_split"))
    S.spamm_set_gemm_sms(ctx, 16)
    try:
        got = S.spamm_to_blocks(ctx, S.spamm_multiply(ctx, GA, GB, 1e-6, "combined", "bf16_split"))
    finally:
        S.spamm_set_gemm_sms(ctx, 0)
    assert np.array_equal(ref[2], got[2])


@pytest.mark.parametrize("prec", ["fp64", "bf16_split", "bf16_split4", "fp16_scaled"])
def test_graph_execute_equals_eager(S, ctx, prec):
    """The execute phase captured as one CUDA graph gives the same leaves and
    the same norms at every quadtree level as the eager launch sequence."""
    plans, keep = [], []
    for n, alpha, tau, mode in REQUESTS:
        GA, GB = _inputs(S, ctx, n, alpha, 64)
        keep.append((GA, GB))
        plans.append(S.spamm_plan_create(ctx, GA, GB, tau, mode, prec))
    eager, st_e = S.spamm_execute(ctx, plans, stats=True)
    S.spamm_set_exec_graph(ctx, True)
    try:
        g0 = S.spamm_exec_graph_info(ctx)
        graph, st_g = S.spamm_execute(ctx, plans, stats=True)
        # same batch again: the kept executable graph is updated in place (the
        # driver may still refuse an update and the graph is then rebuilt)
        again, _ = S.spamm_execute(ctx, plans, stats=True)
        for _ in range(3):
            for m in S.spamm_execute(ctx, plans):
                m.close()
        g1 = S.spamm_exec_graph_info(ctx)
        single = S.spamm_multiply(ctx, keep[0][0], keep[0][1], REQUESTS[0][2], REQUESTS[0][3], prec)
    finally:
        S.spamm_set_exec_graph(ctx, False)
    runs = (g1["updates"] - g0["updates"]) + (g1["instantiations"] - g0["instantiations"])
    assert runs == 5  # every execute ran as the graph
    assert g1["updates"] >= g0["updates"] + 1, S.load().spamm_last_error(ctx.handle)
    for G, A in zip(graph, again):
        assert np.array_equal(S.spamm_to_blocks(ctx, G)[2], S.spamm_to_blocks(ctx, A)[2])
    for r, (E, G) in enumerate(zip(eager, graph)):
        for a, b in zip(S.spamm_to_blocks(ctx, E), S.spamm_to_blocks(ctx, G)):
            assert np.array_equal(a, b), (prec, r)
        L = E.info()["levels"]
        for lev in range(L + 1):
            ce, se = S.spamm_level_norms(ctx, E, lev)
            cg, sg = S.spamm_level_norms(ctx, G, lev)
            assert np.array_equal(ce, cg) and np.array_equal(se, sg), (prec, r, lev)
        assert st_g[r]["ms_gemm"] > 0.0
    assert np.array_equal(S.spamm_to_blocks(ctx, single)[2], S.spamm_to_blocks(ctx, eager[0])[2])


def test_device_timeout_becomes_a_status_and_the_context_stays_usable(S, ctx):
    """A bounded device wait that runs out (an mbarrier phase nothing
    completes, 50 ms bound) is reported as SPAMM_E_TIMEOUT; the error word is
    cleared, so the next multiply on the same context succeeds and is exact."""
    import time
    t0 = time.perf_counter()
    st = S.spamm_check_timeout_path(ctx, 50_000_000)
    took = time.perf_counter() - t0
    assert st == S.E_TIMEOUT
    assert 0.04 <= took < 5.0
    assert "ran out" in S.load().spamm_last_error(ctx.handle).decode()
    assert S.spamm_check_timeout_path(ctx, 0) == S.E_INVALID_ARG
    GA, GB = _inputs(S, ctx, 2048, 0.8, 64)
    C = S.spamm_multiply(ctx, GA, GB, 1e-6, "combined", "fp64")
    D = S.spamm_multiply(ctx, GA, GB, 1e-6, "combined", "fp64")
    assert np.array_equal(S.spamm_to_blocks(ctx, C)[2], S.spamm_to_blocks(ctx, D)[2])


def test_trim_returns_cached_pool_memory(S, ctx):
    import torch
    GA, GB = _inputs(S, ctx, 8192, 0.8, 64)
    C = S.spamm_multiply(ctx, GA, GB, 1e-6, "combined")
    ref = S.spamm_to_dense(ctx, C)
    big = S.spamm_multiply(ctx, GA, GB, 0.0, "spamm")  # a larger output, freed below: cached by the pool
    big.close()
    S.spamm_sync(ctx)
    before = torch.cuda.mem_get_info()[0]
    S.spamm_trim(ctx)
    after = torch.cuda.mem_get_info()[0]
    assert after >= before
    # live handles are untouched
    assert np.array_equal(S.spamm_to_dense(ctx, C), ref)
    assert S.spamm_frob_norm(ctx, C) > 0


@pytest.mark.parametrize("bs", [128, 256])
def test_graph_and_batch_with_subtile_units(S, ctx, bs):
    """128 and 256 leaves run as 64 x 64 sub-tile units whose partial norms a
    second launch adds: eager, graph and alone give the same leaves and norms."""
    plans, keep = [], []
    for n, alpha, tau, mode in [(4096, 0.9, 1e-6, "combined"), (2048, 0.7, 1e-4, "spamm"), (1000, 0.8, 1e-5, "truncate")]:
        GA, GB = _inputs(S, ctx, n, alpha, bs)
        keep.append((GA, GB, tau, mode))
        plans.append(S.spamm_plan_create(ctx, GA, GB, tau, mode, "fp64"))
    eager = S.spamm_execute(ctx, plans)
    S.spamm_set_exec_graph(ctx, True)
    try:
        graph = S.spamm_execute(ctx, plans)
    finally:
        S.spamm_set_exec_graph(ctx, False)
    for (GA, GB, tau, mode), E, G in zip(keep, eager, graph):
        alone = S.spamm_multiply(ctx, GA, GB, tau, mode, "fp64")
        for X in (G, alone):
            for a, b in zip(S.spamm_to_blocks(ctx, E), S.spamm_to_blocks(ctx, X)):
                assert np.array_equal(a, b)
        for lev in range(E.info()["levels"] + 1):
            ce, se = S.spamm_level_norms(ctx, E, lev)
            cg, sg = S.spamm_level_norms(ctx, G, lev)
            assert np.array_equal(ce, cg) and np.array_equal(se, sg)
        # the leaf norms are the norms of the leaves
        bi, bj, pay, sq = S.spamm_to_blocks(ctx, E)
        assert np.allclose(sq, np.sum(pay ** 2, axis=(1, 2)), rtol=1e-13, atol=0)


@pytest.mark.parametrize("prec,bs", [("fp64", 64), ("fp64", 32), ("fp64", 128), ("fp64", 256), ("bf16_split", 64),
                                     ("bf16_split4", 64), ("fp16_scaled", 64), ("bf16_split4", 128),
                                     ("fp16_scaled", 128)])
def test_sliced_jobs_equal_one_execute_bitwise(S, ctx, prec, bs):
    """Sliced execution (spamm_job_begin / spamm_run / spamm_job_finish):
    several jobs run their units in many small launches, a job joining
    while others are half done; every output is bit-identical (leaves,
    norms, quadtree) to executing its plan in one launch."""
    reqs = [(4096, 0.9, 1e-6, "combined"), (2048, 0.7, 1e-4, "spamm"), (4096, 0.6, 1e-8, "combined")]
    plans = []
    for n, alpha, tau, mode in reqs:
        GA, GB = _inputs(S, ctx, n, alpha, bs)
        plans.append(S.spamm_plan_create(ctx, GA, GB, tau, mode, prec))
    ref = [S.spamm_execute(ctx, [p])[0] for p in plans]
    jobs = [S.spamm_job_begin(ctx, plans[0]), S.spamm_job_begin(ctx, plans[1])]
    launches = 0
    while any(j.info()["units_done"] < j.info()["units"] for j in jobs) or len(jobs) < len(plans):
        ran, ms = S.spamm_run(ctx, jobs, [j.info()["work"] / 7.0 + 1.0 for j in jobs])
        launches += 1
        if launches == 2:
            jobs.append(S.spamm_job_begin(ctx, plans[2]))  # joins while the first two are under way
        assert launches < 100
    assert launches >= 4
    for j, C0, p in zip(jobs, ref, plans):
        C, st = S.spamm_job_finish(ctx, j, stats=True)
        assert st["n_kept"] == p.info()["n_kept"] and st["n_launches"] >= 2
        a, b = S.spamm_to_blocks(ctx, C0), S.spamm_to_blocks(ctx, C)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        L = C.info()["levels"]
        for t in range(L + 1):
            assert np.array_equal(S.spamm_level_norms(ctx, C0, t)[1], S.spamm_level_norms(ctx, C, t)[1])
        j.close()
    # a job with units left cannot be finished
    j = S.spamm_job_begin(ctx, plans[0])
    S.spamm_run(ctx, [j], [1.0])
    with pytest.raises(S.SpammError) as err:
        S.spamm_job_finish(ctx, j)
    assert err.value.status == S.E_BUSY
    j.close()


@pytest.mark.parametrize("prec,bs", [("fp64", 64), ("fp64", 128), ("fp16_scaled", 64), ("bf16_split4", 64),
                                     ("bf16_split4", 128)])
def test_claim_order_keeps_results_bitwise(S, ctx, prec, bs):
    """The tile schedule (spamm_set_claim_order) changes only the order in which
    CTAs claim work units: every order gives the same bits, in one launch and
    in sliced execution."""
    GA, GB = _inputs(S, ctx, 4096, 0.8, bs)
    outs = {}
    try:
        for order in ("morton", "longest", "auto"):
            S.spamm_set_claim_order(ctx, order)
            p = S.spamm_plan_create(ctx, GA, GB, 1e-7, "combined", prec)
            C = S.spamm_execute(ctx, [p])[0]
            outs[order] = S.spamm_to_blocks(ctx, C)
            j = S.spamm_job_begin(ctx, p)
            while j.info()["units_done"] < j.info()["units"]:
                S.spamm_run(ctx, [j], [j.info()["work"] / 5.0 + 1.0])
            Cj = S.spamm_job_finish(ctx, j)
            for x, y in zip(outs[order], S.spamm_to_blocks(ctx, Cj)):
                assert np.array_equal(x, y)
            j.close()
    finally:
        S.spamm_set_claim_order(ctx, "auto")
    for order in ("longest", "auto"):
        for x, y in zip(outs["morton"], outs[order]):
            assert np.array_equal(x, y)
    assert S.load().spamm_set_claim_order(ctx.handle, 7) == S.E_INVALID_ARG
