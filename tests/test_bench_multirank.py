"""The N > 1 path of bench.py (independent replicas, one per GPU) on CPU with
gloo, world size 2: the timed region is the slowest rank's and the value is
all ranks' work over it; the reference arm prints only on rank 0."""
import json
import os
import socket
import subprocess
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 * (rank + 1)          # rank 1 is the slower one
    flops = 1e12 * (rank + 1)
    kept = 1000 * (rank + 1)
    res = bench.aggregate_ranks(ms, flops, kept, dist)
    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms, gflops, mults = got[r]
        assert ms == 200.0
        assert abs(gflops - 3e12 / 0.2 / 1e9) < 1e-6
        assert abs(mults - 3000 / 0.2) < 1e-6


def test_single_rank_aggregate_is_local():
    sys.path.insert(0, ROOT)
    import bench
    ms, gflops, mults = bench.aggregate_ranks(50.0, 5e11, 100)
    assert ms == 50.0 and abs(gflops - 1e4) < 1e-9 and abs(mults - 2000.0) < 1e-9


def test_reference_arm_under_torchrun_prints_on_rank0_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--config", "model2048", "--mode", "spamm", "--tau", "1e-8",
           "--steps", "1", "--warmup", "1", "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
