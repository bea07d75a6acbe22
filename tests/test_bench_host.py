"""Host logic of bench.py (no GPU): the roofline entry, the traffic lookup
keyed by kernel source hash, the clock-record summary and the choice of tau
at equal accuracy."""
import json
import os

import pytest

import bench


def test_fp64_roofline_is_kept_flops_over_event_time():
    kept, ms = 1000, 1.0
    r = bench.roofline("fp64", 64, kept, ms, 0.0)
    assert r["bound"] == "alu" and r["unit"] == "GFLOP/s"
    assert r["achieved"] == pytest.approx(2 * 64 ** 3 * kept / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_GFLOPS)
    entry = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["gemm_fp64_kernel<64>"]
    assert r["traffic"] == pytest.approx(entry["dram_bytes_per_product"] * kept)  # capture of the current source


def test_tensor_roofline_reports_kept_and_executed_rates():
    r = bench.roofline("fp16_scaled", 64, 2000, 2.0, 3.0e12)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(2 * 64 ** 3 * 2000 / 2e-3 / 1e12)
    assert r["executed"] == pytest.approx(3.0e12 / 2e-3 / 1e12)
    assert r["executed_frac"] == pytest.approx(r["executed"] / r["peak"])


def test_traffic_is_null_once_the_kernel_source_changed(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("kernel v1\n")
    import hashlib
    h = hashlib.sha256(b"kernel v1\n").hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"k": {"source": "k.cu", "source_sha256_16": h, "dram_bytes_per_product": 100.0}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("k", 10) == 1000.0
    assert bench.load_traffic("other", 10) is None
    (tmp_path / "k.cu").write_text("kernel v2\n")
    assert bench.load_traffic("k", 10) is None


def test_clock_summary_median_under_load_and_reasons(tmp_path):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 345, 2070, 150.0, 0x1, Not Active, Not Active, Not Active, Not Active",  # idle sample
            "0, 1995, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
            "garbage line"]
    open(c.path, "w").write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4
    assert not os.path.exists(c.path)


class _FakeMat:
    def close(self):
        pass


class _FakeS:
    """tau_sweep's calls with a made-up error and product count per (mode, tau)."""
    ERR = {"truncate": {1e-4: 3e-2, 1e-6: 3e-4, 1e-8: 3e-6},
           "spamm": {1e-4: 1e-2, 1e-6: 1e-4, 1e-8: 1e-6},
           "combined": {1e-4: 2e-2, 1e-6: 2e-4, 1e-8: 2e-6}}
    KEPT = {"truncate": 10, "spamm": 4, "combined": 5}

    def __init__(self):
        self.last = None

    def spamm_multiply(self, ctx, A, B, tau, mode, prec="fp64", stats=False):
        self.last = (mode, tau)
        m = _FakeMat()
        if not stats:
            return m
        k = self.KEPT[mode] * (1 if tau > 0 else 10)
        return m, {"n_kept": k, "ms_gemm": 1.0, "kept_flops": 2.0 * 64 ** 3 * k}

    def spamm_error(self, ctx, X, C):
        mode, tau = self.last
        return self.ERR[mode][tau]

    def spamm_frob_norm(self, ctx, X):
        return 1.0


def test_tau_sweep_takes_the_largest_tau_within_each_sigma():
    out = bench.tau_sweep(_FakeS(), None, None, None, [1e-4, 1e-6, 1e-8], [1e-2, 1e-4, 1e-6])
    ch = out["chosen"]
    assert ch["0.01"]["spamm"]["tau"] == 1e-4 and ch["0.01"]["truncate"]["tau"] == 1e-6
    assert ch["0.0001"]["spamm"]["tau"] == 1e-6 and ch["0.0001"]["combined"]["tau"] == 1e-8
    assert ch["1e-06"]["truncate"] is None and ch["1e-06"]["spamm"]["tau"] == 1e-8
    assert ch["0.01"]["spamm"]["gemm_vs_truncmul"] == pytest.approx(4 / 10)
    assert out["exact"]["n_kept"] == 40


@pytest.mark.parametrize("argv", [[], ["--steps", "5", "--warmup", "3"], ["--gpus", "2"], ["--impl", "reference"],
                                  ["--sweep"], ["--model-problem", "--mp-bs", "32", "256"], ["--block-sparse"],
                                  ["--passes"], ["--chain"], ["--sp2"], ["--serve", "--prec", "auto"],
                                  ["--prec", "fp16_scaled", "--config", "lattice16384"]])
def test_every_mode_parses(monkeypatch, argv):
    monkeypatch.setattr("sys.argv", ["bench.py"] + argv)
    a = bench.parse_args()
    assert a.steps >= 1


def test_defaults_are_one_gpu_the_bench_workload_and_three_warmups(monkeypatch):
    monkeypatch.setattr("sys.argv", ["bench.py"])
    a = bench.parse_args()
    assert a.gpus == 1 and a.warmup >= 3 and a.config == "lattice65536"
    assert a.impl != "reference"
    # no form and no tau given: the equal-accuracy headline, tau from the committed oracle table
    bench.resolve_defaults(a)
    assert a.headline and a.prec is None and a.tau == bench.tau_for_sigma("lattice65536", "combined", a.sigma)
    # an explicit tau or form: a plain line, FP64 unless named
    monkeypatch.setattr("sys.argv", ["bench.py", "--tau", "1e-6"])
    b = bench.parse_args()
    bench.resolve_defaults(b)
    assert not b.headline and b.prec == "fp64" and b.tau == 1e-6


def test_sp2_footprint_estimate_admits_the_64_cubed_lattice_and_refuses_two_to_the_20():
    import synth
    est = {n: bench.sp2_estimate(synth.lattice_3d(n, alpha=1.0, seed=1), 64, 6.0, 1e-6, held=1)
           for n in (262144, 1048576)}
    gb300 = 284_208 * 2 ** 20
    assert est[262144]["peak_bytes_est"] < 0.9 * 0.95 * gb300
    assert est[1048576]["peak_bytes_est"] > gb300
    # leaves per block row are about the same for both lattices (the decay sets them)
    per_row = {n: e["x0_leaves_est"] / (n // 64) for n, e in est.items()}
    assert 0.8 < per_row[262144] / per_row[1048576] < 1.25


def test_end_to_end_leg_counts_copied_bytes_and_the_held_block(monkeypatch):
    """run_e2e against a stand-in library and host allocator: the timed steps
    (one untimed sizing pass first), the host-to-device bytes of both inputs'
    leaves and coordinates, the device-to-host bytes of every C leaf with its
    coordinates and norm, and the held pinned block reported when the host
    has room for it (none when it has not)."""
    import types

    import numpy as np
    import torch

    class Torch:
        int32, float64 = torch.int32, torch.float64

        @staticmethod
        def empty(shape, dtype=None, pin_memory=False):
            return torch.empty(shape, dtype=dtype)

        class cuda:
            @staticmethod
            def synchronize():
                pass

    class M:
        def __init__(self, n):
            self.n = n

        def info(self):
            return {"nleaves": self.n, "n": 512, "bs": 64}

        def close(self):
            pass

    calls = {"from_blocks": 0}

    class S:
        @staticmethod
        def spamm_to_blocks(ctx, m, out=None):
            return out

        @staticmethod
        def spamm_trim(ctx):
            pass

        @staticmethod
        def spamm_from_blocks(ctx, n, bs, bi, bj, pay):
            calls["from_blocks"] += 1
            return M(len(bi))

        @staticmethod
        def spamm_multiply(ctx, A, B, tau, mode, prec, stats=False):
            return M(5), {"kept_flops": 1e9}

    args = types.SimpleNamespace(e2e_steps=3, tau=1e-6, mode="combined", prec="fp64")
    monkeypatch.setattr(bench, "host_available_bytes", lambda: 1 << 40)
    r = bench.run_e2e(S, None, M(7), M(6), args, 64, Torch, np)
    assert r["steps"] == 3 and calls["from_blocks"] == 2 * 4
    assert r["h2d_bytes_per_step"] == (7 + 6) * (64 * 64 * 8 + 8)
    assert r["d2h_bytes_per_step"] == 5 * (64 * 64 * 8 + 16)
    assert r["host_reserve_bytes"] == 7 * 64 * 64 * 8
    monkeypatch.setattr(bench, "host_available_bytes", lambda: 0)
    assert bench.run_e2e(S, None, M(7), M(6), args, 64, Torch, np)["host_reserve_bytes"] == 0


def test_latency_percentiles_are_nearest_rank():
    ms = [float(v) for v in range(100, 0, -1)]  # 100 multiplies, 1..100 ms, unsorted
    r = bench.latency_summary(ms)
    assert r == {"p50_ms": 50.0, "p99_ms": 99.0, "steps": 100}
    assert bench.latency_summary(ms[:50])["p99_ms"] == 100.0  # 50 repeats: p99 is the slowest
    assert bench.latency_summary([3.0]) == {"p50_ms": 3.0, "p99_ms": 3.0, "steps": 1}


def test_latency_repeats_default_to_fifty(monkeypatch):
    monkeypatch.setattr("sys.argv", ["bench.py"])
    assert bench.parse_args().latency_repeats == 50


def test_dtype_is_the_arithmetic_type_of_the_form():
    assert [bench.compute_dtype(p) for p in ("fp64", "bf16_split", "bf16_split4", "fp16_scaled", "auto")] == \
        ["f64", "bf16", "bf16", "f16", "mixed"]
