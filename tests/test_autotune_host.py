"""Autotuner decision logic (no GPU): admissibility by error, fastest wins,
nearest calibrated point, determinism, the leaf-size-restricted choice."""
import math

from paper_1906_08148_gb300.autotune import Autotuner, Choice, Point, decide


def _pt(n, alpha, tau, ms, arith, trunc):
    return Point(n, alpha, tau, decide(ms, arith, trunc), ms, arith, trunc)


MS = {"fp64/32": 40.0, "fp64/64": 30.0, "bf16_split/64": 3.0, "fp16_scaled/64": 2.0}


def test_fastest_admissible_form_wins():
    # both tensor forms accurate enough: the faster one
    assert decide(MS, {"bf16_split/64": 1e-6, "fp16_scaled/64": 2e-6}, 1e-4) == Choice("fp16_scaled", 64)
    # FP16 too coarse for this truncation error, BF16 fine
    assert decide(MS, {"bf16_split/64": 1e-6, "fp16_scaled/64": 2e-4}, 1e-4) == Choice("bf16_split", 64)
    # neither tensor form within the truncation error: the faster FP64 leaf size
    assert decide(MS, {"bf16_split/64": 1e-3, "fp16_scaled/64": 2e-3}, 1e-4) == Choice("fp64", 64)
    assert decide({**MS, "fp64/32": 20.0}, {}, 1e-4) == Choice("fp64", 32)
    # missing error measurement: not admissible
    assert decide(MS, {}, 1.0) == Choice("fp64", 64)
    assert decide({}, {}, 1.0) == Choice("fp64", 64)


def test_nearest_point_and_defaults():
    pts = [_pt(4096, 1.0, 1e-4, MS, {"bf16_split/64": 1e-6, "fp16_scaled/64": 1e-6}, 1e-3),
           _pt(65536, 1.0, 1e-8, MS, {"bf16_split/64": 1e-5, "fp16_scaled/64": 1e-5}, 1e-7)]
    t = Autotuner(pts)
    assert t.choose(4000, 1.05, 2e-4) == Choice("fp16_scaled", 64)
    assert t.choose(60000, 0.95, 1e-8) == Choice("fp64", 64)
    assert t.choose(60000, 0.95, 0.0) == Choice("fp64", 64)
    # inputs already built with 32 x 32 leaves: only the FP64 form exists there
    assert t.choose(4000, 1.0, 1e-4, bs=32) == Choice("fp64", 32)
    assert t.choose(4000, 1.0, 1e-4, bs=64) == Choice("fp16_scaled", 64)
    assert Autotuner([]).choose(4096, 1.0, 1e-4) == Choice("fp64", 64)
    # a pure function of the request: repeated and interleaved calls agree
    seq = [(4096, 1.0, 1e-4), (65536, 0.9, 1e-8), (8192, 1.2, 1e-6)]
    first = [t.choose(*q) for q in seq]
    assert [t.choose(*q) for q in seq[::-1]][::-1] == first


def test_table_round_trip(tmp_path):
    from paper_1906_08148_gb300 import autotune
    pts = [_pt(4096, 0.6, 1e-6, MS, {"bf16_split/64": 1e-6, "fp16_scaled/64": 5e-6}, 2e-6)]
    path = str(tmp_path / "t.json")
    autotune.save(pts, path, meta={"x": 1})
    back = autotune.load(path)
    assert back[0].choice == Choice("bf16_split", 64) and math.isclose(back[0].trunc_err, 2e-6)
    assert Autotuner(path=path).choose(4096, 0.6, 1e-6) == Choice("bf16_split", 64)


def test_truncation_error_per_leaf_size_and_rates(tmp_path):
    """The truncation error differs by leaf size (the kept set does): each
    candidate is judged against its own; rates round-trip and their median
    is what the server's slices are sized from."""
    from paper_1906_08148_gb300 import autotune
    ms = {"fp64/64": 30.0, "fp64/128": 35.0, "bf16_split4/64": 3.0, "bf16_split4/128": 2.5}
    arith = {"bf16_split4/64": 1e-8, "bf16_split4/128": 1e-8}
    # the 128 kept set keeps more, its truncation error is below the form's arithmetic error
    assert decide(ms, arith, {"64": 1e-6, "128": 5e-9}) == Choice("bf16_split4", 64)
    assert decide(ms, arith, {"64": 1e-6, "128": 1e-6}) == Choice("bf16_split4", 128)
    pts = [Point(4096, 1.0, 1e-6, decide(ms, arith, {"64": 1e-6, "128": 1e-6}), ms, arith, {"64": 1e-6, "128": 1e-6},
                 {"bf16_split4/64": 50000.0 + 1000 * i}, ("fp64/128",)) for i in range(3)]
    path = str(tmp_path / "t.json")
    autotune.save(pts, path)
    t = Autotuner(path=path)
    assert t.choose(4096, 1.0, 1e-6) == Choice("bf16_split4", 128)
    assert t.rate("bf16_split4", 64) == 51000.0 and t.rate("fp16_scaled", 64) is None
    assert autotune.load(path)[0].estimated == ("fp64/128",)


def test_claim_order_is_part_of_the_choice_and_round_trips(tmp_path):
    from paper_1906_08148_gb300.autotune import Autotuner, Choice, Point, load, save
    pts = [Point(16384, 1.0, 1e-6, Choice("fp16_scaled", 64, "longest"), {"fp16_scaled/64": 5.0, "fp64/64": 900.0},
                 {"fp16_scaled/64": 1e-6}, {"64": 1e-4}, {"fp16_scaled/64": 1.5e5}, (), {"morton": 5.2, "longest": 4.9}),
           Point(4096, 1.0, 1e-8, Choice("fp64", 64), {"fp64/64": 90.0}, {}, {"64": 0.0})]
    path = str(tmp_path / "t.json")
    save(pts, path)
    back = load(path)
    assert back[0].choice == Choice("fp16_scaled", 64, "longest") and back[0].order_ms["longest"] == 4.9
    assert back[1].choice.order == "auto"
    tuner = Autotuner(back)
    assert tuner.choose(16384, 1.0, 1e-6).order == "longest"
    # a given leaf size keeps the point's order when its winner has that size
    assert tuner.choose(16384, 1.0, 1e-6, bs=64) == Choice("fp16_scaled", 64, "longest")
