"""The sampled oracle: windows of output leaves and the stratified estimate
of ||AB - C||_F for problems whose exact product is too large to form.
A census (every output leaf sampled) must reproduce the full oracle error;
with real samples the interval must cover it at about the nominal rate."""
import numpy as np
import pytest

import oracle
import synth
from oracle import sampled


def _truth(pa, pb, bs, tau, mode):
    MA, MB = oracle.from_dense(synth.dense(pa), bs), oracle.from_dense(synth.dense(pb), bs)
    C, _ = oracle.multiply(MA, MB, tau, mode)
    return oracle.error(oracle.exact(MA, MB), C)


def test_leaf_bounds_row_is_the_per_leaf_bound():
    for p in (synth.lattice_3d(4096, alpha=0.8, seed=1), synth.model_1d(2048, alpha=0.05, seed=1)):
        js = np.arange(40)
        row = synth.leaf_bounds_row(p, 64, 5, js)
        assert np.array_equal(row, [synth.leaf_bound(p, 64, 5, int(j)) for j in js])
        # the bound is symmetric in the two leaf indices (B's columns use rows of it)
        assert all(synth.leaf_bound(p, 64, 5, int(j)) == synth.leaf_bound(p, 64, int(j), 5) for j in js)


def test_window_leaf_equals_the_full_product():
    pa, pb = synth.lattice_3d(1024, alpha=0.8, seed=1), synth.lattice_3d(1024, alpha=0.8, seed=2)
    bs, tau = 64, 1e-5
    MA, MB = oracle.from_dense(synth.dense(pa), bs), oracle.from_dense(synth.dense(pb), bs)
    C, _ = oracle.multiply(MA, MB, tau, oracle.COMBINED)
    X = oracle.exact(MA, MB)
    for i, j in ((0, 0), (3, 9), (15, 2)):
        A_row, B_col = sampled.window_inputs(pa, pb, bs, [i], [j])
        Cw, _ = sampled.window_product(A_row, B_col, tau, oracle.COMBINED)
        Xw = sampled.window_exact(A_row, B_col)
        for full, win in ((C, Cw), (X, Xw)):
            a = [q for q in range(full.m) if (full.bi[q], full.bj[q]) == (i, j)]
            b = [q for q in range(win.m) if (win.bi[q], win.bj[q]) == (i, j)]
            assert len(a) == len(b)
            if a:
                assert np.array_equal(full.data[a[0]], win.data[b[0]])


def test_census_reproduces_the_full_error():
    pa, pb = synth.lattice_3d(1024, alpha=0.8, seed=1), synth.lattice_3d(1024, alpha=0.8, seed=2)
    bs, tau = 64, 1e-4
    truth = _truth(pa, pb, bs, tau, oracle.COMBINED)
    r = sampled.error_estimate(pa, pb, bs, tau, oracle.COMBINED, samples=10 ** 6, seed=0)
    assert r["samples"] == 16 * 16
    assert r["estimate"] == pytest.approx(truth, rel=1e-12)
    assert r["low"] == r["high"] == r["estimate"]
    assert r["exact_norm"] == pytest.approx(np.linalg.norm(synth.dense(pa) @ synth.dense(pb)), rel=1e-12)


def test_interval_covers_the_error_at_about_the_nominal_rate():
    pa = pb = synth.model_1d(2048, alpha=0.02, seed=1)
    bs, tau = 32, 1e-6
    truth = _truth(pa, pb, bs, tau, oracle.SPAMM)
    est, cover = [], 0
    for seed in range(12):
        r = sampled.error_estimate(pa, pb, bs, tau, oracle.SPAMM, samples=128, seed=seed)
        assert r["samples"] == 128
        est.append(r["err_sq"])
        cover += r["low"] <= truth <= r["high"]
    assert cover >= 9, cover  # nominal 95 %; measured 16 of 20 seeds at this size
    # the squared-error estimator is unbiased: its mean over seeds is near the truth
    assert np.mean(est) == pytest.approx(truth ** 2, rel=0.12)
