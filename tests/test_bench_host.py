"""Host-side arithmetic of bench.py's roofline lines (no GPU): the per-normal
figure per law, achieved = algorithmic work / kernel time, frac = achieved /
peak, and the gradient kernel's DRAM traffic scaled with N."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")

PEAKS = {"hbm_gbs": 6753.1, "bf16_tflops": 1853.7, "sm_max_mhz": 2070.0, "sm_count": 148}


def test_per_normal_figure_by_law():
    g, l = bench.GEN_INST_GAUSS, bench.GEN_INST_LOGN
    assert bench._gen_per_normal(0) == g and bench._gen_per_normal(2) == g
    assert bench._gen_per_normal(1) == g + l
    assert bench._gen_per_normal(3) == g + 0.5 * l   # half Gaussian, half lognormal


def test_value_roofline_arithmetic():
    d, N, K, t = 128, 1 << 20, 256, 0.37e-3
    r = bench.roofline("f16x3", d, N, K, 3, t, PEAKS, "measured")
    # the method's work only: one draw per normal, S1 and S2 per pair
    ops = N * d * bench._gen_per_normal(3) + N * K * 2.0
    assert r["achieved"] == pytest.approx(ops / t / 1e12)
    assert r["peak"] == pytest.approx(148 * 128 * 2070e6 / 1e12)   # the device's SM count, not a constant
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    issued = N * d * (bench._gen_per_normal(3) + bench.SPLIT_OPS) + N * K * bench.EPI_OPS_TC
    assert r["issued_frac"] == pytest.approx(issued / t / 1e12 / r["peak"])
    assert r["issued_frac"] > r["frac"]
    assert r["traffic"] == 194816
    assert r["tensor"]["achieved"] == pytest.approx(3 * 2.0 * N * d * K / t / 1e12)
    assert bench.roofline("f16x3", 64, N, K, 3, t, PEAKS, "measured")["traffic"] is None


def test_gradient_roofline_counts_one_draw():
    d, N, K, t = 1024, 1 << 20, 64, 2e-3
    r = bench.grad_roofline("f16x3", d, N, K, 0, t, PEAKS)
    ops = N * d * bench._gen_per_normal(0) + N * K * 2.0
    assert r["frac"] == pytest.approx(ops / t / 1e12 / (148 * 128 * 2070e6 / 1e12))
    rf = bench.grad_roofline("fp32", d, N, K, 0, t, PEAKS)
    assert rf["achieved"] == pytest.approx((N * d * bench._gen_per_normal(0) + N * K * (2 * d + 2.0)) / t / 1e12)


def test_gradient_traffic_is_per_launch_or_null():
    for key, fn in bench.GRAD_TRAFFIC.items():
        assert fn(1 << 20) > 0
    assert bench.grad_roofline("fp32", 1024, 1 << 20, 64, 0, 8e-3, PEAKS)["traffic"] is None
