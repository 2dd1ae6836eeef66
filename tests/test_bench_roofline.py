"""The bench's per-stage roofline models (host logic, CPU): the dominant
blending stage's work from the kernels' counters, the FP32 peak from the SM
count and the clock, the HBM stages' algorithmic bytes, and visible-only
Adam counted over the rows it touches."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6800.0, "sm_max_mhz": 2000.0}
COUNTERS = dict(F=1000, evals_fwd=5000, evals_bwd=2000, walked_bwd=3000, contrib_positions=4000)


def test_blend_backward_work_and_peak():
    r = bench.stage_roofline("blend_bwd", 1.0, COUNTERS, N=100, Bv=2, pixels=64, passes=2, peaks=PEAKS,
                             clock_mhz=2000.0, n_sm=150)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(150 * 128 * 2 * 2000e6 / 1e12)          # 76.8 TFLOP/s
    assert r["achieved"] == pytest.approx((7.0 * 3000 + 50.0 * 2000) / 1e-3 / 1e12)
    assert r["survey"] == pytest.approx(70.0 * 4000 / 1e-3 / 1e12)


def test_hbm_stage_bytes():
    r = bench.stage_roofline("preprocess", 2.0, COUNTERS, N=100, Bv=2, pixels=64, passes=2, peaks=PEAKS,
                             clock_mhz=2000.0, n_sm=150)
    assert r["bound"] == "hbm" and r["peak"] == 6800.0
    assert r["achieved"] == pytest.approx((100 * 240.0 + 2 * 100 * 52.0) / 2e-3 / 1e9)
    r = bench.stage_roofline("sort", 1.0, COUNTERS, N=100, Bv=2, pixels=64, passes=2, peaks=PEAKS,
                             clock_mhz=2000.0, n_sm=150)
    assert r["achieved"] == pytest.approx(2 * 1000 * 24.0 / 1e-3 / 1e9)


def test_adam_dense_and_visible_only():
    dense = bench.stage_roofline("adam", 1.0, COUNTERS, N=100, Bv=2, pixels=64, passes=2, peaks=PEAKS,
                                 clock_mhz=2000.0, n_sm=150)
    assert dense["achieved"] == pytest.approx(59 * 28.0 * 100 / 1e-3 / 1e9)
    sparse = bench.stage_roofline("adam", 1.0, dict(COUNTERS, visible_gaussians=30), N=100, Bv=2, pixels=64,
                                  passes=2, peaks=PEAKS, clock_mhz=2000.0, n_sm=150)
    assert sparse["achieved"] == pytest.approx((59 * 28.0 * 30 + 100) / 1e-3 / 1e9)
