"""The bench line's lane-op roofline follows the stated formula (no GPU).

Per proposal, FP32 work 90 (within-dimension move), 150 + n (birth) and
130 + n (death) at the measured move mix and mean vertex count n, plus 120
integer operations for the two Philox4x32-10 blocks of a step; MUFU work 8 /
16 / 14; peaks of 128 FP32+INT and 16 MUFU lanes per clock per SM (or a pipe
microbenchmark's rate where higher).  The expected values below are worked by
hand from those counts, not from bench.py's constants."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def _est(interior, end, birth, death, mean_n):
    return {"proposals": [interior, end, birth, death], "mean_n": mean_n}


def test_detector_mix_worked_by_hand(bench):
    # 60 / 20 / 20 with mean n = 12: FP32 0.6*90 + 0.2*162 + 0.2*142 = 114.8,
    # + 120 INT = 234.8 lane-ops; MUFU 0.6*8 + 0.2*16 + 0.2*14 = 10.8
    est = _est(57, 3, 20, 20, 12.0)
    pipes = {"fp32_per_s": 0.0, "mufu_per_s": 0.0}
    r = bench.lane_op_roofline(est, 1.097e10, 152, 2070.0, pipes)
    ops = r["lane_ops_per_proposal"]
    assert ops["fp32"] == pytest.approx(114.8, rel=1e-12)
    assert ops["int"] == 120.0
    assert ops["mufu"] == pytest.approx(10.8, rel=1e-12)
    peak = 128 * 152 * 2070e6
    assert r["pipe"] == "FP32+INT"
    assert r["peak"] == pytest.approx(peak / 1e12, rel=1e-12)
    assert r["achieved"] == pytest.approx(1.097e10 * 234.8 / 1e12, rel=1e-12)
    # the figure recomputed by hand for 1.097e10 proposals/s: 0.064
    assert r["frac"] == pytest.approx(0.06396, abs=5e-5)


def test_measured_pipe_rate_raises_the_peak(bench):
    est = _est(60, 0, 20, 20, 4.0)
    low = bench.lane_op_roofline(est, 1e10, 152, 2070.0, {"fp32_per_s": 0.0, "mufu_per_s": 0.0})
    high = bench.lane_op_roofline(est, 1e10, 152, 2070.0, {"fp32_per_s": 5e13, "mufu_per_s": 0.0})
    assert high["peak"] == pytest.approx(50.0)
    assert high["frac"] == pytest.approx(low["frac"] * low["peak"] / 50.0, rel=1e-12)


def test_alu_binds_at_the_configured_mix(bench):
    # per proposal MUFU needs 10.8 of 16 lanes/clk/SM against the ALU's 234.8 of
    # 128: the FP32+INT pipes bind (MUFU's peak never drops below its unit count)
    est = _est(60, 0, 20, 20, 12.0)
    r = bench.lane_op_roofline(est, 1e10, 152, 2070.0, {"fp32_per_s": 0.0, "mufu_per_s": 0.0})
    assert r["pipe"] == "FP32+INT"
    mufu_work = 0.6 * 8 + 0.2 * 16 + 0.2 * 14
    alu_work = 0.6 * 90 + 0.2 * 162 + 0.2 * 142 + 120
    assert mufu_work / 16 < alu_work / 128
    assert r["frac"] == pytest.approx(1e10 * alu_work / (128 * 152 * 2070e6), rel=1e-12)
