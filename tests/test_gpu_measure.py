"""Pipe-rate microbenchmark of the benchmark harness (libpmcprobe.so, outside
the product library): measured FP32 and MUFU lane rates lie near the
unit-count peaks.  FP32: 128 lanes per clock per SM.  MUFU: the benchmark
alternates ex2 and lg2; on GB300 it measures ~21.3 lanes per clock per SM,
which is what 32 ex2 lanes/clk (doubled exponential throughput) and 16 lg2
lanes/clk give for an equal mix (2 / (1/32 + 1/16)), so the bounds admit up to
32 lanes per clock."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1811_04156_gb300 import build
    build.build()
    from paper_1811_04156_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def ctx(api):
    return api.Context(0)


def test_measured_pipe_rates_near_unit_counts(api, ctx):
    import torch
    sys.path.insert(0, ROOT)
    import bench
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    r = bench.measure_pipes(0, torch.cuda.current_stream())
    # clock between 1 GHz (power-capped) and 2.2 GHz (above the 2070 MHz maximum)
    assert 128 * n_sm * 1.0e9 * 0.5 < r["fp32_per_s"] < 128 * n_sm * 2.2e9
    assert 16 * n_sm * 1.0e9 * 0.5 < r["mufu_per_s"] < 32 * n_sm * 2.2e9
