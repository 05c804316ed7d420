"""pmc_trace_noalloc: the allocation-free tracer entry point.

It serves callers that cannot allocate device memory (their own pool
allocator holds the device, a fixed memory budget, or no tolerance for the
synchronisation of cudaMalloc / cudaFree).  Its accumulators sit in a device
array that the library holds for the life of the process, so this test calls
it twice in a row (the second call must not see the first call's sums) and
compares both calls, pair by pair, with pmc_trace, which allocates its own
accumulators.  The file is named to be collected last.
"""
import math

import numpy as np
import pytest

from paper_1811_04156_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def test_trace_noalloc_matches_trace_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1811_04156_gb300 import build
    build.build()
    from paper_1811_04156_gb300 import api
    from paper_1811_04156_gb300._lib import PMC_NOALLOC_MAX_PAIRS, PathmcError

    ctx = api.Context(0)
    med = api.Medium(ctx, S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.6))
    sensors = [S.Sensor((0.0, 0.0, 1.5), 0.5), S.Sensor((1.0, 0.5, 2.0), 0.4), S.Sensor((-2.0, 0.0, 0.5), 0.6)]
    pairs = [S.Pair(0, i, 1, 32) for i in range(3)]
    geom = api.Geometry(ctx, [S.Source()], sensors, pairs)
    n_photons = 20_000_000
    for call, ids in enumerate(([0, 1, 2], [2, 0, 1])):
        out = api.trace_noalloc(ctx, med, geom, ids, seed=4242, n_photons=n_photons, max_scatter=30)
        for row, p in enumerate(ids):
            ref = api.trace(ctx, med, geom, p, 4242, n_photons, max_scatter=30)
            raw = out[row]
            N = raw[3]
            assert N == n_photons
            I = raw[0] / N
            se = math.sqrt(max(raw[1] / N - I * I, 0.0) / N)
            # tolerance of the tracer tests: 3 combined standard errors
            assert abs(I - ref["I"]) < 3 * math.hypot(se, ref["se"]), (call, p, I, ref["I"])
            # same photon streams: equal up to the order of the FP64 sums
            assert np.allclose(raw, ref["raw"], rtol=1e-9, atol=0), (call, p, raw, ref["raw"])
    with pytest.raises(PathmcError) as ei:
        api.trace_noalloc(ctx, med, geom, [0] * (PMC_NOALLOC_MAX_PAIRS + 1), seed=1, n_photons=10)
    assert ei.value.code == 1
