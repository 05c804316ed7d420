"""pmc_trace_noalloc: the allocation-free tracer entry point.

It serves callers that cannot allocate device memory (their own pool
allocator holds the device, a fixed memory budget, or no tolerance for the
synchronisation of cudaMalloc / cudaFree).  Its accumulators sit in a device
array that the library holds for the life of the process, so this test calls
it twice in a row (the second call must not see the first call's sums) and
compares both calls, pair by pair, with pmc_trace, which allocates its own
accumulators: on a homogeneous scene, and on a layered medium with a
von Mises-Fisher source and sensors with the paper's detection probability.
Around the compared calls the device's free memory must not change.  The
file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1811_04156_gb300 import scenes as S

pytestmark = pytest.mark.gpu

FIELDS = ("sum_w", "sum_w2", "detected", "emitted", "sum_wl")


def _scenes():
    homogeneous = (S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.6), [S.Source()],
                   [S.Sensor((0.0, 0.0, 1.5), 0.5), S.Sensor((1.0, 0.5, 2.0), 0.4), S.Sensor((-2.0, 0.0, 0.5), 0.6)])
    rng = np.random.default_rng(11)
    layered = (S.Medium(S.LAYERED, g=0.9, f_sl=0.45, z0=-2.0, dz=0.5,
                        lambda_s_layers=0.8 * np.exp(0.3 * rng.normal(size=12)),
                        lambda_a_layers=5.0 * np.exp(0.3 * rng.normal(size=12))),
               [S.Source((0.1, -0.1, -0.5), S.EMIT_VMF, 5.0, (0.0, 0.0, 1.0))],
               [S.Sensor((0.2, 0.1, 0.9), 0.3, S.RHO_PAPER, (0.0, -1.0, 0.0)),
                S.Sensor((-0.6, 0.4, 0.2), 0.35, S.RHO_PAPER, (1.0, 0.0, 0.0))])
    return {"homogeneous": homogeneous, "layered_vmf_rho": layered}


@pytest.mark.parametrize("name", ["homogeneous", "layered_vmf_rho"])
def test_trace_noalloc_matches_trace_on_two_calls(name):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1811_04156_gb300 import build
    build.build()
    from paper_1811_04156_gb300 import api
    from paper_1811_04156_gb300._lib import PMC_NOALLOC_MAX_PAIRS, PathmcError

    ctx = api.Context(0)
    med_desc, sources, sensors = _scenes()[name]
    med = api.Medium(ctx, med_desc)
    pairs = [S.Pair(0, i, 1, 32) for i in range(len(sensors))]
    geom = api.Geometry(ctx, sources, sensors, pairs)
    n_photons = 20_000_000
    orders = (list(range(len(pairs))), list(reversed(range(len(pairs)))))
    refs = {p: api.trace(ctx, med, geom, p, 4242, n_photons, max_scatter=30) for p in range(len(pairs))}
    api.trace_noalloc(ctx, med, geom, [0], seed=1, n_photons=1000, max_scatter=30)  # first call: set-up
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    outs = [api.trace_noalloc(ctx, med, geom, ids, seed=4242, n_photons=n_photons, max_scatter=30)
            for ids in orders]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before                  # the calls allocated nothing
    for ids, out in zip(orders, outs):
        for row, p in enumerate(ids):
            got, ref = out[row], refs[p]
            assert got["emitted"] == n_photons and got["detected"] > 1000
            # same photon streams: equal up to the order of the FP64 sums
            for k in FIELDS:
                assert np.isclose(got[k], ref[k], rtol=1e-9, atol=0), (name, ids, p, k, got[k], ref[k])
            assert np.isclose(got["intensity"], ref["intensity"], rtol=1e-9, atol=0)
            assert np.isclose(got["std_err"], ref["std_err"], rtol=1e-6, atol=0)
    with pytest.raises(PathmcError) as ei:
        api.trace_noalloc(ctx, med, geom, [0] * (PMC_NOALLOC_MAX_PAIRS + 1), seed=1, n_photons=10, max_scatter=30)
    assert ei.value.code == 1
