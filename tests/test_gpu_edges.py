"""Argument checking and degenerate inputs of the relative-light-yield,
bridge, histogram and tree/HMC entry points (errors come back as statuses,
nothing runs on bad input)."""
import math

import numpy as np
import pytest

from paper_1811_04156_gb300 import scenes as S

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


def _two(api, ctx, src1=(0.0, 0.0, 0.0), c1=(1.0, 0.0, 1.0)):
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.5)
    srcs = [S.Source(), S.Source(src1)]
    sens = [S.Sensor((0.0, 0.0, 1.5), 0.3), S.Sensor(c1, 0.3)]
    pairs = [S.Pair(0, 0, 64, 16), S.Pair(1, 1, 64, 16)]
    return api.Medium(ctx, med), api.Geometry(ctx, srcs, sens, pairs)


def test_yield_argument_errors(api, ctx):
    import torch
    from paper_1811_04156_gb300._lib import PathmcError
    medium, geom = _two(api, ctx)
    xyz = torch.zeros((3, 4, 16), device="cuda")
    n = torch.full((4,), 2, dtype=torch.int32, device="cuda")
    with pytest.raises(PathmcError):  # equal pairs
        api.yield_logratio(ctx, medium, geom, 0, 0, 0, xyz, n)
    with pytest.raises(PathmcError):  # side must be 0 or 1
        api.yield_logratio(ctx, medium, geom, 0, 1, 2, xyz, n)
    m2, g2 = _two(api, ctx, src1=(0.1, 0.0, 0.0))
    with pytest.raises(PathmcError):  # the pairs must share a source position
        api.yield_logratio(ctx, m2, g2, 0, 1, 0, xyz, n)
    m3, g3 = _two(api, ctx, c1=(0.0, 0.0, 3.0))
    with pytest.raises(PathmcError):  # sensors collinear with the source
        api.yield_logratio(ctx, m3, g3, 0, 1, 0, xyz, n)


def test_yield_logratio_degenerate_counts(api, ctx):
    """n outside [2, cap] gives NaN; an empty batch is a no-op."""
    import torch
    medium, geom = _two(api, ctx)
    xyz = torch.zeros((3, 3, 16), device="cuda")
    n = torch.tensor([1, 17, 0], dtype=torch.int32, device="cuda")
    out = api.yield_logratio(ctx, medium, geom, 0, 1, 0, xyz, n).cpu().numpy()
    assert np.all(np.isnan(out))
    e = api.yield_logratio(ctx, medium, geom, 0, 1, 0, torch.zeros((3, 0, 16), device="cuda"),
                           torch.zeros((0,), dtype=torch.int32, device="cuda"))
    assert e.numel() == 0


def test_bridge_and_histogram_argument_errors(api, ctx):
    import torch
    from paper_1811_04156_gb300._lib import PathmcError
    L = torch.zeros((5, 10), device="cuda")
    with pytest.raises(PathmcError):  # more groups than chains on a side
        api.bridge_ratio(ctx, L, 6, 4, groups=5)
    with pytest.raises(PathmcError):
        api.bridge_ratio(ctx, L[:0], 6, 4, groups=2)
    medium, geom = _two(api, ctx)
    with pytest.raises(PathmcError):  # empty length range
        api.trace_lengths(ctx, medium, geom, 0, 1, 1000, 2.0, 2.0, 8)
    ch = api.Chains(ctx, medium, geom, S.Run(seed=1, burn_in=0))
    hist = torch.zeros((2, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(PathmcError):
        ch.length_hist(3.0, 1.0, hist)
    ch.length_hist(0.0, 100.0, hist)  # direct paths of length ~1.2 m all land in bin 0
    h = hist.cpu().numpy()
    assert h[:, 0].sum() == 128 and h[:, 1:].sum() == 0


def test_tree_and_hmc_settings_are_checked(api, ctx):
    from paper_1811_04156_gb300._lib import PathmcError
    medium, geom = _two(api, ctx)
    with pytest.raises(PathmcError):  # HMC needs leapfrog steps
        api.Chains(ctx, medium, geom, S.Run(seed=1, within=S.WITHIN_HMC, mala_step=0.01, hmc_steps=0))
    with pytest.raises(PathmcError):  # HMC needs a step size
        api.Chains(ctx, medium, geom, S.Run(seed=1, within=S.WITHIN_HMC, mala_step=0.0))
    geom64 = api.Geometry(ctx, [S.Source()], [S.Sensor((0.0, 0.0, 1.5), 0.3)], [S.Pair(0, 0, 32, 64)])
    with pytest.raises(PathmcError):  # tree moves keep the whole cap in shared memory
        api.Chains(ctx, medium, geom64, S.Run(seed=1, within=S.WITHIN_TREE, sigma=0.3), smem_window=32,
                   warps_per_block=1)
    with pytest.raises(PathmcError):
        api.Chains(ctx, medium, geom, S.Run(seed=1, within=7))


def test_tree_and_hmc_from_direct_paths(api, ctx):
    """n = 2 has no tree node and no interior vertex: tree proposals move only
    the end vertex, HMC proposals fall back to end moves; chains stay finite."""
    medium, geom = _two(api, ctx)
    for run in (S.Run(seed=2, burn_in=0, within=S.WITHIN_TREE, sigma=0.3, p_within=1.0, p_birth=0.0, p_death=0.0),
                S.Run(seed=2, burn_in=0, within=S.WITHIN_HMC, mala_step=0.01, p_within=1.0, p_birth=0.0,
                      p_death=0.0)):
        ch = api.Chains(ctx, medium, geom, run)
        ch.run_steps(200)
        xyz, n, _ = ch.read_states()
        assert np.all(n == 2) and ch.status() == 0
        acc = ch.read_accumulators()
        assert acc[:, 8:12].sum() == 128 * 200
        assert np.all(np.isfinite(xyz[:, :, :2]))
