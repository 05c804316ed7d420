"""Parity of the lane-per-chain kernel (PMC_LAYOUT_LANE) with the FP64 oracle
and with the warp-per-chain kernel: the same Markov chain (section "Numerical
path integration", Eq. acceptFact; appendix "Jump proposal") and the same
Philox stream, one chain per lane.

Replays: every chain whose accept decisions never came within 1e-3 of the
threshold ends in the oracle's state (vertex count, positions within 2e-4 m,
proposal and acceptance counts exactly).
"""
import math

import numpy as np
import pytest

import quadrature as Q
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


def _chains(api, ctx, sc, **kw):
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    return medium, geom, api.Chains(ctx, medium, geom, sc.run, **kw)


def _replay(O, sc, ch, steps, cap, n_chains, min_clean):
    xyz, n, st = ch.read_states()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, n_chains, cap)
    margin = oc.run(steps, margins=True)
    assert np.all(st == steps)
    clean = np.nonzero(margin > 1e-3)[0]
    assert len(clean) >= min_clean, len(clean)
    acc = ch.read_accumulators()
    oa = oc.accumulators()
    for c in clean:
        assert n[c] == oc.n[c], (c, n[c], oc.n[c])
        k = int(n[c])
        assert np.allclose(xyz[c, :, :k].T, oc.xyz[c, :k], atol=2e-4), (c, np.abs(xyz[c, :, :k].T - oc.xyz[c, :k]).max())
        assert np.array_equal(acc[c, 8:12], oa["prop"][c]) and np.array_equal(acc[c, 12:16], oa["acc"][c])
        assert acc[c, 0] == oa["n_rec"][c] and acc[c, 1] == oa["n_direct"][c] and acc[c, 2] == oa["sum_n"][c]
        assert abs(acc[c, 3] / oa["sum_L"][c] - 1) < 1e-5
    return n


@pytest.mark.parametrize("window", [16, 64])
def test_lane_trajectory_replay(api, ctx, oracle_lib, window):
    """Plain scene, 64 chains (two work items of 32) x 400 steps."""
    sc = S.plain(n_chains=64, n_steps=400)
    sc.run.burn_in = 50
    sc.run.layout = S.LAYOUT_LANE
    _, _, ch = _chains(api, ctx, sc, smem_window=window)
    info = ch.launch_info()[0]
    assert info["general"] == 4 and info["smem_cap"] == window
    ch.run_steps(400)
    assert ch.status() == 0
    _replay(oracle_lib, sc, ch, 400, 64, 64, 40)


def test_lane_spill_and_ragged_chain_count(api, ctx, oracle_lib):
    """A 4-vertex shared window with paths of 10-40 vertices (births, deaths
    and shifts across the window edge in global memory) and 70 chains (a
    partial last work item)."""
    sc = S.plain(n_chains=70, n_steps=300, cap=64)
    sc.medium.lambda_s = 0.05
    sc.run.init = S.INIT_STRAIGHT
    sc.run.init_k = 20
    sc.run.init_jitter = 0.002
    sc.run.layout = S.LAYOUT_LANE
    _, _, ch = _chains(api, ctx, sc, smem_window=4, warps_per_block=2)
    ch.run_steps(300)
    assert ch.status() == 0
    n = _replay(oracle_lib, sc, ch, 300, 64, 70, 24)
    assert (n > 4).sum() >= 20


def test_lane_vertex_cap_reached(api, ctx, oracle_lib):
    """Cap 6: births at the cap are proposed and rejected, as in the oracle."""
    sc = S.plain(n_chains=96, n_steps=500, cap=6)
    sc.medium.lambda_s = 0.1
    sc.run.layout = S.LAYOUT_LANE
    _, _, ch = _chains(api, ctx, sc)
    ch.run_steps(500)
    assert ch.status() == 0
    n = _replay(oracle_lib, sc, ch, 500, 6, 96, 40)
    assert (n == 6).sum() >= 10


def test_lane_matches_warp_kernel(api, ctx):
    """Detector geometry, 4,096 chains x 3,000 steps from the configured
    straight starts: the lane and warp kernels take the same decisions (they
    differ only in the rounding of a few sums), so nearly every chain ends in
    the same state and the estimates agree."""
    res = {}
    for layout in (S.LAYOUT_WARP, S.LAYOUT_LANE):
        sc = S.detector(n_chains=4096, n_steps=3000)
        sc.run.layout = layout
        _, _, ch = _chains(api, ctx, sc)
        assert ch.launch_info()[0]["general"] == (4 if layout == S.LAYOUT_LANE else 0)
        ch.run_steps(3000)
        assert ch.status() == 0
        res[layout] = (ch.read_states(), ch.read_accumulators())
    (xw, nw, _), aw = res[S.LAYOUT_WARP]
    (xl, nl, _), al = res[S.LAYOUT_LANE]
    same = nw == nl
    assert same.mean() > 0.97, same.mean()
    close = [np.allclose(xw[c, :, :nw[c]], xl[c, :, :nl[c]], atol=1e-3) for c in np.nonzero(same)[0]]
    assert np.mean(close) > 0.97
    for k in range(8, 16):  # proposal and acceptance totals
        assert abs(al[:, k].sum() / aw[:, k].sum() - 1) < 0.01, k


def test_lane_single_scatter_sector(api, ctx):
    """Cap 3: I = Z2 + Z3 by independent quadrature."""
    sc = S.plain(n_chains=4096, n_steps=20000, cap=3)
    sc.run.layout = S.LAYOUT_LANE
    _, _, ch = _chains(api, ctx, sc)
    ch.run_steps(20000)
    e = ch.read_estimator()[0]
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(e["intensity"] - ref) < 3 * e["std_err"], (e["intensity"], e["std_err"], ref)
    assert e["rel_err"] < 0.003


def test_lane_chains_match_tracer(api, ctx):
    """Well-mixing scene (isotropic scattering, large close sensor, cap 24):
    the lane kernel's intensity equals the GPU tracer's truncated at the same
    number of scatterings."""
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.0)
    src, sen = S.Source(), S.Sensor((0.0, 0.0, 1.5), 0.5)
    cap = 24
    run = S.Run(seed=99, n_steps=40000, burn_in=4000, sigma=0.3, layout=S.LAYOUT_LANE)
    medium = api.Medium(ctx, med)
    geom = api.Geometry(ctx, [src], [sen], [S.Pair(0, 0, 8192, cap)])
    ch = api.Chains(ctx, medium, geom, run)
    ch.run_steps(run.n_steps)
    e = ch.read_estimator()[0]
    tr = api.trace(ctx, medium, geom, 0, 7, 400_000_000, max_scatter=cap - 2)
    assert abs(e["intensity"] - tr["I"]) < 3 * math.hypot(e["std_err"], tr["se"]), (e, tr)
    assert e["rel_err"] < 0.01


def test_lane_split_runs_are_bit_exact(api, ctx):
    """1,500 steps in one launch or in 500 + 1,000 give the same states."""
    out = []
    for parts in ((1500,), (500, 1000)):
        sc = S.plain(n_chains=256, n_steps=1500)
        sc.run.layout = S.LAYOUT_LANE
        _, _, ch = _chains(api, ctx, sc)
        for k in parts:
            ch.run_steps(k)
        out.append((ch.read_states(), ch.read_accumulators()))
    (xa, na, sa), aa = out[0]
    (xb, nb, sb), ab = out[1]
    assert np.array_equal(na, nb) and np.array_equal(xa, xb) and np.array_equal(sa, sb)
    assert np.array_equal(aa[:, 8:], ab[:, 8:])


def test_lane_gradient_accumulators_replay_oracle(api, ctx, oracle_lib):
    """Gaussian-step chains with score accumulation (PMC_FLAG_GRADIENTS) on
    the lane layout: for every chain whose decisions stayed away from the
    threshold the FP64 accumulators equal the oracle's (sum of d log sigma/dg
    within the warp kernel's 1e-3 tolerance, see the accumulator replay of the
    parity tests)."""
    O = oracle_lib
    sc = S.plain(n_chains=64, n_steps=600)
    sc.run.burn_in = 100
    sc.run.gradients = True
    sc.run.layout = S.LAYOUT_LANE
    _, _, ch = _chains(api, ctx, sc)
    assert ch.launch_info()[0]["general"] == 4
    ch.run_steps(600)
    assert ch.status() == 0
    acc = ch.read_accumulators()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 64)
    margin = oc.run(600, margins=True)
    oa = oc.accumulators()
    clean = np.nonzero(margin > 1e-3)[0]
    assert len(clean) >= 32
    for c in clean:
        assert acc[c, 0] == oa["n_rec"][c] and acc[c, 1] == oa["n_direct"][c] and acc[c, 2] == oa["sum_n"][c]
        assert abs(acc[c, 3] / oa["sum_L"][c] - 1) < 1e-5
        assert abs(acc[c, 5] - oa["sum_score"][c, 2]) < 1e-3 * (abs(oa["sum_score"][c, 2]) + oa["n_rec"][c])
        assert np.array_equal(acc[c, 8:12], oa["prop"][c]) and np.array_equal(acc[c, 12:16], oa["acc"][c])


def test_lane_gradients_match_warp_layout(api, ctx):
    """The score-function gradient estimator of the intensity from the lane
    and the warp layouts (same decisions, so nearly the same states) agree."""
    out = {}
    for layout in (S.LAYOUT_WARP, S.LAYOUT_LANE):
        sc = S.plain(n_chains=8192, n_steps=4000)
        sc.run.gradients = True
        sc.run.layout = layout
        _, _, ch = _chains(api, ctx, sc)
        ch.run_steps(4000)
        assert ch.status() == 0
        out[layout] = ch.grad_estimator()
    (gw, sw), (gl, sl) = out[S.LAYOUT_WARP], out[S.LAYOUT_LANE]
    for i in range(3):
        assert abs(gl[0][i] - gw[0][i]) <= 0.3 * sw[0][i], (i, gl, gw, sw)


def test_lane_mala_accumulators_replay_oracle(api, ctx, oracle_lib):
    """MALA chains with gradients (the gradients workload's moves) on the lane
    layout: every chain whose decisions stayed away from the threshold has the
    oracle's accumulators."""
    O = oracle_lib
    sc = S.gradients(n_chains=64, n_steps=600)
    sc.run.burn_in = 100
    sc.run.layout = S.LAYOUT_LANE
    _, _, ch = _chains(api, ctx, sc)
    assert ch.launch_info()[0]["general"] == 5
    ch.run_steps(600)
    assert ch.status() == 0
    acc = ch.read_accumulators()
    xyz, n, _ = ch.read_states()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 64)
    margin = oc.run(600, margins=True)
    oa = oc.accumulators()
    clean = np.nonzero(margin > 1e-3)[0]
    assert len(clean) >= 32
    for c in clean:
        assert n[c] == oc.n[c]
        assert np.allclose(xyz[c, :, :n[c]].T, oc.xyz[c, :n[c]], atol=2e-4), c
        assert acc[c, 0] == oa["n_rec"][c] and acc[c, 1] == oa["n_direct"][c] and acc[c, 2] == oa["sum_n"][c]
        assert abs(acc[c, 3] / oa["sum_L"][c] - 1) < 1e-5
        assert abs(acc[c, 5] - oa["sum_score"][c, 2]) < 1e-3 * (abs(oa["sum_score"][c, 2]) + oa["n_rec"][c])
        assert np.array_equal(acc[c, 8:12], oa["prop"][c]) and np.array_equal(acc[c, 12:16], oa["acc"][c])


def test_lane_mala_single_scatter_sector(api, ctx):
    """MALA on the lane layout, cap 3: I = Z2 + Z3 by independent quadrature."""
    sc = S.plain(n_chains=4096, n_steps=20000, cap=3)
    sc.run.within = S.WITHIN_MALA
    sc.run.layout = S.LAYOUT_LANE
    _, _, ch = _chains(api, ctx, sc)
    ch.run_steps(20000)
    e = ch.read_estimator()[0]
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(e["intensity"] - ref) < 3 * e["std_err"], (e["intensity"], e["std_err"], ref)
    assert e["rel_err"] < 0.003


def test_autotuner_cache_keeps_kernels_apart(api, ctx):
    """Tuned launch shapes are cached per context: a lean MALA run (which may
    take the lane layout) and a general MALA run of the same cap and chain
    count must not share an entry, or the second would run the lean kernel."""
    sc = S.plain(n_chains=65536, n_steps=100, cap=3)
    sc.run.within = S.WITHIN_MALA
    _, _, a = _chains(api, ctx, sc)
    sc2 = S.plain(n_chains=65536, n_steps=100, cap=3)
    sc2.run.within = S.WITHIN_MALA
    sc2.medium.f_sl = 0.45
    _, _, b = _chains(api, ctx, sc2)
    assert a.launch_info()[0]["general"] in (1, 5)
    assert b.launch_info()[0]["general"] == 1


def test_lane_layout_rejects_general_runs(api, ctx):
    """The lane layout runs the lean physics only (here: a simplified-Liu mixture)."""
    sc = S.plain(n_chains=64, n_steps=100)
    sc.medium.f_sl = 0.45
    sc.run.layout = S.LAYOUT_LANE
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    with pytest.raises(RuntimeError):
        api.Chains(ctx, medium, geom, sc.run)
