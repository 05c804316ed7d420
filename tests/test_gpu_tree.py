"""GPU parity of the tree-coordinate within-dimension move (section "Path
proposal distribution"; appendix "Path space coordinate system") with the
FP64 oracle: the same Philox stream on both sides replays the oracle's
trajectories, and the chains' intensity equals the independent quadrature
(vertex cap 3) and the forward tracer (a well-mixing scene).
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


def _tree_scene(name, n_chains=64):
    if name == "general":
        sc = S.general_small(n_chains=n_chains, n_steps=300)
    else:
        sc = S.plain(n_chains=n_chains, n_steps=300)
    sc.run.within = S.WITHIN_TREE
    sc.run.sigma = 0.5
    sc.run.init = S.INIT_STRAIGHT
    sc.run.init_k = 40 if name.endswith("_long") else 6
    sc.run.init_jitter = 0.002 if name.endswith("_long") else 0.02  # 40 vertices keep clear of the sensor
    sc.run.layout = S.LAYOUT_LANE if name.startswith("plain_lane") else S.LAYOUT_WARP
    return sc


# kernel kind, shared window and chain count per case: 7 the lean warp-per-chain tree
# kernel, 8 the lane-per-chain one (window 16; or 4, so that most of every path lives in
# the global block, with 50 chains, so that the second work item has lanes without a
# chain; or paths of 42 vertices, more than the warp's proposal pool holds, so that most
# proposals live in the chains' global blocks), 2 the general warp-per-chain one
TREE_CASES = {"plain": (7, 0, 64), "plain_lane": (8, 16, 64), "plain_lane_spill": (8, 4, 50),
              "plain_lane_long": (8, 16, 64), "general": (2, 0, 64)}


@pytest.mark.parametrize("name", list(TREE_CASES))
def test_tree_trajectory_replay(api, ctx, oracle_lib, name):
    """Every chain whose accept decisions never came within 1e-3 of the
    threshold ends in the oracle's state (vertex count and positions), with
    the lean tree kernels (homogeneous medium, isotropic source, rho = 1,
    Henyey-Greenstein; one warp or one lane per chain) and the general one."""
    O = oracle_lib
    kind, window, n_chains = TREE_CASES[name]
    sc = _tree_scene(name, n_chains)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run, smem_window=window)
    assert ch.launch_info()[0]["general"] == kind
    if window:
        assert ch.launch_info()[0]["smem_cap"] == window
    ch.run_steps(sc.run.n_steps)
    assert ch.status() == 0
    xyz, n, st = ch.read_states()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, n_chains, sc.pairs[0].cap)
    margin = oc.run(sc.run.n_steps, margins=True)
    assert np.all(st == sc.run.n_steps)
    clean = margin > 1e-3
    assert clean.sum() >= 18
    for c in np.nonzero(clean)[0]:
        assert n[c] == oc.n[c], (c, n[c], oc.n[c])
        k = int(n[c])
        assert np.allclose(xyz[c, :, :k].T, oc.xyz[c, :k], atol=2e-4), (c, np.abs(xyz[c, :, :k].T - oc.xyz[c, :k]).max())
    acc = ch.read_accumulators()
    oacc = oc.accumulators()
    for c in np.nonzero(clean)[0]:
        assert np.array_equal(acc[c, 8:12], oacc["prop"][c])
        assert np.array_equal(acc[c, 12:16], oacc["acc"][c])
    # tree proposals are accepted at a useful rate
    assert 0.05 < acc[:, 12].sum() / acc[:, 8].sum() < 0.95


@pytest.mark.parametrize("window", [16, 4])
def test_lane_tree_gradient_accumulators_replay_oracle(api, ctx, oracle_lib, window):
    """Tree-move chains with score accumulation on the lane layout (the
    rebuild of every cached factor after an accepted tree move, including
    d log sigma / dg per vertex): for every chain whose decisions stayed away
    from the threshold the FP64 accumulators equal the oracle's."""
    O = oracle_lib
    sc = _tree_scene("plain_lane")
    sc.run.n_steps, sc.run.burn_in, sc.run.gradients = 600, 100, True
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run, smem_window=window)
    assert ch.launch_info()[0]["general"] == 8
    ch.run_steps(600)
    assert ch.status() == 0
    acc = ch.read_accumulators()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, sc.pairs[0].cap)
    margin = oc.run(600, margins=True)
    oa = oc.accumulators()
    clean = np.nonzero(margin > 1e-3)[0]
    assert len(clean) >= 24
    for c in clean:
        assert acc[c, 0] == oa["n_rec"][c] and acc[c, 1] == oa["n_direct"][c] and acc[c, 2] == oa["sum_n"][c]
        assert abs(acc[c, 3] / oa["sum_L"][c] - 1) < 1e-5 and abs(acc[c, 4] / oa["sum_L2"][c] - 1) < 1e-5
        assert abs(acc[c, 5] - oa["sum_score"][c, 2]) < 1e-3 * (abs(oa["sum_score"][c, 2]) + oa["n_rec"][c])
        assert np.array_equal(acc[c, 8:12], oa["prop"][c]) and np.array_equal(acc[c, 12:16], oa["acc"][c])


@pytest.mark.parametrize("layout", [S.LAYOUT_WARP, S.LAYOUT_LANE])
def test_tree_single_scatter_sector(api, ctx, layout):
    """Cap 3 with tree moves: I = Z2 + Z3 by independent quadrature."""
    sc = S.plain(n_chains=4096, n_steps=20000, cap=3)
    sc.run.within = S.WITHIN_TREE
    sc.run.sigma = 0.6
    sc.run.layout = layout
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(20000)
    e = ch.read_estimator()[0]
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(e["intensity"] - ref) < 3 * e["std_err"], (e["intensity"], e["std_err"], ref)
    assert e["rel_err"] < 0.005


@pytest.mark.parametrize("layout", [S.LAYOUT_WARP, S.LAYOUT_LANE])
def test_tree_chains_match_tracer(api, ctx, layout):
    """Well-mixing scene (isotropic scattering, large close sensor, cap 24):
    the intensity of tree-move chains equals the GPU tracer's (truncated at
    the same number of scatterings).  The lane layout runs with an 8-vertex
    window, so that longer paths and proposals reach the global block."""
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.0)
    src, sen = S.Source(), S.Sensor((0.0, 0.0, 1.5), 0.5)
    cap = 24
    run = S.Run(seed=99, n_steps=30000, burn_in=3000, within=S.WITHIN_TREE, sigma=0.8, layout=layout)
    medium = api.Medium(ctx, med)
    geom = api.Geometry(ctx, [src], [sen], [S.Pair(0, 0, 4096, cap)])
    ch = api.Chains(ctx, medium, geom, run, smem_window=8 if layout == S.LAYOUT_LANE else 0)
    ch.run_steps(run.n_steps)
    e = ch.read_estimator()[0]
    tr = api.trace(ctx, medium, geom, 0, 7, 400_000_000, max_scatter=cap - 2)
    assert abs(e["intensity"] - tr["I"]) < 3 * math.hypot(e["std_err"], tr["se"]), (e, tr)
    assert e["rel_err"] < 0.01


@pytest.mark.parametrize("b1,steps", [(0.1, 120_000), (0.3, 200_000), (0.5, 400_000)])
def test_paper_table_relative_yield(api, ctx, b1, steps):
    """The paper's worked example (Table tbl:results, tests/golden): B of the
    two-sensor scene from tree-move chains started on straight paths agrees
    with the paper's ray-tracer value within three combined uncertainties
    (the printed tracer uncertainty and our standard error).  Longer paths
    (larger b1) need longer runs to forget the straight starts: at b1 = 0.5
    1.2e5 steps still leave B at 0.52."""
    import os
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "paper_relative_yield.txt"))
    row = rows[np.isclose(rows[:, 0], b1)][0]
    sc = S.two_sensor(b1, n_chains=1024, n_steps=steps)
    sc.run.within = S.WITHIN_TREE
    sc.run.sigma = 0.3
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(sc.run.burn_in)
    Y = api.YieldRatio(ch, 0, 1)
    for _ in range((sc.run.n_steps - sc.run.burn_in) // 400):
        ch.run_steps(400)
        Y.observe()
    est = Y.estimate()
    assert abs(est["B"] - row[1]) < 3 * math.hypot(row[2], est["se"]), (b1, est, row)
    assert est["se"] < 0.01
    e = ch.read_estimator()
    assert max(e[0]["rhat"], e[1]["rhat"]) < 1.3
