"""The sharded form on one GPU: a chain set split into windows of global
chain indices (pmc_shard_range over 2 and 3 ranks, the windows run one
after the other on this GPU, never concurrently) evolves every chain
exactly as the whole set does, and the summed per-pair moments give the
whole set's estimates (chains and pairs are independent: section
"Implementation")."""
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


@pytest.mark.parametrize("layout,world,within", [(S.LAYOUT_WARP, 2, S.WITHIN_PERTURB),
                                                 (S.LAYOUT_LANE, 3, S.WITHIN_PERTURB),
                                                 (S.LAYOUT_LANE, 3, S.WITHIN_TREE)])
def test_windows_replay_the_whole_set(api, ctx, layout, world, within):
    """With tree moves on the lane layout the warp pools its chains' moves, so
    a window regroups the chains that share a warp (and leaves lanes without
    a chain): a chain's arithmetic must not depend on its warp-mates."""
    sc = S.batched_small(n_chains=256, n_steps=3000)
    if layout == S.LAYOUT_LANE:
        sc.pairs = [p for p in sc.pairs if p.cap == 3] + [S.Pair(0, 4, 256, 64)]
    sc.run.layout = layout
    sc.run.within = within
    if within == S.WITHIN_TREE:
        sc.run.sigma = 0.5
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    shape = dict(warps_per_block=2, smem_window=16 if layout == S.LAYOUT_LANE else 0)
    whole = api.Chains(ctx, medium, geom, sc.run, **shape)
    whole.run_steps(3000)
    xw, nw, sw = whole.read_states()
    aw = whole.read_accumulators()
    est_w = whole.read_estimator()
    mom = np.zeros((len(sc.pairs), 40))
    for r in range(world):
        lo, hi = api.shard_range(sc.pairs, r, world)
        part = api.Chains(ctx, medium, geom, sc.run, chain_window=(lo, hi), **shape)
        assert part.total == hi - lo
        part.run_steps(3000)
        x, n, s = part.read_states()
        assert np.array_equal(n, nw[lo:hi]) and np.array_equal(s, sw[lo:hi])
        assert np.array_equal(x, xw[lo:hi])
        assert np.array_equal(part.read_accumulators(), aw[lo:hi])
        mom += part.read_moments()
        part.close()
    est, _, _ = api.estimate_from_moments(mom, whole.pair_z2())
    for a, b in zip(est, est_w):
        for k in ("intensity", "std_err", "rhat", "mean_n", "n_samples"):
            assert np.isclose(a[k], b[k], rtol=1e-11, atol=0), (k, a[k], b[k])


def test_window_errors(api, ctx):
    from paper_1811_04156_gb300._lib import PathmcError
    sc = S.plain(n_chains=64)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    for win in ((10, 10), (-1, 5), (0, 65), (40, 30)):
        with pytest.raises(PathmcError):
            api.Chains(ctx, medium, geom, sc.run, chain_window=win)


def test_one_launch_replays_the_per_class_launches(api, ctx):
    """PMC_FLAG_ONE_LAUNCH (every chain of an uneven batch in one persistent
    launch, longest caps first) runs the same Markov chains as one launch per
    vertex-cap class: identical states, counts and estimates."""
    from paper_1811_04156_gb300._lib import PMC_FLAG_ONE_LAUNCH
    sc = S.batched_small(n_chains=256, n_steps=2000)
    sc.run.layout = S.LAYOUT_WARP
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    per_class = api.Chains(ctx, medium, geom, sc.run, warps_per_block=2)
    one = api.Chains(ctx, medium, geom, sc.run, warps_per_block=2, flags=PMC_FLAG_ONE_LAUNCH)
    assert len(per_class.launch_info()) == 3 and len(one.launch_info()) == 1
    for ch in (per_class, one):
        ch.run_steps(2000)
    xa, na, sa = per_class.read_states()
    xb, nb, sb = one.read_states()
    assert np.array_equal(na, nb) and np.array_equal(sa, sb) and np.array_equal(xa, xb)
    assert np.array_equal(per_class.read_accumulators(), one.read_accumulators())
    for a, b in zip(per_class.read_estimator(), one.read_estimator()):
        assert a["intensity"] == b["intensity"] and a["std_err"] == b["std_err"]


def test_windows_seed_from_the_tracer_as_the_whole_set(api, ctx):
    """pmc_seed_from_tracer gives chain i of a pair the i-th accepted photon
    whatever chain window holds it: windows seed, and then step, exactly as
    the whole set."""
    sc = S.plain(n_chains=1000, n_steps=0, cap=64)
    sc.pairs = [S.Pair(0, 0, 700, 64), S.Pair(0, 0, 300, 64)]
    sc.run.burn_in = 0
    sc.run.layout = S.LAYOUT_WARP
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    shape = dict(warps_per_block=2)
    whole = api.Chains(ctx, medium, geom, sc.run, **shape)
    api.seed_from_tracer(whole, seed=31, photons_per_round=1 << 22)
    whole.run_steps(500)
    xw, nw, _ = whole.read_states()
    for win in ((0, 350), (350, 820), (820, 1000)):
        part = api.Chains(ctx, medium, geom, sc.run, chain_window=win, **shape)
        api.seed_from_tracer(part, seed=31, photons_per_round=1 << 22)
        part.run_steps(500)
        x, n, _ = part.read_states()
        assert np.array_equal(n, nw[win[0]:win[1]]) and np.array_equal(x, xw[win[0]:win[1]]), win
        part.close()
