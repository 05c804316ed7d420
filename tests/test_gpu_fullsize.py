"""Parity at the detector workload's full size (65,536 chains, vertex cap 256,
straight jittered starts) in the launch configuration bench.py times (the
autotuned persistent launch of a lean chain kernel: one warp or one lane per
chain, whichever the autotuner timed faster):

* the first 2,000 steps of 96 chains sampled across the whole launch replay
  the FP64 oracle's trajectories (same Philox streams, chain by chain);
* after the full 100,000 steps every chain is healthy and its bookkeeping
  exact, and the final states of 512 sampled chains have the oracle's log
  density (|delta log p| <= 1e-5 + 2e-6 n on identical states).
"""
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


def _detector(api, ctx, n_steps):
    sc = S.detector(n_chains=65_536, n_steps=n_steps)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    return sc, medium, geom, api.Chains(ctx, medium, geom, sc.run)


def test_full_launch_replays_sampled_chains(api, ctx, oracle_lib):
    O = oracle_lib
    steps = 2000
    sc, medium, geom, ch = _detector(api, ctx, steps)
    li = ch.launch_info()
    assert len(li) == 1 and li[0]["general"] in (0, 4) and li[0]["hi"] == 65_536
    ch.run_steps(steps)
    xyz, n, st = ch.read_states()
    acc = ch.read_accumulators()
    assert np.all(st == steps)
    sample = np.arange(96) * 682 + 5
    clean = 0
    for c in sample:
        oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 1, 256, chain_offset=int(c))
        margin = oc.run(steps, margins=True)
        if not margin[0] > 1e-3:
            continue
        clean += 1
        k = int(n[c])
        assert k == oc.n[0], (c, k, oc.n[0])
        assert np.allclose(xyz[c, :, :k].T, oc.xyz[0, :k], atol=2e-4), c
        oa = oc.accumulators()
        assert np.array_equal(acc[c, 8:12], oa["prop"][0]) and np.array_equal(acc[c, 12:16], oa["acc"][0])
    assert clean >= 24, clean  # ~35 of 96 stay clear of the threshold for 2,000 steps


def test_full_size_run_health_and_densities(api, ctx, oracle_lib):
    import torch
    O = oracle_lib
    steps = 100_000
    sc, medium, geom, ch = _detector(api, ctx, steps)
    ch.run_steps(steps)
    assert ch.status() == 0
    xyz, n, st = ch.read_states()
    acc = ch.read_accumulators()
    assert np.all(st == steps)
    assert n.min() >= 2 and n.max() <= 256
    assert np.all(acc[:, 8:12].sum(axis=1) == steps)          # every step is one proposal
    assert np.all(acc[:, 12:16] <= acc[:, 8:12])              # acceptances <= proposals
    assert np.all(acc[:, 0] == steps - sc.run.burn_in)        # recorded states
    mean_n = acc[:, 2] / acc[:, 0]
    assert np.all((mean_n >= 2) & (mean_n <= 256))
    # identical-state densities of sampled final paths (absolute frame for pmc_logp)
    rng = np.random.default_rng(0)
    sample = rng.choice(65_536, size=512, replace=False)
    cap = 256
    batch = np.zeros((3, len(sample), cap), dtype=np.float32)
    for b, c in enumerate(sample):
        batch[:, b, : n[c]] = xyz[c, :, : n[c]]
    lp = api.logp(ctx, medium, geom, 0, torch.from_numpy(batch).cuda(),
                  torch.from_numpy(n[sample].astype(np.int32)).cuda()).cpu().numpy()
    m, s, d = O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[0])
    for b, c in enumerate(sample):
        k = int(n[c])
        ref = O.logp(m, s, d, batch[:, b, :k].T.astype(np.float64))
        assert np.isfinite(ref)
        assert abs(lp[b] - ref) <= 1e-5 + 2e-6 * k, (c, k, lp[b], ref)


@pytest.mark.parametrize("name", ["batched", "layered"])
def test_full_size_multi_pair_launch_replays_sampled_chains(api, ctx, oracle_lib, name):
    """The batched workload (4,096 pairs, ~1.08 M chains, caps 64-1,024 in
    four classes, long classes with a shared window and global spill) and the
    layered one (60 sensors x 8,192 chains, cap 1,024, general kernel) at full
    size: 64 chains sampled across all pairs replay the oracle for 1,000 steps."""
    O = oracle_lib
    steps = 1000
    sc = S.batched(n_steps=steps) if name == "batched" else S.layered(n_steps=steps)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(steps)
    assert ch.status() == 0
    xyz, n, st = ch.read_states()
    acc = ch.read_accumulators()
    total = sum(p.n_chains for p in sc.pairs)
    starts = np.cumsum([0] + [p.n_chains for p in sc.pairs])
    rng = np.random.default_rng(1)
    sample = rng.choice(total, size=64, replace=False)
    clean = 0
    for c in sample:
        p = int(np.searchsorted(starts, c, side="right") - 1)
        pr = sc.pairs[p]
        oc = O.Chains(sc.medium, sc.sources[pr.source], sc.sensors[pr.sensor], sc.run, 1, pr.cap,
                      chain_offset=int(c))
        margin = oc.run(steps, margins=True)
        if not margin[0] > 1e-3:
            continue
        clean += 1
        k = int(n[c])
        assert k == oc.n[0], (c, p, k, oc.n[0])
        assert np.allclose(xyz[c, :, :k].T, oc.xyz[0, :k], atol=5e-4), (c, p)
        oa = oc.accumulators()
        assert np.array_equal(acc[c, 8:12], oa["prop"][0]) and np.array_equal(acc[c, 12:16], oa["acc"][0])
    assert clean >= 16, clean
