"""The sharded form of the chain sets on the host (no GPU): the partition of
(pair, chain) work items over ranks, the per-pair moments that add across
ranks, and the estimate computed from them, against a plain two-pass
computation and across a world-size-2 gloo all-reduce.

Chains and pairs are independent (section "Implementation"; section
"Discussion" on running chains in parallel), so the only exchange step is the
sum of the per-pair moments at read time."""
import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1811_04156_gb300 import scenes as S  # noqa: E402


def _api():
    from paper_1811_04156_gb300 import build
    build.build()
    from paper_1811_04156_gb300 import api
    return api


def _standin_acc(n_pairs, per_pair, seed=5, ls=0.5, la=5.0):
    """Valid accumulator rows: N recorded states, n2 <= N direct ones, path
    lengths with sum_L2 >= sum_L^2 / N, vertex counts >= 2 per state."""
    rng = np.random.default_rng(seed)
    rows, pair = [], []
    for p in range(n_pairs):
        for _ in range(per_pair[p]):
            N = float(rng.integers(0, 4000)) if rng.random() > 0.05 else 0.0
            n2 = float(rng.binomial(int(N), 0.1 + 0.05 * p)) if N > 0 else 0.0
            meanL = 1.0 + rng.gamma(2.0, 0.3)
            sumL = meanL * N
            sumL2 = (meanL ** 2 + rng.gamma(2.0, 0.05)) * N
            sumn = (2.0 + rng.gamma(3.0, 1.0)) * N
            sumG = rng.normal(0.0, 5.0) * N
            prop = rng.integers(0, 1000, 4).astype(float)
            acc = np.floor(prop * rng.random(4))
            rows.append([N, n2, sumn, sumL, sumL2, sumG, 0.0, 0.0, *prop, *acc])
            pair.append(p)
    return np.array(rows), np.array(pair, dtype=np.int32)


def _two_pass(acc, pair, p, z2, ls, la):
    """Plain two-pass estimate of pair p (the definitions written out)."""
    a = acc[pair == p]
    N = a[:, 0]
    Nt = N.sum()
    pi = a[:, 1].sum() / Nt
    C = len(a)
    w = N / Nt
    ok = N > 0
    f = np.where(ok, a[:, 1] / np.where(ok, N, 1.0), 0.0)
    var_pi = np.sum(np.where(ok, w * w * (f - pi) ** 2, 0.0)) * C / (C - 1)
    I = z2 / pi
    se = I * math.sqrt(var_pi) / pi
    A = np.stack([a[:, 3] / ls ** 2 - (a[:, 2] - 2 * N) / ls, a[:, 3] / la ** 2, a[:, 5]], axis=1)
    sbar = A.sum(axis=0) / Nt
    s = np.where(ok[:, None], A / np.where(ok, N, 1.0)[:, None], 0.0)
    vs = np.sum(np.where(ok[:, None], (w[:, None] ** 2) * (s - sbar) ** 2, 0.0), axis=0) * C / (C - 1)
    cv = np.sum(np.where(ok[:, None], (w[:, None] ** 2) * (f - pi)[:, None] * (s - sbar), 0.0), axis=0) * C / (C - 1)
    dpi = I * sbar / pi
    gse = np.sqrt(I * I * vs + dpi * dpi * var_pi - 2 * I * dpi * cv)
    m1 = N > 1
    mL = a[m1, 3] / N[m1]
    vL = (a[m1, 4] / N[m1] - mL ** 2) * N[m1] / (N[m1] - 1)
    K = m1.sum()
    W = vL.mean()
    B = mL.var(ddof=1)
    nper = Nt / K
    rhat = math.sqrt(((nper - 1) / nper * W + B) / W)
    return I, se, rhat, I * sbar, gse


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_range_covers_every_chain_once_balanced_by_cap(world):
    api = _api()
    sc = S.batched()
    pairs = sc.pairs
    total = sum(p.n_chains for p in pairs)
    caps = np.repeat([p.cap for p in pairs], [p.n_chains for p in pairs]).astype(float)
    ranges = [api.shard_range(pairs, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == total
    for (lo, hi), (lo2, _) in zip(ranges, ranges[1:]):
        assert hi == lo2
    assert all(hi > lo for lo, hi in ranges)
    cost = np.array([caps[lo:hi].sum() for lo, hi in ranges])
    assert abs(cost.sum() - caps.sum()) < 1e-6
    # each rank within one chain's cost of the ideal share
    assert np.all(np.abs(cost - caps.sum() / world) <= caps.max())


def test_shard_range_edges():
    api = _api()
    pairs = [S.Pair(0, 0, 3, 1024), S.Pair(0, 0, 1, 64)]
    ranges = [api.shard_range(pairs, r, 4) for r in range(4)]
    assert ranges == [(0, 1), (1, 2), (2, 3), (3, 4)]
    from paper_1811_04156_gb300._lib import PathmcError
    with pytest.raises(PathmcError):
        api.shard_range(pairs, 0, 5)             # fewer chains than ranks
    with pytest.raises(PathmcError):
        api.shard_range(pairs, 2, 2)             # rank outside [0, world)


def test_estimate_from_moments_matches_two_pass():
    api = _api()
    ls, la = 0.5, 5.0
    acc, pair = _standin_acc(3, [40, 200, 7], ls=ls, la=la)
    z2 = np.array([3.2e-4, 1.1e-5, 2.0e-3])
    mom = api.moments_from_accumulators(acc, pair, 3, ls, la)
    est, g, gs = api.estimate_from_moments(mom, z2)
    for p in range(3):
        I, se, rhat, grad, gse = _two_pass(acc, pair, p, z2[p], ls, la)
        e = est[p]
        assert math.isclose(e["intensity"], I, rel_tol=1e-12)
        assert math.isclose(e["std_err"], se, rel_tol=1e-9)
        assert math.isclose(e["rhat"], rhat, rel_tol=1e-9)
        assert np.allclose(g[p], grad, rtol=1e-12)
        assert np.allclose(gs[p], gse, rtol=1e-8)
        a = acc[pair == p]
        assert e["n_samples"] == a[:, 0].sum()
        assert np.allclose(e["proposals"], a[:, 8:12].sum(axis=0))
    # the intensity and its error against the oracle's own reduction
    import oracle as O
    for p in range(3):
        a = acc[pair == p]
        I, se, _ = O.direct_estimate({"n_rec": a[:, 0], "n_direct": a[:, 1]}, z2[p])
        assert math.isclose(est[p]["intensity"], I, rel_tol=1e-12)
        assert math.isclose(est[p]["std_err"], se, rel_tol=1e-9)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    api = _api()
    ls, la = 0.5, 5.0
    acc, pair = _standin_acc(4, [100, 37, 512, 16], seed=9, ls=ls, la=la)
    caps = [64, 128, 1024, 96]
    pairs = [S.Pair(0, 0, int((pair == p).sum()), caps[p]) for p in range(4)]
    lo, hi = api.shard_range(pairs, rank, world)
    mom = api.moments_from_accumulators(acc[lo:hi], pair[lo:hi], 4, ls, la)
    t = torch.from_numpy(mom)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    z2 = np.array([1e-3, 2e-4, 3e-5, 4e-6])
    est, g, gs = api.estimate_from_moments(t.numpy(), z2)
    q.put((rank, lo, hi, [e["intensity"] for e in est], [e["std_err"] for e in est], [e["rhat"] for e in est],
           g.tolist(), gs.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_moments_all_reduce_equals_one_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, lo0, hi0, *v0), (r1, lo1, hi1, *v1) = res
    assert lo0 == 0 and hi0 == lo1 and hi1 == 665
    # both ranks hold the same all-reduced estimate, equal to one rank's over all chains
    api = _api()
    acc, pair = _standin_acc(4, [100, 37, 512, 16], seed=9)
    est, g, gs = api.estimate_from_moments(api.moments_from_accumulators(acc, pair, 4, 0.5, 5.0),
                                           np.array([1e-3, 2e-4, 3e-5, 4e-6]))
    one = ([e["intensity"] for e in est], [e["std_err"] for e in est], [e["rhat"] for e in est], g.tolist(),
           gs.tolist())
    for got in (v0, v1):
        for a, b in zip(got, one):
            assert np.allclose(a, b, rtol=1e-12, atol=0), (a, b)
