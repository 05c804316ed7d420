"""Parity of the GPU relative-light-yield path and path-length distributions
with the FP64 oracle (section "Comparison of relative light yield"; appendix
"Relative light yield transformation"; section "Comparison of timing
distributions").

Tolerances.  Log ratios on identical states: each of the two log densities
within 1e-5 + 2e-6 n of the oracle (the density tolerance), plus 2e-7 per
vertex for the FP32 log volume ratios of T, so |delta| <= 2 (1e-5 + 2e-6 n)
+ 2e-7 n.  Mapped vertices: within 5e-7 (1 + |y|) per coordinate (a few FP32
roundings of coordinates of size |y|).  Estimates: within 3 combined standard
errors.
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


def _two_sensor_scenes():
    full = S.two_sensor(0.3, n_chains=1, cap=128)
    mini = S.Scene("mini", S.Medium(S.LAYERED, g=0.8, f_sl=0.3, z0=-1.0, dz=1.0,
                                    lambda_s_layers=np.array([1.0, 0.6]), lambda_a_layers=np.array([8.0, 8.0])),
                   [S.Source((0.2, -0.1, 0.3), S.EMIT_VMF, 5.0, (0.1, 0.0, 1.0))],
                   [S.Sensor((0.2, -0.1, 2.3), 0.3, S.RHO_PAPER, (0.0, -1.0, 0.0)),
                    S.Sensor((1.4, 0.0, 1.9), 0.25, S.RHO_PAPER, (0.0, -1.0, 0.0))],
                   [S.Pair(0, 0, 1, 48), S.Pair(0, 1, 1, 48)], S.Run())
    return {"full": (full, 2.0), "mini": (mini, 0.3)}


def _side_batch(sc, side, lateral, batch, seed):
    src, sen = sc.sources[0], sc.sensors[side]
    cap = sc.pairs[side].cap
    xyz, n = S.random_paths(src.pos, sen.centre, sen.radius, batch, cap, 2, cap, seed, lateral=lateral)
    xs, ns = S.random_paths(src.pos, sen.centre, sen.radius, batch, cap, 2, 4, seed + 1, lateral=lateral)
    xyz[:, ::4, :] = xs[:, ::4, :]
    n[::4] = ns[::4]
    return xyz, n


@pytest.mark.parametrize("name", ["full", "mini"])
@pytest.mark.parametrize("side", [0, 1])
def test_yield_logratio_matches_oracle(api, ctx, oracle_lib, name, side):
    import torch
    O = oracle_lib
    sc, lateral = _two_sensor_scenes()[name]
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    m, s = O.medium(sc.medium), O.source(sc.sources[0])
    d0, d1 = O.sensor(sc.sensors[0]), O.sensor(sc.sensors[1])
    T = O.ymap(s, d0, d1)
    xyz, n = _side_batch(sc, side, lateral, 256, 31 + side)
    # a few paths with a vertex outside T's one-to-one domain (behind the cylinder axis)
    bad = [5, 77, 150]
    if side == 0:
        for b in bad:
            if n[b] >= 3:
                xyz[:, b, 1] = (np.asarray(sc.sources[0].pos) - 1.5 * T.rC * T.b0 / T.b1 * np.asarray(T.m))
    lr, mapped = api.yield_logratio(ctx, medium, geom, 0, 1, side, torch.from_numpy(xyz).cuda(),
                                    torch.from_numpy(n).cuda(), mapped=True)
    lr, mapped = lr.cpu().numpy(), mapped.cpu().numpy()
    dself, doth = (d0, d1) if side == 0 else (d1, d0)
    checked = 0
    for b in range(len(n)):
        k = int(n[b])
        x = xyz[:, b, :k].T.astype(np.float64)
        y_ref, lj = (O.ymap_forward if side == 0 else O.ymap_inverse)(T, x)
        if not np.isfinite(lj):
            assert lr[b] == -np.inf, (b, lr[b])
            continue
        y = mapped[:, b, :k].T.astype(np.float64)
        tol_pos = 5e-7 * (1.0 + np.abs(y_ref).max())
        assert np.abs(y - y_ref).max() <= tol_pos, (b, np.abs(y - y_ref).max(), tol_pos)
        ls = O.logp(m, s, dself, x)
        lo = O.logp(m, s, doth, y)
        if not (np.isfinite(ls) and np.isfinite(lo)):
            assert lr[b] == -np.inf, (b, lr[b], ls, lo)
            continue
        ref = (lo + lj - ls) if side == 0 else (lo - lj - ls)
        tol = 2 * (1e-5 + 2e-6 * k) + 2e-7 * k
        assert abs(lr[b] - ref) <= tol, (b, k, lr[b], ref)
        checked += 1
    assert checked > 100
    if side == 0:
        assert all(lr[b] == -np.inf for b in bad if n[b] >= 3)


def _run_yield(api, ctx, sc, rounds, thin, burn_rounds, tracer_seeds=False, keep_logs=False):
    """Chains of both pairs, observed every `thin` steps after `burn_rounds`.
    With tracer_seeds every chain starts from a weight-thinned tracer path (an
    exact draw from its target), as the paper seeds its chains; direct-path
    starts leave a burn-in transient of ~10^4 steps in these scenes."""
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    if tracer_seeds:
        api.seed_from_tracer(ch, seed=4242, photons_per_round=1 << 24)
    Y = api.YieldRatio(ch, 0, 1, max_obs=rounds if keep_logs else 0)
    for r in range(rounds):
        ch.run_steps(thin)
        if r >= burn_rounds:
            Y.observe()
    if keep_logs:
        return Y.estimate(), ch, Y
    return Y.estimate(), ch


def test_yield_ratio_symmetric_sensors(api, ctx):
    """Two sensors equidistant from an isotropic source in a homogeneous medium: B = 1."""
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.0)
    a = math.radians(70.0)
    sensors = [S.Sensor((0.0, 0.0, 1.2), 0.3), S.Sensor((1.2 * math.sin(a), 0.0, 1.2 * math.cos(a)), 0.3)]
    sc = S.Scene("sym", med, [S.Source()], sensors, [S.Pair(0, 0, 4096, 16), S.Pair(0, 1, 4096, 16)],
                 S.Run(seed=77, burn_in=0, sigma=0.1))
    est, _ = _run_yield(api, ctx, sc, 300, 20, 5, tracer_seeds=True)
    assert abs(est["B"] - 1.0) < 3 * est["se"], est
    assert est["se"] < 0.01


def test_yield_ratio_single_scatter_quadrature(api, ctx):
    """Cap 3: B = (Z2 + Z3)(sensor 1) / (Z2 + Z3)(sensor 0) by independent quadrature."""
    ls, la, g, R = 0.5, 5.0, 0.9, 0.3
    a = math.radians(50.0)
    sensors = [S.Sensor((0.0, 0.0, 1.0), R), S.Sensor((1.4 * math.sin(a), 0.0, 1.4 * math.cos(a)), R)]
    sc = S.Scene("cap3", S.Medium(lambda_s=ls, lambda_a=la, g=g), [S.Source()], sensors,
                 [S.Pair(0, 0, 4096, 3), S.Pair(0, 1, 4096, 3)], S.Run(seed=91, burn_in=0, sigma=0.05))
    est, _ = _run_yield(api, ctx, sc, 300, 10, 30)
    cext = 1.0 / ls + 1.0 / la
    ref = (Q.z2_closed(1.4, R, cext) + Q.z3(1.4, R, ls, la, g)) / (Q.z2_closed(1.0, R, cext) + Q.z3(1.0, R, ls, la, g))
    assert abs(est["B"] - ref) < 3 * est["se"], (est, ref)
    assert est["se"] / est["B"] < 0.01


def test_yield_ratio_matches_tracer_and_oracle(api, ctx, oracle_lib):
    """The paper's comparison in miniature: vMF emission, simplified-Liu/HG
    mixture, detection probability rho and a medium split by a plane; B from
    the chains through T equals I_1 / I_0 from the GPU forward tracer (both
    truncated at the chains' vertex cap), and the FP64 oracle chains agree."""
    O = oracle_lib
    sc, _ = _two_sensor_scenes()["mini"]
    cap = 24
    nc = 4096
    sc.pairs = [S.Pair(0, 0, nc, cap), S.Pair(0, 1, nc, cap)]
    sc.run = S.Run(seed=5, burn_in=0, sigma=0.1)
    est, _, Y = _run_yield(api, ctx, sc, 600, 25, 5, tracer_seeds=True, keep_logs=True)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    t0 = api.trace(ctx, medium, geom, 0, 11, 400_000_000, max_scatter=cap - 2)
    t1 = api.trace(ctx, medium, geom, 1, 12, 400_000_000, max_scatter=cap - 2)
    Bt = t1["I"] / t0["I"]
    se_t = Bt * math.hypot(t0["se"] / t0["I"], t1["se"] / t1["I"])
    assert abs(est["B"] - Bt) < 3 * math.hypot(est["se"], se_t), (est, Bt, se_t)
    assert est["se"] / est["B"] < 0.01
    # the optimal bridge on the same observations (Meng & Wong)
    ob = Y.estimate_bridge(groups=32)
    assert abs(ob["r"] - Bt) < 3 * math.hypot(ob["se"], se_t), (ob, Bt, se_t)
    assert abs(ob["geometric"] / est["B"] - 1) < 1e-6  # same draws, same geometric estimate
    # FP64 oracle chains: same estimator, fewer chains
    m, s = O.medium(sc.medium), O.source(sc.sources[0])
    d0, d1 = O.sensor(sc.sensors[0]), O.sensor(sc.sensors[1])
    T = O.ymap(s, d0, d1)
    n_or = 96
    chs = [O.Chains(sc.medium, sc.sources[0], sc.sensors[k], sc.run, n_or, cap, chain_offset=k * n_or)
           for k in (0, 1)]
    sums = [np.zeros(n_or), np.zeros(n_or)]
    for r in range(200):
        for k in (0, 1):
            chs[k].run(25)
        if r < 50:
            continue
        for k in (0, 1):
            for c in range(n_or):
                lr = O.ymap_logratio(m, s, d0, d1, T, k, chs[k].xyz[c, : chs[k].n[c]])
                sums[k][c] += math.exp(0.5 * lr) if np.isfinite(lr) else 0.0
    Bo, se_o = O.yield_ratio_estimate(sums[0], sums[1])
    assert abs(est["B"] - Bo) < 3 * math.hypot(est["se"], se_o), (est, Bo, se_o)


def test_yield_estimate_reduction_matches_host(api, ctx):
    """The device reduction of the per-chain sums equals the host formula."""
    import torch
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.5)
    sensors = [S.Sensor((0.0, 0.0, 1.5), 0.3), S.Sensor((1.0, 0.0, 1.0), 0.2)]
    sc = S.Scene("red", med, [S.Source()], sensors, [S.Pair(0, 0, 300, 16), S.Pair(0, 1, 517, 16)],
                 S.Run(seed=3, burn_in=0, sigma=0.1))
    est, ch = _run_yield(api, ctx, sc, 12, 10, 2)
    Y = api.YieldRatio(ch, 0, 1)
    rng = np.random.default_rng(8)
    vals = rng.uniform(0.1, 3.0, size=817)
    Y.sums.copy_(torch.from_numpy(vals))
    Y.n_obs = 7
    e = Y.estimate()
    a, b = vals[:300] / 7, vals[300:] / 7
    B = a.mean() / b.mean()
    se = B * math.sqrt(a.var(ddof=1) / 300 / a.mean() ** 2 + b.var(ddof=1) / 517 / b.mean() ** 2)
    assert abs(e["B"] - B) < 1e-12 * B and abs(e["se"] - se) < 1e-10 * se


def test_length_histogram_of_chain_states(api, ctx):
    import torch
    sc = S.plain(n_chains=2048, n_steps=3000, cap=64)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(3000)
    lo, hi, nb = 0.9, 2.5, 40
    hist = torch.zeros((1, nb), dtype=torch.float64, device="cuda")
    ch.length_hist(lo, hi, hist)
    ch.length_hist(lo, hi, hist)  # a second observation of the same states doubles every bin
    h = hist.cpu().numpy()[0]
    xyz, n, _ = ch.read_states()
    L = np.array([np.linalg.norm(np.diff(xyz[c, :, : n[c]].astype(np.float64), axis=1), axis=0).sum()
                  for c in range(len(n))])
    ref = 2.0 * np.histogram(L, bins=nb, range=(lo, hi))[0]
    edges = np.linspace(lo, hi, nb + 1)
    near = np.min(np.abs(L[:, None] - edges[None, :]), axis=1) < 1e-4
    assert np.abs(h - ref).sum() <= 2.0 * 2 * near.sum()
    assert h.sum() > 0.5 * 2 * len(n)


def test_tracer_length_histogram(api, ctx, oracle_lib):
    """GPU tracer's length histogram sums to its intensity and agrees bin by
    bin with the oracle tracer's (statistically)."""
    O = oracle_lib
    med, src, sen = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.5), S.Source(), S.Sensor((0.0, 0.0, 1.5), 0.5)
    medium = api.Medium(ctx, med)
    geom = api.Geometry(ctx, [src], [sen], [S.Pair(0, 0, 1, 32)])
    lo, hi, nb = 1.0, 6.0, 10
    g, hg = api.trace_lengths(ctx, medium, geom, 0, 21, 100_000_000, lo, hi, nb, max_scatter=30)
    go, hall = api.trace_lengths(ctx, medium, geom, 0, 21, 100_000_000, 0.0, 1e4, 4, max_scatter=30)
    assert abs(go["I"] - g["I"]) < 1e-9 * g["I"]  # same photons
    assert abs(hall.sum() - go["I"]) < 1e-9 * go["I"]  # every detected weight lands in a bin
    ref, hr = O.trace_lengths(O.medium(med), O.source(src), O.sensor(sen), 22, 4_000_000, lo, hi, nb,
                              max_scatter=30)
    assert abs(hg.sum() - g["I"]) < 0.2 * g["I"]
    # per-bin: weights w <= 1, so a bin's variance per photon is at most its mean
    for k in range(nb):
        se = math.sqrt(hg[k] / g["photons"] + hr[k] / ref["photons"])
        assert abs(hg[k] - hr[k]) < 4 * se + 1e-12, (k, hg[k], hr[k], se)


def test_bridge_ratio_matches_oracle_on_stored_logs(api, ctx, oracle_lib):
    """The device iteration equals the oracle's on identical stored log ratios."""
    import torch
    O = oracle_lib
    rng = np.random.default_rng(3)
    rows, n0, n1 = 64, 700, 500
    x0 = rng.normal(size=(rows, n0))
    x1 = 1.5 + 0.8 * rng.normal(size=(rows, n1))
    lq0 = lambda x: -0.5 * x * x  # noqa: E731
    lq1 = lambda x: math.log(2.0) - 0.5 * ((x - 1.5) / 0.8) ** 2  # noqa: E731
    L = np.concatenate([lq1(x0) - lq0(x0), lq0(x1) - lq1(x1)], axis=1).astype(np.float32)
    L[3, 5] = -np.inf  # a draw outside the other density's support
    g = api.bridge_ratio(ctx, torch.from_numpy(L).cuda(), n0, n1, groups=20, max_iter=300, tol=1e-12)
    r, se, it, geo = O.optimal_bridge(L[:, :n0].astype(np.float64), L[:, n0:].astype(np.float64), groups=20,
                                      max_iter=300, tol=1e-12)
    assert abs(g["r"] / r - 1) < 1e-9, (g, r)
    assert abs(g["geometric"] / geo - 1) < 1e-9
    assert abs(g["se"] / se - 1) < 1e-6
    assert abs(g["r"] - 1.6) < 4 * g["se"]


def test_chain_length_distribution_matches_tracer(api, ctx):
    """Section "Comparison of timing distributions" in miniature: the
    path-length distribution of tracer-seeded chains (observed every 25
    steps) equals the detected-weight distribution of the GPU tracer, both
    truncated at the chains' vertex cap."""
    import torch
    sc, _ = _two_sensor_scenes()["mini"]
    cap = 24
    sc.pairs = [S.Pair(0, 0, 4096, cap), S.Pair(0, 1, 4096, cap)]
    sc.run = S.Run(seed=17, burn_in=0, sigma=0.1)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    api.seed_from_tracer(ch, seed=99, photons_per_round=1 << 24)
    lo, hi, nb = 1.0, 9.0, 32
    hist = torch.zeros((2, nb), dtype=torch.float64, device="cuda")
    total = sum(p.n_chains for p in sc.pairs)
    centres = lo + (np.arange(nb) + 0.5) * (hi - lo) / nb
    # per chain: the bin centres of its observed lengths inside [lo, hi), the
    # same binned and clipped quantity as the tracer's histogram mean
    csum, ccnt = np.zeros(total), np.zeros(total)
    n_obs = 100
    for _ in range(n_obs):
        ch.run_steps(100)
        ch.length_hist(lo, hi, hist)
        xyz, n, _ = ch.read_states()
        seg = np.diff(xyz.astype(np.float64), axis=2)
        ln = np.sqrt((seg ** 2).sum(axis=1))
        mask = np.arange(ln.shape[1])[None, :] < (n[:, None] - 1)
        L = (ln * mask).sum(axis=1)
        inr = (L >= lo) & (L < hi)
        b = np.clip(((L - lo) / (hi - lo) * nb).astype(int), 0, nb - 1)
        csum += np.where(inr, centres[b], 0.0)
        ccnt += inr
    h = hist.cpu().numpy()
    c0 = 0
    for p, pr in enumerate(sc.pairs):
        tr, th = api.trace_lengths(ctx, medium, geom, p, 31 + p, 400_000_000, lo, hi, nb, max_scatter=cap - 2)
        # the chains' draws are dominated by their 4,096 independent seeds: errors across chains
        a = np.cumsum(h[p]) / h[p].sum()
        b = np.cumsum(th) / th.sum()
        assert np.abs(a - b).max() < 0.03, (p, np.abs(a - b).max())
        s_, c_ = csum[c0:c0 + pr.n_chains], ccnt[c0:c0 + pr.n_chains]
        c0 += pr.n_chains
        mc = s_.sum() / c_.sum()
        # ratio estimator over independent chains
        se_c = np.sqrt(((s_ - mc * c_) ** 2).sum() * len(c_) / (len(c_) - 1)) / c_.sum()
        mt = (centres * th).sum() / th.sum()           # binned tracer mean (0.25 m bins)
        assert abs(mc - mt) < 4 * se_c + 0.002, (p, mc, mt, se_c)


def test_score_observe_matches_per_path_scores(api, ctx):
    """pmc_score_observe sums, per pair, the per-layer scores of the chains'
    current paths: the same sums as pmc_score on those paths (read back and
    evaluated as a caller batch)."""
    import torch
    sc, _ = _two_sensor_scenes()["mini"]
    sc.pairs = [S.Pair(0, 0, 256, 24), S.Pair(0, 1, 300, 24)]
    sc.run = S.Run(seed=21, burn_in=0, sigma=0.1, init=S.INIT_STRAIGHT, init_k=4, init_jitter=0.05)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(500)
    nth = medium.n_theta
    sums = torch.zeros((2, 2 * nth), dtype=torch.float64, device="cuda")
    ch.score_observe(sums)
    got = sums.cpu().numpy()
    xyz, n, _ = ch.read_states()
    c0 = 0
    for p, pr in enumerate(sc.pairs):
        sl = slice(c0, c0 + pr.n_chains)
        c0 += pr.n_chains
        batch = np.ascontiguousarray(xyz[sl, :, :24].transpose(1, 0, 2))
        sco = api.score(ctx, medium, geom, p, torch.from_numpy(batch).cuda(),
                        torch.from_numpy(n[sl].astype(np.int32)).cuda()).cpu().numpy().astype(np.float64)
        ref = sco.sum(axis=0)
        assert np.allclose(got[p, :nth], ref, rtol=2e-3, atol=1e-3 * np.abs(sco).max()), (p, got[p, :nth], ref)
        assert np.allclose(got[p, nth:], (sco ** 2).sum(axis=0), rtol=5e-3, atol=1e-3 * (sco ** 2).max())
