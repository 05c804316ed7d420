"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: |delta log p| <= 1e-5 + 2e-6 n on identical states; intensities
within 3 combined standard errors and <= 1% relative; gradients within 1e-3
relative of the FP64 reference.
"""
import json
import math
import os

import numpy as np
import pytest

import quadrature as Q
from paper_1811_04156_gb300 import scenes as S

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def _oracle_objs(O, med, src, sen):
    return O.medium(med), O.source(src), O.sensor(sen)


def _fp32_floor(fun, path, src, rng, draws=4, ulps=4.0, factor=4.0):
    """Absolute error floor of an FP32 evaluation of fun (an FP64 oracle
    function of a path) at `path`: the device works on positions relative to
    the source, rounded to FP32, so every coordinate carries a relative error
    of about 2^-24.  The floor is `factor` times the largest change of fun over
    `draws` random perturbations of every relative coordinate by up to `ulps`
    FP32 units in the last place; components that cancel to a small value
    get this floor instead of a relative bound they cannot meet."""
    base = fun(path)
    rel = path - np.asarray(src, float)[None, :]
    worst = np.zeros_like(base)
    for _ in range(draws):
        d = rng.uniform(-1.0, 1.0, rel.shape) * ulps * 2.0 ** -24 * np.maximum(np.abs(rel), 1e-30)
        d[0] = 0.0  # the source itself is the frame origin: exact
        worst = np.maximum(worst, np.abs(fun(path + d) - base))
    return factor * worst


SCENES = {
    "plain": (S.Medium(lambda_s=0.5, lambda_a=5.0, g=0.9), S.Source(), S.Sensor((0.0, 0.0, 1.0), 0.1), 64, 0.3),
    "detector": (S.Medium(lambda_s=5.0, lambda_a=100.0, g=0.94), S.Source(), S.Sensor((0.0, 0.0, 50.0), 0.165),
                 256, 3.0),
    "vmf_rho_sl": (S.Medium(lambda_s=0.8, lambda_a=6.0, g=0.95, f_sl=0.45),
                   S.Source((0.3, -0.2, 0.1), S.EMIT_VMF, 38.0, (0.0, 0.0, 1.0)),
                   S.Sensor((0.5, 0.4, 3.0), 0.15, S.RHO_PAPER, (0.0, -1.0, 0.0)), 96, 0.4),
    "layered": (S.Medium(S.LAYERED, g=0.94, z0=-20.0, dz=2.0,
                         lambda_s_layers=5.0 * np.exp(0.3 * np.random.default_rng(5).normal(size=20)),
                         lambda_a_layers=100.0 * np.exp(0.3 * np.random.default_rng(6).normal(size=20))),
                S.Source((1.0, 0.0, -3.0)), S.Sensor((0.0, 2.0, 9.0), 0.165), 128, 1.5),
}


def _batch(name, batch=384, seed=7):
    """Random paths with n in [2, cap]; every third path has n in {2, 3} (edge cases)."""
    med, src, sen, cap, lateral = SCENES[name]
    xyz, n = S.random_paths(src.pos, sen.centre, sen.radius, batch, cap, 2, cap, seed, lateral=lateral)
    xs, ns = S.random_paths(src.pos, sen.centre, sen.radius, batch, cap, 2, 3, seed + 1, lateral=lateral)
    xyz[:, ::3, :] = xs[:, ::3, :]
    n[::3] = ns[::3]
    return med, src, sen, cap, xyz, n


@pytest.mark.parametrize("name", list(SCENES))
def test_logp_parity_identical_states(api, ctx, oracle_lib, name):
    import torch
    O = oracle_lib
    med, src, sen, cap, xyz, n = _batch(name)
    medium = api.Medium(ctx, med)
    geom = api.Geometry(ctx, [src], [sen], [S.Pair(0, 0, 1, cap)])
    lp = api.logp(ctx, medium, geom, 0, torch.from_numpy(xyz).cuda(), torch.from_numpy(n).cuda()).cpu().numpy()
    m, s, d = _oracle_objs(O, med, src, sen)
    n_fin = 0
    for b in range(len(n)):
        k = int(n[b])
        path = xyz[:, b, :k].T.astype(np.float64)
        ref = O.logp(m, s, d, path)
        if not np.isfinite(ref):
            assert lp[b] == -np.inf, (b, lp[b], ref)
            continue
        n_fin += 1
        tol = 1e-5 + 2e-6 * k
        assert abs(lp[b] - ref) <= tol, (name, b, k, lp[b], ref, lp[b] - ref)
    assert n_fin >= len(n) // 3


@pytest.mark.parametrize("name", list(SCENES))
def test_adjoint_parity(api, ctx, oracle_lib, name):
    import torch
    O = oracle_lib
    med, src, sen, cap, xyz, n = _batch(name, batch=128, seed=11)
    medium = api.Medium(ctx, med)
    geom = api.Geometry(ctx, [src], [sen], [S.Pair(0, 0, 1, cap)])
    xt = torch.from_numpy(xyz).cuda().requires_grad_(True)
    nt = torch.from_numpy(n).cuda()
    lp = api.LogP.apply(xt, nt, (ctx, medium, geom, 0))
    lp_f = torch.where(torch.isfinite(lp), lp, torch.zeros_like(lp))
    lp_f.sum().backward()
    g = xt.grad.cpu().numpy()
    m, s, d = _oracle_objs(O, med, src, sen)
    rng = np.random.default_rng(23)
    checked = 0
    for b in range(len(n)):
        k = int(n[b])
        path = xyz[:, b, :k].T.astype(np.float64)
        ref_lp, ref = O.grad_logp(m, s, d, path)
        if not np.isfinite(ref_lp):
            continue
        floor = _fp32_floor(lambda f: O.grad_logp(m, s, d, f)[1], path, src.pos, rng)
        mine = g[:, b, :k].T
        # every component: 1e-3 relative, plus the FP32 rounding floor
        bad = np.abs(mine - ref) > 1e-3 * np.abs(ref) + floor
        assert not bad.any(), (name, b, k, np.argwhere(bad)[:4].tolist(), mine[bad][:4], ref[bad][:4], floor[bad][:4])
        assert np.all(g[:, b, k:] == 0)
        checked += 1
    assert checked >= 20


@pytest.mark.parametrize("name", ["plain", "detector", "layered"])
def test_score_parity(api, ctx, oracle_lib, name):
    import torch
    O = oracle_lib
    med, src, sen, cap, xyz, n = _batch(name, batch=128, seed=13)
    medium = api.Medium(ctx, med)
    geom = api.Geometry(ctx, [src], [sen], [S.Pair(0, 0, 1, cap)])
    sc = api.score(ctx, medium, geom, 0, torch.from_numpy(xyz).cuda(), torch.from_numpy(n).cuda()).cpu().numpy()
    m, s, d = _oracle_objs(O, med, src, sen)
    rng = np.random.default_rng(29)
    checked = 0
    for b in range(len(n)):
        k = int(n[b])
        path = xyz[:, b, :k].T.astype(np.float64)
        ref = O.score(m, s, d, path)
        if not np.isfinite(O.logp(m, s, d, path)):
            continue
        floor = _fp32_floor(lambda f: O.score(m, s, d, f), path, src.pos, rng)
        # every parameter: 1e-3 relative, plus the FP32 rounding floor
        bad = np.abs(sc[b] - ref) > 1e-3 * np.abs(ref) + floor
        assert not bad.any(), (name, b, k, np.nonzero(bad)[0][:4].tolist(), sc[b][bad][:4], ref[bad][:4],
                               floor[bad][:4])
        checked += 1
    assert checked >= 20


def _plain_sampler(api, ctx, n_chains, n_steps, cap=64, flags=0, seed=None, within=S.WITHIN_PERTURB):
    sc = S.plain(n_chains=n_chains, n_steps=n_steps, cap=cap)
    if seed is not None:
        sc.run.seed = seed
    sc.run.within = within
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    return sc, medium, geom, api.Chains(ctx, medium, geom, sc.run, flags=flags)


@pytest.mark.parametrize("flags", [0, 2])
def test_trajectory_replay(api, ctx, oracle_lib, flags):
    """Same Philox stream on both sides: every chain whose decisions never came
    within 1e-3 of the threshold ends in the oracle's state."""
    O = oracle_lib
    steps = 400
    sc, medium, geom, ch = _plain_sampler(api, ctx, 64, steps, flags=flags)
    ch.run_steps(steps)
    xyz, n, st = ch.read_states()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 64)
    margin = oc.run(steps, margins=True)
    assert np.all(st == steps)
    clean = margin > 1e-3
    assert clean.sum() >= 40
    for c in np.nonzero(clean)[0]:
        assert n[c] == oc.n[c], (c, n[c], oc.n[c])
        k = int(n[c])
        assert np.allclose(xyz[c, :, :k].T, oc.xyz[c, :k], atol=2e-4), c
    acc = ch.read_accumulators()
    oacc = oc.accumulators()
    for c in np.nonzero(clean)[0]:
        assert np.array_equal(acc[c, 8:12], oacc["prop"][c])
        assert np.array_equal(acc[c, 12:16], oacc["acc"][c])


def test_split_runs_and_checkpoint_are_bit_exact(api, ctx):
    _, _, _, a = _plain_sampler(api, ctx, 256, 0)
    _, _, _, b = _plain_sampler(api, ctx, 256, 0)
    a.run_steps(1500)
    b.run_steps(500)
    blob = b.save_state()
    b.run_steps(1000)
    xa, na, sa = a.read_states()
    xb, nb, sb = b.read_states()
    assert np.array_equal(na, nb) and np.array_equal(xa, xb) and np.array_equal(sa, sb)
    aa, ab = a.read_accumulators(), b.read_accumulators()
    assert np.array_equal(aa[:, 8:], ab[:, 8:])          # proposal / acceptance counts
    # FP32 partial sums are flushed into the FP64 words at other points
    scale = np.abs(aa[:, :8]).max(axis=0) + 1.0
    assert np.all(np.abs(aa[:, :8] - ab[:, :8]) <= 1e-5 * scale)
    b.load_state(blob)
    b.run_steps(1000)
    xc, nc_, _ = b.read_states()
    assert np.array_equal(xa, xc) and np.array_equal(na, nc_)


def test_intensity_single_scatter_sector(api, ctx):
    sc, medium, geom, ch = _plain_sampler(api, ctx, 4096, 20000, cap=3)
    ch.run_steps(20000)
    e = ch.read_estimator()[0]
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(e["z2"] / Q.z2_closed(1.0, 0.1, 2.2) - 1) < 1e-5
    assert abs(e["intensity"] - ref) < 3 * e["std_err"], (e["intensity"], e["std_err"], ref)
    assert e["rel_err"] < 0.003


def test_intensity_matches_oracle_plain(api, ctx):
    g = json.load(open(os.path.join(GOLDEN, "plain_intensity.json")))
    sc, medium, geom, ch = _plain_sampler(api, ctx, g["n_chains"], g["n_steps"], seed=g["seed"])
    assert sc.run.burn_in == g["burn_in"]
    ch.run_steps(g["n_steps"])
    e = ch.read_estimator()[0]
    diff = abs(e["intensity"] - g["intensity"])
    assert diff < 3 * math.hypot(e["std_err"], g["std_err"]), (e, g)
    assert diff < 0.01 * g["intensity"]
    assert abs(e["mean_n"] / g["mean_n"] - 1) < 0.01


def test_mala_single_scatter_sector(api, ctx):
    sc, medium, geom, ch = _plain_sampler(api, ctx, 4096, 20000, cap=3, within=S.WITHIN_MALA)
    ch.run_steps(20000)
    e = ch.read_estimator()[0]
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(e["intensity"] - ref) < 3 * e["std_err"], (e["intensity"], e["std_err"], ref)


def test_gpu_tracer_matches_oracle_tracer(api, ctx, oracle_lib):
    O = oracle_lib
    med, src, sen = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.6), S.Source(), S.Sensor((0.0, 0.0, 1.5), 0.5)
    medium = api.Medium(ctx, med)
    geom = api.Geometry(ctx, [src], [sen], [S.Pair(0, 0, 1, 32)])
    gt = api.trace(ctx, medium, geom, 0, 4242, 200_000_000, max_scatter=30)
    m, s, d = _oracle_objs(O, med, src, sen)
    ot = O.trace(m, s, d, 4242, 4_000_000, max_scatter=30)
    assert abs(gt["I"] - ot["I"]) < 3 * math.hypot(gt["se"], ot["se"])
    # without scattering the tracer reproduces the closed form
    med0 = S.Medium(lambda_s=1e9, lambda_a=2.0)
    g0 = api.trace(ctx, api.Medium(ctx, med0), geom, 0, 5, 100_000_000, max_scatter=0)
    assert abs(g0["I"] - Q.z2_closed(1.5, 0.5, 0.5 + 1e-9)) < 3 * g0["se"]


def test_abort_request_stops_and_context_survives(api, ctx):
    from paper_1811_04156_gb300._lib import PathmcError
    _, _, _, ch = _plain_sampler(api, ctx, 128, 0)
    ch.request_abort(True)
    ch.run_steps(5000)
    with pytest.raises(PathmcError) as ei:
        ch.read_estimator()
    assert ei.value.code == 5
    ch.request_abort(False)
    _, _, _, ch2 = _plain_sampler(api, ctx, 128, 0)
    ch2.run_steps(2000)
    assert ch2.read_estimator()[0]["n_samples"] > 0


@pytest.mark.parametrize("layout,within", [(S.LAYOUT_WARP, S.WITHIN_PERTURB), (S.LAYOUT_LANE, S.WITHIN_PERTURB),
                                           (S.LAYOUT_LANE, S.WITHIN_TREE)])
def test_abort_mid_run_stops_at_a_poll(api, ctx, layout, within):
    """pmc_request_abort from the host while a long pmc_run_steps executes:
    the kernels poll the flag every 1,024 steps, so the run ends long before
    its steps are done; the next synchronising call reports PMC_ERR_ABORTED,
    every chain stopped at a poll boundary with consistent bookkeeping, and
    the context then runs a new chain set.  With tree moves on the lane
    layout the warp stops as a whole (its pooled passes need every lane)."""
    import time
    import torch
    from paper_1811_04156_gb300._lib import PathmcError
    sc = S.plain(n_chains=65536, n_steps=0)
    sc.run.layout = layout
    sc.run.within = within
    if within == S.WITHIN_TREE:
        sc.run.sigma = 0.5
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(1024)
    ch.read_estimator()
    t = time.perf_counter()
    ch.run_steps(4096)
    ch.read_estimator()
    per_step = (time.perf_counter() - t) / 4096
    n_long = int(round(6.0 / per_step / 1024)) * 1024          # about 6 s of stepping
    ch.run_steps(n_long)                                          # asynchronous: enqueue only
    time.sleep(0.3)
    ch.request_abort(True)
    t0 = time.perf_counter()
    with pytest.raises(PathmcError) as ei:
        ch.read_estimator()
    waited = time.perf_counter() - t0
    assert ei.value.code == 5
    assert waited < 2.0, (waited, n_long, per_step)
    ch.request_abort(False)
    xyz, n, steps = ch.read_states()
    done = steps.astype(np.int64) - 5120
    # a chain stops at a poll (a multiple of 1,024 steps into the launch); with
    # one warp per chain the first wave of chains may have finished already
    assert np.all(done >= 0) and np.all(done <= n_long) and np.all(done % 1024 == 0), np.unique(done)[:8]
    assert done.max() > 0                                          # the long run had started
    assert (done < n_long).mean() > 0.5                            # and most chains stopped early
    assert np.all((n >= 2) & (n <= 64)) and np.all(np.isfinite(xyz))
    acc = ch.read_accumulators()
    assert np.array_equal(acc[:, 8:12].sum(axis=1), steps.astype(np.float64))
    # the context is still usable: a new chain set runs and reads cleanly
    _, _, _, ch2 = _plain_sampler(api, ctx, 128, 0)
    ch2.run_steps(2000)
    assert ch2.read_estimator()[0]["n_samples"] > 0
    torch.cuda.synchronize()


def test_batched_uneven_pairs(api, ctx):
    """One chain set over six pairs in three vertex-cap classes: the cap-3 pairs
    match the single-scatter quadrature, the long pairs the oracle."""
    sc = S.batched_small()
    g = json.load(open(os.path.join(GOLDEN, "batched_small_intensity.json")))
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(sc.run.n_steps)
    est = ch.read_estimator()
    assert ch.status() == 0
    xyz, n, steps = ch.read_states()
    caps = np.repeat([p.cap for p in sc.pairs], [p.n_chains for p in sc.pairs])
    assert np.all((n >= 2) & (n <= caps)) and np.all(steps == sc.run.n_steps)
    for i, (p, e) in enumerate(zip(sc.pairs, est)):
        assert sum(e["proposals"]) == p.n_chains * sc.run.n_steps
        D = float(np.linalg.norm(sc.sensors[p.sensor].centre))
        if p.cap == 3:
            ref = Q.z2_closed(D, 0.3, 2.2) + Q.z3(D, 0.3, 0.5, 5.0, 0.9)
            assert abs(e["intensity"] - ref) < 3 * e["std_err"], (i, e["intensity"], e["std_err"], ref)
        else:
            o = g["pairs"][str(i)]
            assert abs(e["intensity"] - o["intensity"]) < 3 * math.hypot(e["std_err"], o["std_err"]), (i, e, o)
            assert abs(e["mean_n"] / o["mean_n"] - 1) < 0.03


def test_general_kernel_trajectory_replay(api, ctx, oracle_lib):
    """Layered medium, vMF emission, detection probability and the SL mixture
    (the general kernel) replay the oracle's trajectories."""
    O = oracle_lib
    sc = S.general_small()
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(sc.run.n_steps)
    xyz, n, _ = ch.read_states()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 64)
    margin = oc.run(sc.run.n_steps, margins=True)
    clean = margin > 1e-3
    assert clean.sum() >= 32
    for c in np.nonzero(clean)[0]:
        assert n[c] == oc.n[c], (c, n[c], oc.n[c])
        k = int(n[c])
        assert np.allclose(xyz[c, :, :k].T, oc.xyz[c, :k], atol=2e-4), c
    # the general kernel keeps every state's density finite
    import torch
    lp = api.logp(ctx, medium, geom, 0, torch.from_numpy(np.ascontiguousarray(xyz.transpose(1, 0, 2))).cuda(),
                  torch.from_numpy(n).cuda()).cpu().numpy()
    assert np.all(np.isfinite(lp))


def test_gradient_estimator_fd_and_fp64(api, ctx, oracle_lib):
    """Score-function gradients of the intensity (MALA chains): the per-state
    scores match the FP64 oracle, central finite differences of the density at
    h = 1e-3 relative on common samples, and the accumulated estimator."""
    import copy
    import torch
    O = oracle_lib
    sc = S.gradients(n_chains=16384, n_steps=4000)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(sc.run.n_steps)
    grad, grad_se = ch.grad_estimator()
    e = ch.read_estimator()[0]
    xyz, n, _ = ch.read_states()
    xt = torch.from_numpy(np.ascontiguousarray(xyz.transpose(1, 0, 2))).cuda()
    nt = torch.from_numpy(n).cuda()
    sc_gpu = api.score(ctx, medium, geom, 0, xt, nt).cpu().numpy().astype(np.float64)
    # FP64 reference on the same states
    m, s, d = O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[0])
    rng = np.random.default_rng(31)
    for c in range(0, len(n), 64):
        path = xyz[c, :, : n[c]].T.astype(np.float64)
        ref = O.score(m, s, d, path)
        floor = _fp32_floor(lambda f: O.score(m, s, d, f), path, sc.sources[0].pos, rng)
        assert np.all(np.abs(sc_gpu[c] - ref) <= 1e-3 * np.abs(ref) + floor), (c, sc_gpu[c], ref, floor)
    # central differences of log p at theta (1 +- 1e-3) on the same states
    lp0 = api.logp(ctx, medium, geom, 0, xt, nt).cpu().numpy().astype(np.float64)
    for i, name in enumerate(("lambda_s", "lambda_a", "g")):
        v = getattr(sc.medium, name)
        h = 1e-3 * v
        ratios = []
        for sgn in (+1, -1):
            mm = copy.deepcopy(sc.medium)
            setattr(mm, name, v + sgn * h)
            lp = api.logp(ctx, api.Medium(ctx, mm), geom, 0, xt, nt).cpu().numpy().astype(np.float64)
            ratios.append(np.exp(lp - lp0))
        fd = (ratios[0] - ratios[1]) / (2 * h)
        assert abs(fd.mean() - sc_gpu[:, i].mean()) <= 1e-3 * np.abs(sc_gpu[:, i]).mean(), (name, fd.mean(),
                                                                                            sc_gpu[:, i].mean())
    # the reduction formula: grad = I * E[score], E[score] from the raw
    # accumulators (the comparison with the oracle's own chains is
    # test_grad_estimator_matches_oracle_chains)
    acc = ch.read_accumulators()
    N = acc[:, 0].sum()
    ls, la = sc.medium.lambda_s, sc.medium.lambda_a
    es = np.array([(acc[:, 3].sum() / ls ** 2 - (acc[:, 2].sum() - 2 * N) / ls) / N,
                   acc[:, 3].sum() / la ** 2 / N, acc[:, 5].sum() / N])
    assert np.allclose(grad[0], e["intensity"] * es, rtol=1e-9)
    assert np.all(grad_se[0] > 0)


def _jackknife(est, n_items, groups=32):
    """Grouped jackknife standard error of est(mask) over items mod groups."""
    full = est(np.ones(n_items, bool))
    g = np.arange(n_items) % groups
    jk = np.array([est(g != k) for k in range(groups)])
    return full, np.sqrt((groups - 1) / groups * ((jk - jk.mean(axis=0)) ** 2).sum(axis=0))


@pytest.mark.parametrize("layout", [S.LAYOUT_WARP, S.LAYOUT_LANE])
def test_grad_estimator_matches_oracle_chains(api, ctx, oracle_lib, layout):
    """pmc_grad_estimator on MALA chains of the gradients workload's geometry
    against the FP64 oracle's own chains on the same Philox stream: the
    oracle's estimate is I * E_p[score] with I = Z2 / pi(n = 2) and E_p[score]
    the mean of its per-state FP64 scores (d log p / d lambda_s, lambda_a, g),
    its standard error a grouped jackknife over chains.  Each component agrees
    within 1e-3 relative or 3 combined standard errors (FP32 and FP64 chains
    part after a near-threshold decision, so the agreement is statistical)."""
    O = oracle_lib
    n_chains, n_steps = 1024, 20_000
    sc = S.gradients(n_chains=n_chains, n_steps=n_steps)
    sc.run.layout = layout
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(n_steps)
    grad, grad_se = ch.grad_estimator()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, n_chains, sc.pairs[0].cap)
    oc.run(n_steps)
    acc = oc.accumulators()
    z2 = O.z2(O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[0]))

    def est(mask):
        sub = {k: v[mask] for k, v in acc.items()}
        I, _, _ = O.direct_estimate(sub, z2)
        return I * sub["sum_score"].sum(axis=0) / sub["n_rec"].sum()

    ref, ref_se = _jackknife(est, n_chains)
    for i in range(3):
        diff = abs(grad[0, i] - ref[i])
        assert diff <= max(1e-3 * abs(ref[i]), 3 * math.hypot(grad_se[0, i], ref_se[i])), \
            (i, grad[0, i], grad_se[0, i], ref[i], ref_se[i])
    # the standard errors describe the same spread
    assert np.all(grad_se[0] < 3 * ref_se) and np.all(ref_se < 3 * grad_se[0]), (grad_se[0], ref_se)


def test_accumulators_replay_oracle(api, ctx, oracle_lib):
    """MALA chains with gradients: for every chain whose decisions stayed away
    from the threshold, the FP64 accumulators (recorded states, n = 2 count,
    sums of n, L, L^2 and d log sigma/dg, proposals, acceptances) equal the
    oracle's."""
    O = oracle_lib
    sc = S.gradients(n_chains=64, n_steps=600)
    sc.run.burn_in = 100
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(sc.run.n_steps)
    acc = ch.read_accumulators()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 64)
    margin = oc.run(sc.run.n_steps, margins=True)
    oa = oc.accumulators()
    clean = np.nonzero(margin > 1e-3)[0]
    assert len(clean) >= 32
    for c in clean:
        assert acc[c, 0] == oa["n_rec"][c] and acc[c, 1] == oa["n_direct"][c] and acc[c, 2] == oa["sum_n"][c]
        assert abs(acc[c, 3] / oa["sum_L"][c] - 1) < 1e-5
        assert abs(acc[c, 4] / oa["sum_L2"][c] - 1) < 1e-5
        # gradient tolerance (1e-3 relative): per-vertex d log sigma / dg terms are large and cancel,
        # and the running sum is kept in FP32 between exact refreshes
        assert abs(acc[c, 5] - oa["sum_score"][c, 2]) < 1e-3 * (abs(oa["sum_score"][c, 2]) + oa["n_rec"][c])
        assert np.array_equal(acc[c, 8:12], oa["prop"][c]) and np.array_equal(acc[c, 12:16], oa["acc"][c])


@pytest.mark.parametrize("name", ["plain", "layered", "vmf_rho_sl"])
def test_reference_density_parity(api, ctx, oracle_lib, name):
    """log q_ref of identical states against the oracle."""
    import torch
    O = oracle_lib
    med, src, sen, cap, xyz, n = _batch(name, batch=256, seed=17)
    medium = api.Medium(ctx, med)
    geom = api.Geometry(ctx, [src], [sen], [S.Pair(0, 0, 1, cap)])
    lq = api.qref_logdensity(ctx, medium, geom, 0, torch.from_numpy(xyz).cuda(),
                             torch.from_numpy(n).cuda()).cpu().numpy()
    m, s, d = _oracle_objs(O, med, src, sen)
    fin = 0
    for b in range(len(n)):
        k = int(n[b])
        ref = O.qref_logdensity(m, s, d, cap, xyz[:, b, :k].T.astype(np.float64))
        if not np.isfinite(ref):
            assert lq[b] == -np.inf
            continue
        fin += 1
        assert abs(lq[b] - ref) <= 1e-5 + 2e-6 * k + 2e-6 * abs(ref), (name, b, k, lq[b], ref)
    assert fin >= len(n) // 4


def test_reference_draws_match_oracle(api, ctx, oracle_lib):
    """Same Philox counters: the GPU draws the oracle's reference paths."""
    O = oracle_lib
    sc = S.plain(cap=64)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    xyz, n = api.qref_sample(ctx, medium, geom, 0, 99, 512)
    xyz, n = xyz.cpu().numpy(), n.cpu().numpy()
    m, s, d = _oracle_objs(O, sc.medium, sc.sources[0], sc.sensors[0])
    same = 0
    for q in range(512):
        ref = O.qref_sample(m, s, d, 64, 99, 0, q)
        if len(ref) != n[q]:
            continue
        same += 1
        assert np.allclose(xyz[:, q, : n[q]].T, ref, atol=1e-4, rtol=1e-4), q
    assert same >= 500


def test_bridge_intensity_single_scatter(api, ctx):
    """The bridge with the reference density estimates Z2 + Z3 at cap 3."""
    sc, medium, geom, ch = _plain_sampler(api, ctx, 4096, 20000, cap=3)
    ch.run_steps(20000)
    I, se = ch.bridge(4_000_000, seed=5)[0]
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(I - ref) < 3 * se, (I, se, ref)
    assert se / I < 0.02


def test_optimal_bridge_intensity_single_scatter(api, ctx, oracle_lib):
    """The optimal (Meng & Wong) bridge against the normalised reference
    density estimates Z2 + Z3 at cap 3 from per-observation log ratios, and
    the device iteration equals the oracle's on the same stored rows."""
    import torch
    O = oracle_lib
    sc, medium, geom, ch = _plain_sampler(api, ctx, 4096, 20000, cap=3)
    ch.run_steps(2000)
    n_draws, rows = 4096, 60
    logr = torch.zeros((rows, n_draws + 4096), dtype=torch.float32, device="cuda")
    for r in range(rows):
        ch.run_steps(100)
        ch.bridge_observe_log(0, n_draws, r * n_draws, 11, logr[r])
    ob = api.bridge_ratio(ctx, logr, n_draws, 4096, groups=32)
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(ob["r"] - ref) < 3 * ob["se"], (ob, ref)
    assert ob["se"] / ob["r"] < 0.01
    L = logr.cpu().numpy().astype(np.float64)
    r, se, it, geo = O.optimal_bridge(L[:, :n_draws], L[:, n_draws:], groups=32)
    assert abs(ob["r"] / r - 1) < 1e-9 and abs(ob["geometric"] / geo - 1) < 1e-9


def _layered_small(n_chains, n_steps, cap):
    rng = np.random.default_rng(31)
    med = S.Medium(S.LAYERED, g=0.9, z0=-1.0, dz=0.4, lambda_s_layers=0.6 * np.exp(0.3 * rng.normal(size=8)),
                   lambda_a_layers=5.0 * np.exp(0.3 * rng.normal(size=8)))
    run = S.Run(seed=77, n_steps=n_steps, burn_in=n_steps // 10, sigma=0.05)
    return S.Scene("layered_small", med, [S.Source((0.0, 0.0, -0.4))], [S.Sensor((0.3, 0.0, 0.6), 0.2)],
                   [S.Pair(0, 0, n_chains, cap)], run)


def test_layered_intensity_matches_oracle(api, ctx, oracle_lib):
    """Layered medium: the direct-sector integral and the cap-3 intensity of the
    general kernel agree with the oracle's."""
    O = oracle_lib
    sc = _layered_small(4096, 20000, 3)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(sc.run.n_steps)
    e = ch.read_estimator()[0]
    m, s, d = _oracle_objs(O, sc.medium, sc.sources[0], sc.sensors[0])
    assert abs(e["z2"] / O.z2(m, s, d) - 1) < 1e-5
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 256, 3)
    oc.run(sc.run.n_steps)
    I, se, _ = O.direct_estimate(oc.accumulators(), O.z2(m, s, d))
    assert abs(e["intensity"] - I) < 3 * math.hypot(se, e["std_err"]), (e["intensity"], e["std_err"], I, se)


def test_layered_gradients(api, ctx, oracle_lib):
    """Per-layer score-function gradients (2L parameters): the estimator equals
    I times the mean per-state score of pmc_score, whose every component
    matches the FP64 oracle on the chains' own states; the estimate agrees
    with the one the oracle's FP64 chains give on the same Philox stream; and
    the mean score matches central finite differences of the density at
    h = 1e-3."""
    import copy
    import torch
    O = oracle_lib
    sc = _layered_small(8192, 4000, 64)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(sc.run.n_steps)
    grad, grad_se = ch.grad_estimator()
    I = ch.read_estimator()[0]["intensity"]
    xyz, n, _ = ch.read_states()
    xt = torch.from_numpy(np.ascontiguousarray(xyz.transpose(1, 0, 2))).cuda()
    nt = torch.from_numpy(n).cuda()
    scr = api.score(ctx, medium, geom, 0, xt, nt).cpu().numpy().astype(np.float64)
    scale = np.abs(scr.mean(axis=0)).max()
    assert np.all(np.abs(grad[0] / I - scr.mean(axis=0)) <= 1e-4 * scale)
    varies = scr.std(axis=0) > 0          # layers no path enters have a zero score and zero SE
    assert np.all(grad_se[0][varies] > 0) and np.all(grad_se[0] >= 0)
    m, s, d = _oracle_objs(O, sc.medium, sc.sources[0], sc.sensors[0])
    rng = np.random.default_rng(37)
    # every per-layer score of every 32nd state: 1e-3 relative plus the FP32 rounding floor
    for c in range(0, len(n), 32):
        path = xyz[c, :, : n[c]].T.astype(np.float64)
        ref = O.score(m, s, d, path)
        floor = _fp32_floor(lambda f: O.score(m, s, d, f), path, sc.sources[0].pos, rng)
        bad = np.abs(scr[c] - ref) > 1e-3 * np.abs(ref) + floor
        assert not bad.any(), (c, int(n[c]), np.nonzero(bad)[0][:4].tolist(), scr[c][bad][:4], ref[bad][:4])
    # the estimate against the FP64 oracle's own chains on the same Philox stream:
    # I * E_p[score] over their final states, jackknife standard error over chains
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, len(n), sc.pairs[0].cap)
    oc.run(sc.run.n_steps)
    acc = oc.accumulators()
    oscr = np.array([O.score(m, s, d, oc.xyz[c, : oc.n[c]]) for c in range(len(n))])
    z2 = O.z2(m, s, d)

    def est(mask):
        I_o, _, _ = O.direct_estimate({k: v[mask] for k, v in acc.items()}, z2)
        return I_o * oscr[mask].mean(axis=0)

    ref, ref_se = _jackknife(est, len(n))
    tol = np.maximum(1e-3 * np.abs(ref), 3 * np.hypot(grad_se[0], ref_se))
    assert np.all(np.abs(grad[0] - ref) <= tol), (grad[0], grad_se[0], ref, ref_se)
    assert np.count_nonzero(ref) >= sc.medium.n_layers     # the comparison covers the layers paths enter
    lp0 = api.logp(ctx, medium, geom, 0, xt, nt).cpu().numpy().astype(np.float64)
    L = sc.medium.n_layers
    for j in (2, 3, L + 2):
        arr = "lambda_s_layers" if j < L else "lambda_a_layers"
        v = getattr(sc.medium, arr)[j % L]
        h = 1e-3 * v
        ratios = []
        for sgn in (+1, -1):
            mm = copy.deepcopy(sc.medium)
            getattr(mm, arr)[j % L] = v + sgn * h
            lp = api.logp(ctx, api.Medium(ctx, mm), geom, 0, xt, nt).cpu().numpy().astype(np.float64)
            ratios.append(np.exp(lp - lp0))
        fd = ((ratios[0] - ratios[1]) / (2 * h)).mean()
        assert abs(fd - scr[:, j].mean()) <= 1e-3 * scale, (j, fd, scr[:, j].mean())


def test_tracer_seeds_are_exact_draws(api, ctx, oracle_lib):
    """Weight-thinned detected tracer paths at cap 3: the share of n = 2 paths
    is Z2 / (Z2 + Z3) (independent quadrature), and every seed is a valid state."""
    import torch
    O = oracle_lib
    sc = S.plain(cap=3)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    xyz, n, acc = api.trace_paths(ctx, medium, geom, 0, 11, 400_000_000, 200_000)
    assert acc >= 200_000 and len(n) == 200_000
    n = n.cpu().numpy()
    z2 = Q.z2_closed(1.0, 0.1, 2.2)
    frac = z2 / (z2 + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9))
    se = math.sqrt(frac * (1 - frac) / len(n))
    assert abs((n == 2).mean() - frac) < 4 * se, ((n == 2).mean(), frac, se)
    lp = api.logp(ctx, medium, geom, 0, xyz.contiguous(), torch.from_numpy(n).cuda()).cpu().numpy()
    assert np.all(np.isfinite(lp))
    m, s, d = _oracle_objs(O, sc.medium, sc.sources[0], sc.sensors[0])
    X = xyz.cpu().numpy()
    for q in range(0, 2000, 97):
        assert np.isfinite(O.logp(m, s, d, X[:, q, : n[q]].T.astype(np.float64)))


def test_seed_from_tracer_takes_the_first_accepted_photons(api, ctx):
    """pmc_seed_from_tracer: a first round far too large for the index buffer
    is traced again with fewer photons; every seed is an accepted path of the
    traced photon range (the same paths pmc_trace_paths keeps), the seeding is
    deterministic, and at vertex cap 3 the share of direct (n = 2) seeds is
    Z2 / (Z2 + Z3) of the independent quadrature."""
    sc = S.plain(n_chains=4096, n_steps=0, cap=3)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    used = api.seed_from_tracer(ch, seed=77, photons_per_round=1 << 26)
    xyz, n, steps = ch.read_states()
    assert np.all(steps == 0) and ch.status() == 0 and set(np.unique(n)) <= {2, 3}
    X, N, acc = api.trace_paths(ctx, medium, geom, 0, 77, used[0], max_paths=3 * 4096, max_scatter=1)
    assert 4096 <= acc <= 3 * 4096
    X, N = X.cpu().numpy(), N.cpu().numpy()
    found = {tuple(X[:, q, : N[q]].T.ravel().tolist()) for q in range(len(N))}
    assert all(tuple(xyz[c, :, : n[c]].T.ravel().tolist()) in found for c in range(4096))
    ch2 = api.Chains(ctx, medium, geom, sc.run)
    assert api.seed_from_tracer(ch2, seed=77, photons_per_round=1 << 26) == used
    assert np.array_equal(ch2.read_states()[0], xyz)
    z2 = Q.z2_closed(1.0, 0.1, 2.2)
    frac = z2 / (z2 + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9))
    se = math.sqrt(frac * (1 - frac) / 4096)
    assert abs((n == 2).mean() - frac) < 4 * se, ((n == 2).mean(), frac, se)


def test_tracer_seeded_chains_are_unbiased(api, ctx):
    """Chains started from tracer seeds are stationary from the first step: a
    short run agrees with a long forward-tracer reference to <= 1 %."""
    sc = S.plain(n_chains=16384, n_steps=3000, cap=64)
    sc.run.burn_in = 0
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    api.seed_from_tracer(ch, seed=21)
    ch.run_steps(sc.run.n_steps)
    e = ch.read_estimator()[0]
    ref = api.trace(ctx, medium, api.Geometry(ctx, sc.sources, sc.sensors, [S.Pair(0, 0, 1, 64)]), 0, 777,
                    2_000_000_000, max_scatter=62)
    diff = abs(e["intensity"] - ref["I"])
    assert diff < 3 * math.hypot(e["std_err"], ref["se"]), (e["intensity"], e["std_err"], ref["I"], ref["se"])
    assert diff < 0.01 * ref["I"]


@pytest.mark.parametrize("window", [32, 64])
def test_shared_window_spill_replays_oracle(api, ctx, oracle_lib, window):
    """Paths longer than the shared-memory window (entries beyond it in global
    memory) replay the oracle's trajectories."""
    O = oracle_lib
    # deaths outnumber births in this medium: after 100 steps most paths are
    # still longer than the window, after 300 few are
    sc = S.plain(n_chains=64, n_steps=100, cap=128)
    sc.medium.lambda_s = 0.05
    sc.run.init = S.INIT_STRAIGHT
    sc.run.init_k = window + 16
    sc.run.init_jitter = 0.002  # keeps every initial vertex outside the sensor ball
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run, warps_per_block=2, smem_window=window)
    assert ch.launch_info()[0]["smem_cap"] == window
    ch.run_steps(sc.run.n_steps)
    assert ch.status() == 0
    xyz, n, _ = ch.read_states()
    assert (n > window).sum() >= 16
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 128)
    margin = oc.run(sc.run.n_steps, margins=True)
    clean = np.nonzero(margin > 1e-3)[0]
    assert len(clean) >= 24
    for c in clean:
        assert n[c] == oc.n[c], (c, n[c], oc.n[c])
        k = int(n[c])
        assert np.allclose(xyz[c, :, :k].T, oc.xyz[c, :k], atol=2e-4), c
