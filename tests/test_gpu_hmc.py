"""GPU parity of the full-path gradient (HMC) move (section "Discussion")
with the FP64 oracle: the same Philox stream replays the oracle's
trajectories, tiny leapfrog steps are almost always accepted (the gradient
the kernel follows matches the density it accepts with), and the chains'
intensity equals the quadrature (vertex cap 3) and the forward tracer.
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


def _hmc_scene(name, steps=5):
    """Replay scenes.  The leapfrog step stays well inside the stable range of
    the dynamics: the curvature of log p grows like 1/l^2 for short segments
    (times ~300 for the forward-peaked phase function at g = 0.9), and where a
    kick overshoots, FP32 and FP64 trajectories separate chaotically.
    "iso": isotropic scattering, 1 m scattering length, eps = 5 mm;
    "general": the general-kernel scene (g = 0.9 SL/HG mixture), eps = 0.2 mm."""
    if name == "general":
        sc = S.general_small(n_chains=64, n_steps=300)
        sc.run.mala_step = 2e-4
    else:
        sc = S.Scene("iso", S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.0), [S.Source()],
                     [S.Sensor((0.0, 0.0, 1.5), 0.5)], [S.Pair(0, 0, 64, 24)],
                     S.Run(seed=4321, n_steps=300, burn_in=0, sigma=0.1))
        sc.run.mala_step = 5e-3
    sc.run.within = S.WITHIN_HMC
    sc.run.hmc_steps = steps
    sc.run.init = S.INIT_STRAIGHT
    sc.run.init_k = 6
    sc.run.init_jitter = 0.02
    return sc


def _stiff_length(sc):
    """Shortest segment for which a leapfrog step of size eps stays well
    inside the stable range.  Near a segment of length l the curvature of
    log p is about c / l^2, with c = 2 from the -2 log l factor plus
    3 g / (1 - g)^2 from the Henyey-Greenstein peak at forward angles; the
    leapfrog integrator is stable for eps * sqrt(c) / l < 2 and here it must
    stay at half that: l >= eps * sqrt(c).  Below it, FP32 and FP64
    trajectories separate exponentially within one move (seen at 5e-4 m on
    a 4 mm segment with eps = 5 mm)."""
    g = sc.medium.g
    return sc.run.mala_step * math.sqrt(2.0 + 3.0 * g / (1.0 - g) ** 2)


@pytest.mark.parametrize("name", ["iso", "general"])
def test_hmc_trajectory_replay(api, ctx, oracle_lib, name):
    """Same Philox stream on both sides.  Every chain whose decisions never
    came within 1e-3 of the threshold and whose leapfrog trajectories never
    met a segment shorter than the stiffness length (_stiff_length, from the
    oracle's own record of each trajectory) ends in the oracle's exact state
    and counts.  Chains below that length are excluded for a stated cause:
    there the FP32 and FP64 trajectories part legitimately."""
    O = oracle_lib
    sc = _hmc_scene(name)
    sc.run.n_steps = 150
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    assert ch.launch_info()[0]["general"] == 3
    ch.run_steps(sc.run.n_steps)
    xyz, n, st = ch.read_states()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, sc.pairs[0].cap)
    margin, shortest = oc.run(sc.run.n_steps, hmc_seg=True)
    l_stiff = _stiff_length(sc)
    clean = np.nonzero((margin > 1e-3) & (shortest >= l_stiff))[0]
    assert len(clean) >= 12, (len(clean), l_stiff)
    acc = ch.read_accumulators()
    oacc = oc.accumulators()
    parted = []
    for c in clean:
        k = int(n[c])
        if not (n[c] == oc.n[c] and np.allclose(xyz[c, :, :k].T, oc.xyz[c, :k], atol=2e-4)
                and np.array_equal(acc[c, 8:12], oacc["prop"][c]) and np.array_equal(acc[c, 12:16], oacc["acc"][c])):
            parted.append((int(c), float(shortest[c]), float(margin[c])))
    assert not parted, (l_stiff, len(clean), parted)
    # HMC proposals happen and are accepted
    assert oacc["prop"][:, 0].sum() > 0 and acc[:, 12].sum() > 0


def test_hmc_small_steps_conserve_energy(api, ctx):
    sc = _hmc_scene("general", steps=5)
    sc.pairs = [S.Pair(0, 0, 1024, 64)]
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(400)
    acc = ch.read_accumulators()
    assert acc[:, 12].sum() / acc[:, 8].sum() > 0.98


def test_hmc_single_scatter_sector(api, ctx):
    sc = S.plain(n_chains=4096, n_steps=20000, cap=3)
    sc.run.within = S.WITHIN_HMC
    sc.run.mala_step = 0.03
    sc.run.hmc_steps = 4
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    ch = api.Chains(ctx, medium, geom, sc.run)
    ch.run_steps(20000)
    e = ch.read_estimator()[0]
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(e["intensity"] - ref) < 3 * e["std_err"], (e["intensity"], e["std_err"], ref)
    assert e["rel_err"] < 0.005


def test_hmc_chains_match_tracer(api, ctx):
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.0)
    src, sen = S.Source(), S.Sensor((0.0, 0.0, 1.5), 0.5)
    cap = 24
    run = S.Run(seed=98, n_steps=30000, burn_in=3000, within=S.WITHIN_HMC, mala_step=0.08, hmc_steps=5, sigma=0.1)
    medium = api.Medium(ctx, med)
    geom = api.Geometry(ctx, [src], [sen], [S.Pair(0, 0, 4096, cap)])
    ch = api.Chains(ctx, medium, geom, run)
    ch.run_steps(run.n_steps)
    e = ch.read_estimator()[0]
    tr = api.trace(ctx, medium, geom, 0, 7, 400_000_000, max_scatter=cap - 2)
    assert abs(e["intensity"] - tr["I"]) < 3 * math.hypot(e["std_err"], tr["se"]), (e, tr)
    assert e["rel_err"] < 0.01
