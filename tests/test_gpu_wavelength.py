"""GPU parity of the wavelength sampled with the path (section "Discussion":
a wavelength parameter added to the path density and sampled along with the
vertices): the same Philox stream replays the oracle's (path, wavelength)
trajectories; at vertex cap 3 the intensity and the wavelength marginal match
the spectrum integral of the independent single-scatter quadrature; the
spectrum-weighted direct sector matches the oracle's; runs split or
checkpointed replay exactly; unsupported combinations are refused."""
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


def _spectrum_integral(sc, fun):
    m = sc.medium
    return Q.spectrum_integral(sc.run.spectrum_nm, sc.run.spectrum, m.lambda_s, m.lambda_a, m.lambda0, m.k_s, m.k_a,
                               fun)


def test_wavelength_trajectory_replay(api, ctx, oracle_lib):
    O = oracle_lib
    sc = S.wavelength(n_chains=64, n_steps=400, cap=64)
    _, _, ch = _chains(api, ctx, sc)
    assert ch.launch_info()[0]["general"] == 6
    lam0 = ch.read_lambda()
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 64)
    assert np.allclose(lam0, oc.lam, rtol=0, atol=1e-3)                # the same initial wavelengths
    ch.run_steps(sc.run.n_steps)
    xyz, n, _ = ch.read_states()
    lam = ch.read_lambda()
    margin = oc.run(sc.run.n_steps, margins=True)
    clean = np.nonzero(margin > 1e-3)[0]
    assert len(clean) >= 32
    acc, oacc = ch.read_accumulators(), oc.accumulators()
    moved = 0
    for c in clean:
        assert n[c] == oc.n[c], (c, n[c], oc.n[c])
        k = int(n[c])
        assert np.allclose(xyz[c, :, :k].T, oc.xyz[c, :k], atol=2e-4), c
        assert abs(lam[c] - oc.lam[c]) < 1e-3, (c, lam[c], oc.lam[c])
        assert np.array_equal(acc[c, 8:16], np.concatenate([oacc["prop"][c], oacc["acc"][c]]))
        moved += lam[c] != lam0[c]
    assert moved > len(clean) // 2                                       # wavelength moves were accepted


def test_wavelength_single_scatter_sector(api, ctx, oracle_lib):
    O = oracle_lib
    sc = S.wavelength(n_chains=8192, n_steps=20_000, cap=3)
    _, _, ch = _chains(api, ctx, sc)
    z2_gpu = ch.pair_z2()[0]
    m, s, d, r = O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[0]), O.run(sc.run, 0.1)
    assert abs(z2_gpu / O.z2_spectrum(m, s, d, r) - 1.0) < 1e-4
    ch.run_steps(sc.run.n_steps)
    e = ch.read_estimator()[0]
    ref = _spectrum_integral(sc, lambda ls, la, lam: Q.z2_closed(1.0, 0.1, 1.0 / ls + 1.0 / la) +
                             Q.z3(1.0, 0.1, ls, la, 0.9))
    assert abs(e["intensity"] - ref) < 3 * e["std_err"] and e["rel_err"] < 0.005, (e["intensity"], e["std_err"], ref)
    mean_ref = _spectrum_integral(sc, lambda ls, la, lam: lam * (Q.z2_closed(1.0, 0.1, 1.0 / ls + 1.0 / la) +
                                                                 Q.z3(1.0, 0.1, ls, la, 0.9))) / ref
    lam = ch.read_lambda().astype(np.float64)
    assert abs(lam.mean() - mean_ref) < 4 * lam.std() / math.sqrt(len(lam)), (lam.mean(), mean_ref)


def test_wavelength_split_and_checkpoint_replay(api, ctx):
    sc = S.wavelength(n_chains=256, n_steps=0, cap=64)
    _, _, a = _chains(api, ctx, sc)
    _, _, b = _chains(api, ctx, sc)
    a.run_steps(1500)
    b.run_steps(500)
    blob = b.save_state()
    b.run_steps(1000)
    assert np.array_equal(a.read_lambda(), b.read_lambda())
    assert np.array_equal(a.read_states()[0], b.read_states()[0])
    b.load_state(blob)
    b.run_steps(1000)
    assert np.array_equal(a.read_lambda(), b.read_lambda())


def test_wavelength_refusals(api, ctx):
    from paper_1811_04156_gb300._lib import PathmcError
    sc = S.wavelength(n_chains=64)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    import dataclasses
    for run in (dataclasses.replace(sc.run, within=S.WITHIN_MALA), dataclasses.replace(sc.run, gradients=True),
                dataclasses.replace(sc.run, layout=S.LAYOUT_LANE), dataclasses.replace(sc.run, sigma_lambda=0.0),
                dataclasses.replace(sc.run, spectrum_nm=(300.0, 300.0), spectrum=(1.0, 1.0)),
                dataclasses.replace(sc.run, spectrum_nm=(300.0, 400.0), spectrum=(0.0, 0.0))):
        with pytest.raises(PathmcError):
            api.Chains(ctx, medium, geom, run)
    ch = api.Chains(ctx, medium, geom, sc.run)
    with pytest.raises(PathmcError):
        api.seed_from_tracer(ch)
    plain = S.plain(n_chains=64)
    chp = api.Chains(ctx, api.Medium(ctx, plain.medium), api.Geometry(ctx, plain.sources, plain.sensors, plain.pairs),
                     plain.run)
    with pytest.raises(PathmcError):
        chp.read_lambda()
