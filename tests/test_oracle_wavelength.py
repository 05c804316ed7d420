"""Pins of the oracle's wavelength sampling (section "Discussion": a
wavelength parameter added to the path density and sampled along with the
path vertices).  The paper gives no wavelength model; the reading is a
normalised piecewise-linear emission-times-detection spectrum S(l) and power
laws of the scattering and absorption coefficients about a reference
wavelength.  The chains sample the joint density S(l) p_l(path), so the
detected intensity is the integral over l of S(l) I(l), and at vertex cap 3
that is the integral of S(l) (Z2(l) + Z3(l)), computed here by Gauss-Legendre
in l over the independent quadrature of tests/quadrature.py."""
import dataclasses
import math

import numpy as np
import pytest

import quadrature as Q
from paper_1811_04156_gb300 import scenes as S


def _integral_over_spectrum(sc, fun, nodes=6):
    """int S(l) fun(lambda_s(l), lambda_a(l), l) dl over the spectrum table."""
    m = sc.medium
    return Q.spectrum_integral(sc.run.spectrum_nm, sc.run.spectrum, m.lambda_s, m.lambda_a, m.lambda0, m.k_s, m.k_a,
                               fun, nodes)


def test_spectrum_normalised_and_quantile_inverts_it(oracle_lib):
    O = oracle_lib
    sc = S.wavelength()
    sc.run.spectrum_nm, sc.run.spectrum = (300.0, 380.0, 450.0, 600.0), (0.2, 1.5, 0.7, 0.0)
    r = O.run(sc.run, 0.1)
    xs = np.linspace(300.0, 600.0, 60001)                    # the table's range: S is linear between nodes
    v = np.array([math.exp(O.log_spectrum(r, x)) for x in xs])
    assert abs(np.trapezoid(v, xs) - 1.0) < 1e-9
    assert O.log_spectrum(r, 299.9) == -math.inf and O.log_spectrum(r, 600.1) == -math.inf
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (v[1:] + v[:-1]) * np.diff(xs))])
    for u in (0.01, 0.2, 0.5, 0.77, 0.999):
        q = O.spectrum_quantile(r, u)
        assert abs(np.interp(q, xs, cdf) - u) < 1e-6, (u, q)


def test_medium_follows_the_power_laws(oracle_lib):
    O = oracle_lib
    sc = S.wavelength()
    m = O.medium(sc.medium)
    m2 = O.medium_at(m, 800.0)                               # twice the reference wavelength
    assert math.isclose(1.0 / m2.lambda_s, (1.0 / 0.5) / 16.0, rel_tol=1e-12)   # b ~ l^-4
    assert math.isclose(1.0 / m2.lambda_a, (1.0 / 5.0) / 4.0, rel_tol=1e-12)    # a ~ l^-2
    m1 = O.medium_at(m, 400.0)
    assert m1.lambda_s == m.lambda_s and m1.lambda_a == m.lambda_a


def test_wavelength_chains_single_scatter_sector(oracle_lib):
    """Cap 3: the joint chains' intensity Z2_S / pi(n = 2), Z2_S the
    spectrum-weighted direct sector, against the spectrum integral of the
    independent single-scatter quadrature; the chains' wavelengths follow
    S(l) (Z2 + Z3)(l) / I."""
    O = oracle_lib
    sc = S.wavelength(n_chains=2048, n_steps=6000, cap=3)
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 2048, 3)
    oc.run(sc.run.n_steps)
    m, s, d, r = O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[0]), O.run(sc.run, 0.1)
    z2s = O.z2_spectrum(m, s, d, r)
    ref_z2 = _integral_over_spectrum(sc, lambda ls, la, lam: Q.z2_closed(1.0, 0.1, 1.0 / ls + 1.0 / la))
    assert abs(z2s / ref_z2 - 1.0) < 1e-5
    ref = _integral_over_spectrum(sc, lambda ls, la, lam: Q.z2_closed(1.0, 0.1, 1.0 / ls + 1.0 / la) +
                                  Q.z3(1.0, 0.1, ls, la, 0.9))
    I, se, _ = O.direct_estimate(oc.accumulators(), z2s)
    assert abs(I - ref) < 3 * se and se / I < 0.01, (I, se, ref)
    # wavelength marginal: mean and the share below 420 nm against the quadrature
    mean_ref = _integral_over_spectrum(sc, lambda ls, la, lam: lam * (Q.z2_closed(1.0, 0.1, 1.0 / ls + 1.0 / la) +
                                                                      Q.z3(1.0, 0.1, ls, la, 0.9))) / ref
    lam = oc.lam
    assert abs(lam.mean() - mean_ref) < 4 * lam.std() / math.sqrt(len(lam)), (lam.mean(), mean_ref)


def test_wavelength_independent_medium_keeps_the_spectrum(oracle_lib):
    """Without wavelength dependence (k = 0) the wavelength marginal is S and
    the intensity is the wavelength-free one."""
    O = oracle_lib
    sc = S.wavelength(n_chains=2048, n_steps=6000, cap=3)
    sc.medium = dataclasses.replace(sc.medium, k_s=0.0, k_a=0.0)
    oc = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 2048, 3)
    oc.run(sc.run.n_steps)
    m, s, d, r = O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[0]), O.run(sc.run, 0.1)
    I, se, _ = O.direct_estimate(oc.accumulators(), O.z2_spectrum(m, s, d, r))
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(I - ref) < 3 * se, (I, se, ref)
    # triangular spectrum on [300, 600] peaking at 420: mean (300 + 420 + 600) / 3 = 440
    lam = oc.lam
    assert abs(lam.mean() - 440.0) < 4 * lam.std() / math.sqrt(len(lam))
    # the CDF of the triangle at 420 nm is (420 - 300) / (600 - 300) = 0.4
    share = (lam < 420.0).mean()
    assert abs(share - 0.4) < 4 * math.sqrt(0.4 * 0.6 / len(lam))
