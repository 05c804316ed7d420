"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a published test
vector, a normalisation, a closed form, an independent quadrature
(tests/quadrature.py), a finite difference, or the forward tracer of the
appendix (Algorithm 1) against the RJMCMC estimate.
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import quadrature as Q
from paper_1811_04156_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene_objs(O, med, src, sen):
    return O.medium(med), O.source(src), O.sensor(sen)


# --------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------
def test_philox_known_answers(oracle_lib):
    O = oracle_lib
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


def test_u01_range_and_resolution(oracle_lib):
    O = oracle_lib
    lo = O.lib().or_u01(0)
    hi = O.lib().or_u01(0xFFFFFFFF)
    assert lo == 0.5 / 2**23 and hi == 1 - 0.5 / 2**23
    assert 0 < lo < hi < 1


def test_onb_is_orthonormal(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(1)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        e1, e2 = np.zeros(3), np.zeros(3)
        O.lib().or_onb(O._ptr(n), O._ptr(e1), O._ptr(e2))
        M = np.stack([e1, e2, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
        assert np.linalg.det(M) > 0


# --------------------------------------------------------------------------
# Factors of the path density
# --------------------------------------------------------------------------
@pytest.mark.parametrize("G", [0.3, 0.9, 0.94, 0.95])
def test_kappa_eq_solves_langevin(oracle_lib, G):
    k = oracle_lib.kappa_eq(G)
    assert abs(1 / math.tanh(k) - 1 / k - G) < 1e-12
    if G >= 0.9:  # coth k -> 1 so kappa_eq -> 1/(1 - G)
        assert abs(k - 1 / (1 - G)) < 1e-5 * k


@pytest.mark.parametrize("G,fsl", [(0.0, 0.0), (0.5, 0.0), (0.9, 0.0), (0.94, 0.0), (0.95, 0.45), (0.95, 1.0)])
def test_phase_function_normalised_with_mean_G(oracle_lib, G, fsl):
    O = oracle_lib
    m = O.medium(S.Medium(g=G, f_sl=fsl))
    f = lambda c: math.exp(O.log_sigma_cos(m, c))
    pts = [1 - 1e-3, 1 - 1e-2] if G > 0.5 else None
    norm = quad(f, -1, 1, points=pts, limit=400, epsabs=0, epsrel=1e-11)[0]
    mean = quad(lambda c: c * f(c), -1, 1, points=pts, limit=400, epsabs=1e-13, epsrel=1e-11)[0]
    assert abs(norm - 1) < 1e-8
    assert abs(mean - G) < 1e-8
    # per-steradian density = per-cos density / 2 pi
    assert abs(O.log_sigma(m, 0.3) - (O.log_sigma_cos(m, 0.3) - math.log(2 * math.pi))) < 1e-14


@pytest.mark.parametrize("kappa", [0.0, 1.0, 38.0])
def test_emission_integrates_to_one(oracle_lib, kappa):
    O = oracle_lib
    s = O.source(S.Source(emission=S.EMIT_VMF if kappa > 0 else S.EMIT_ISOTROPIC, kappa=kappa,
                          direction=(0.0, 0.0, 1.0)))
    f = lambda w: 2 * math.pi * math.exp(O.log_emission(s, [math.sqrt(max(0, 1 - w * w)), 0.0, w]))
    assert abs(quad(f, -1, 1, points=[1 - 1e-2] if kappa > 10 else None, epsabs=0, epsrel=1e-11, limit=200)[0]
               - 1) < 1e-9


def test_detection_probability_is_a_probability(oracle_lib):
    O = oracle_lib
    d = O.sensor(S.Sensor(rho=S.RHO_PAPER, rho_hat=(0.0, -1.0, 0.0)))
    xs = np.linspace(-1, 1, 201)
    vals = [math.exp(O.log_rho(d, [0.0, -x, math.sqrt(max(0, 1 - x * x))])) for x in xs]
    assert all(0 < v <= 1 for v in vals)
    assert all(b > a for a, b in zip(vals, vals[1:]))  # the preferred direction is the most sensitive


def test_detection_probability_values(oracle_lib):
    """rho at the preferred direction, across it and against it, from the
    closed form of Eq. detection_prob (tests/golden/detection_prob.txt): a
    changed constant, a swapped sign or cosh for cos fails one of the three."""
    O = oracle_lib
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "detection_prob.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for rho_hat in ((0.0, -1.0, 0.0), (0.6, 0.0, 0.8)):
        d = O.sensor(S.Sensor(rho=S.RHO_PAPER, rho_hat=rho_hat))
        h = np.asarray(rho_hat)
        # a second direction normal to rho_hat for the x = 0 case
        perp = np.cross(h, [0.0, 0.0, 1.0] if abs(h[2]) < 0.9 else [1.0, 0.0, 0.0])
        perp /= np.linalg.norm(perp)
        for x, want in rows:
            nu = h if x > 0 else (-h if x < 0 else perp)
            got = math.exp(O.log_rho(d, list(nu)))
            assert abs(got / want - 1) < 1e-8, (rho_hat, x, got, want)


def test_layered_depths_brute_force(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(3)
    L = 12
    ls, la = rng.uniform(1, 10, L), rng.uniform(20, 200, L)
    med = S.Medium(S.LAYERED, z0=-30.0, dz=5.0, lambda_s_layers=ls, lambda_a_layers=la)
    m = O.medium(med)
    for _ in range(20):
        P, Qp = rng.uniform(-40, 40, 3), rng.uniform(-40, 40, 3)
        ta, tb = O.segment_depths(m, P, Qp)
        # midpoint rule with 2e5 points in FP64
        u = (np.arange(200000) + 0.5) / 200000
        z = P[2] + u * (Qp[2] - P[2])
        lay = np.clip(np.floor((z + 30.0) / 5.0), 0, L - 1).astype(int)
        ell = np.linalg.norm(Qp - P)
        assert abs(ta - (ell / la[lay]).mean()) < 2e-4 * max(ta, 1e-9)
        assert abs(tb - (ell / ls[lay]).mean()) < 2e-4 * max(tb, 1e-9)
    # one layer reduces to the homogeneous medium
    one = O.medium(S.Medium(S.LAYERED, z0=0.0, dz=1.0, lambda_s_layers=np.array([2.0]),
                            lambda_a_layers=np.array([7.0])))
    hom = O.medium(S.Medium(lambda_s=2.0, lambda_a=7.0))
    P, Qp = np.array([0.1, 0.2, -3.0]), np.array([1.0, -2.0, 4.0])
    assert np.allclose(O.segment_depths(one, P, Qp), O.segment_depths(hom, P, Qp), rtol=1e-13)


# --------------------------------------------------------------------------
# Dimension matching transformation
# --------------------------------------------------------------------------
def test_bispherical_roundtrip_and_jacobian(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(4)
    for _ in range(30):
        fk, fk1 = rng.normal(size=3), rng.normal(size=3)
        s, t, phi = rng.uniform(0.2, 2.9), rng.normal(), rng.uniform(0.1, 6.2)
        f = O.bisph_point(fk, fk1, s, t, phi)
        s2, t2, p2 = O.bisph_coords(fk, fk1, f)
        assert abs(s2 - s) < 1e-9 and abs(t2 - t) < 1e-9 and abs(p2 - phi) < 1e-9
        h = 1e-6
        J = np.zeros((3, 3))
        for i, dv in enumerate(np.eye(3) * h):
            J[:, i] = (O.bisph_point(fk, fk1, s + dv[0], t + dv[1], phi + dv[2]) -
                       O.bisph_point(fk, fk1, s - dv[0], t - dv[1], phi - dv[2])) / (2 * h)
        gamma = np.linalg.norm(fk1 - fk) / 2
        assert abs(abs(np.linalg.det(J)) / math.exp(O.lib().or_log_bisph_jacobian(gamma, s, t)) - 1) < 1e-6
    # s -> pi puts the vertex on the segment, t = 0 at its midpoint
    fk, fk1 = np.array([0.0, 0, 0]), np.array([2.0, 0, 0])
    assert np.allclose(O.bisph_point(fk, fk1, math.pi - 1e-12, 0.0, 0.3), [1, 0, 0], atol=1e-9)


@pytest.mark.parametrize("beta", [0.01, 1.0, 10.0, 16.7])
def test_insertion_densities_normalised(oracle_lib, beta):
    O = oracle_lib
    qs = quad(lambda s: math.exp(O.lib().or_log_q_s(beta, s)), 0, math.pi, epsabs=0, epsrel=1e-11, limit=200)[0]
    qt = quad(lambda t: math.exp(O.lib().or_log_q_t(t)), -60, 60, epsabs=0, epsrel=1e-11, limit=200)[0]
    assert abs(qs - 1) < 1e-9 and abs(qt - 1) < 1e-9


# --------------------------------------------------------------------------
# Gradients
# --------------------------------------------------------------------------
def _rand_path(rng, n, D=3.0, R=0.4):
    c = np.array([0.0, 0.0, D])
    pts = [np.zeros(3)]
    for i in range(1, n - 1):
        pts.append(np.array([0.0, 0.0, D * i / n]) + rng.normal(scale=0.4, size=3))
    nu = np.array([0.2, -0.1, -1.0]) + 0.3 * rng.normal(size=3)
    pts.append(c + R * nu / np.linalg.norm(nu))
    return np.array(pts)


MEDIA = [
    S.Medium(lambda_s=0.7, lambda_a=4.0, g=0.8),
    S.Medium(lambda_s=0.7, lambda_a=4.0, g=0.9, f_sl=0.45),
    S.Medium(S.LAYERED, g=0.85, z0=-1.0, dz=0.8, lambda_s_layers=np.array([0.5, 1.0, 0.7, 2.0, 0.9]),
             lambda_a_layers=np.array([5.0, 3.0, 9.0, 4.0, 6.0])),
]


@pytest.mark.parametrize("mi", range(len(MEDIA)))
def test_adjoint_matches_finite_differences(oracle_lib, mi):
    O = oracle_lib
    rng = np.random.default_rng(10 + mi)
    src = S.Source(emission=S.EMIT_VMF, kappa=3.0, direction=(0.1, 0.0, 1.0))
    sen = S.Sensor((0.0, 0.0, 3.0), 0.4, rho=S.RHO_PAPER, rho_hat=(0.0, -1.0, 0.0))
    m, s, d = _scene_objs(O, MEDIA[mi], src, sen)
    done = 0
    for _ in range(40):
        f = _rand_path(rng, int(rng.integers(3, 9)))
        lp, g = O.grad_logp(m, s, d, f)
        if not np.isfinite(lp):
            continue
        h = 1e-6
        fd = np.zeros_like(f)
        for i in range(len(f)):
            for k in range(3):
                fp, fm = f.copy(), f.copy()
                fp[i, k] += h
                fm[i, k] -= h
                fd[i, k] = (O.logp(m, s, d, fp) - O.logp(m, s, d, fm)) / (2 * h)
        assert np.allclose(g, fd, rtol=1e-5, atol=1e-5 * (1 + np.abs(fd).max()))
        done += 1
    assert done >= 10


def test_score_matches_finite_differences(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(21)
    sen = S.Sensor((0.0, 0.0, 3.0), 0.4)
    src = S.Source()
    for mi in (0, 1, 2):
        base = MEDIA[mi]
        m, s, d = _scene_objs(O, base, src, sen)
        f = None
        while f is None:
            cand = _rand_path(rng, 6)
            if np.isfinite(O.logp(m, s, d, cand)):
                f = cand
        sc = O.score(m, s, d, f)
        import copy
        if base.kind == S.HOMOGENEOUS:
            names = ["lambda_s", "lambda_a", "g"]
            for i, nm in enumerate(names):
                v = getattr(base, nm)
                h = 1e-6 * max(abs(v), 1e-3)
                up, dn = copy.deepcopy(base), copy.deepcopy(base)
                setattr(up, nm, v + h)
                setattr(dn, nm, v - h)
                fd = (O.logp(O.medium(up), s, d, f) - O.logp(O.medium(dn), s, d, f)) / (2 * h)
                assert abs(sc[i] - fd) < 1e-6 * (1 + abs(fd))
        else:
            L = base.n_layers
            for i in range(2 * L):
                arr = "lambda_s_layers" if i < L else "lambda_a_layers"
                j = i % L
                up, dn = copy.deepcopy(base), copy.deepcopy(base)
                v = getattr(base, arr)[j]
                h = 1e-6 * v
                getattr(up, arr)[j] = v + h
                getattr(dn, arr)[j] = v - h
                fd = (O.logp(O.medium(up), s, d, f) - O.logp(O.medium(dn), s, d, f)) / (2 * h)
                assert abs(sc[i] - fd) < 1e-6 * (1 + abs(fd))


# --------------------------------------------------------------------------
# Normalisation: zero- and single-scattering parts
# --------------------------------------------------------------------------
@pytest.mark.parametrize("D,R,ls,la", [(1.0, 0.1, 1e30, 1e30), (1.0, 0.1, 1e30, 5.0), (1.0, 0.1, 0.5, 5.0),
                                       (50.0, 0.165, 5.0, 100.0), (1.5, 0.5, 1.0, 5.0)])
def test_direct_sector_quadrature(oracle_lib, D, R, ls, la):
    O = oracle_lib
    m, s, d = _scene_objs(O, S.Medium(lambda_s=ls, lambda_a=la), S.Source(), S.Sensor((0.0, 0.0, D), R))
    z2 = O.z2(m, s, d)
    if ls > 1e20 and la > 1e20:  # solid angle / 4 pi
        assert abs(z2 - (1 - math.sqrt(1 - (R / D) ** 2)) / 2) < 1e-12
    assert abs(z2 / Q.z2_closed(D, R, 1 / ls + 1 / la) - 1) < 1e-8


def test_tracer_without_scattering_matches_closed_form(oracle_lib):
    O = oracle_lib
    m, s, d = _scene_objs(O, S.Medium(lambda_s=1e9, lambda_a=2.0), S.Source(), S.Sensor((0.0, 0.0, 1.5), 0.5))
    tr = O.trace(m, s, d, 5, 2_000_000, max_scatter=0)
    ref = Q.z2_closed(1.5, 0.5, 0.5 + 1e-9)
    assert abs(tr["I"] - ref) < 3 * tr["se"] + 1e-12


def test_chain_single_scatter_sector_matches_quadrature(oracle_lib):
    """Cap 3: I = Z2 + Z3 exactly; birth/death, Jacobian and q are all exercised."""
    O = oracle_lib
    sc = S.plain()
    sc.run.burn_in = 2000
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 3)
    ch.run(60000)
    m, s, d = _scene_objs(O, sc.medium, sc.sources[0], sc.sensors[0])
    I, se, _ = O.direct_estimate(ch.accumulators(), O.z2(m, s, d))
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(I - ref) < 3 * se, (I, se, ref)
    assert se / I < 0.01


def test_mala_chain_single_scatter_sector(oracle_lib):
    O = oracle_lib
    sc = S.gradients(n_chains=64, n_steps=60000, cap=3)
    sc.run.burn_in = 2000
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 3)
    ch.run(60000)
    m, s, d = _scene_objs(O, sc.medium, sc.sources[0], sc.sensors[0])
    I, se, _ = O.direct_estimate(ch.accumulators(), O.z2(m, s, d))
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(I - ref) < 3 * se, (I, se, ref)


def test_chain_matches_forward_tracer_all_orders(oracle_lib):
    """Well-mixing scene (isotropic scattering, large close sensor): RJMCMC
    intensity and per-vertex-count split agree with Algorithm 1."""
    O = oracle_lib
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.0)
    src, sen = S.Source(), S.Sensor((0.0, 0.0, 1.5), 0.5)
    run = S.Run(seed=1234, burn_in=3000, sigma=0.1)
    cap = 24
    ch = O.Chains(med, src, sen, run, 96, cap)
    H = np.zeros((96, cap + 1))
    ch.run(60000, n_hist=H)
    m, s, d = _scene_objs(O, med, src, sen)
    z2 = O.z2(m, s, d)
    I, se, _ = O.direct_estimate(ch.accumulators(), z2)
    tr = O.trace(m, s, d, 77, 4_000_000, max_scatter=cap - 2, hist=True)
    assert abs(I - tr["I"]) < 3 * math.hypot(se, tr["se"]), (I, se, tr["I"], tr["se"])
    h = H.sum(0)
    zc = z2 * h / h[2]
    for n in (3, 4, 5):
        assert abs(zc[n] / tr["hist"][n - 2] - 1) < 0.04


def test_reference_density_is_normalised(oracle_lib):
    """Importance sampling from q_ref with cap 3 recovers Z2 + Z3."""
    O = oracle_lib
    sc = S.plain()
    m, s, d = _scene_objs(O, sc.medium, sc.sources[0], sc.sensors[0])
    out = O.qref_bridge_sums(m, s, d, 3, 99, 0, 400_000)
    mean = out[1] / out[3]
    se = math.sqrt(max(out[2] / out[3] - mean ** 2, 0) / out[3])
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(mean - ref) < 3 * se + 1e-3 * ref, (mean, se, ref)


def test_counter_based_resume_is_exact(oracle_lib):
    O = oracle_lib
    sc = S.plain()
    a = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 8, 64)
    b = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 8, 64)
    a.run(3000)
    b.run(1000)
    b.run(2000)
    assert np.array_equal(a.n, b.n) and np.array_equal(a.xyz, b.xyz)


def test_dimension_jumps_balance_a_toy_target(oracle_lib):
    """Detailed balance of the birth/death machinery on its own: the chains'
    moves (Gaussian steps, vMF end steps, tau_b-weighted births by bispherical
    insertion, uniform deaths, Green's acceptance) run on a product target
    with known sector weights -- P(n) proportional to w_n, interior vertices
    ~ N(mu_k, s^2 I), the end vertex uniform on the sensor -- and the visited
    vertex counts reproduce w_n / sum w.  A missing reverse-move factor, a
    wrong Jacobian or a transposed birth/death ratio shifts P(n) by factors
    of order (n - 2)/(n - 1) or more."""
    import ctypes as C
    O = oracle_lib
    cap = 6
    w = np.zeros(cap + 1)
    w[2:] = [1.0, 2.0, 1.5, 0.7, 0.3]
    sc = S.plain()
    sc.run.burn_in = 2000
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, cap)
    ch.r.toy_s = 0.1
    ch.r.toy_w = w.ctypes.data_as(C.POINTER(C.c_double))
    H = np.zeros((64, cap + 1))
    ch.run(100_000, n_hist=H)
    P = H / H.sum(axis=1, keepdims=True)
    mean, se = P.mean(axis=0), P.std(axis=0, ddof=1) / math.sqrt(64)
    ref = w / w.sum()
    for n in range(2, cap + 1):
        assert abs(mean[n] - ref[n]) < 4 * se[n], (n, mean[n], ref[n], se[n])
    assert np.abs(mean - ref).max() < 0.01
    acc = ch.accumulators()
    assert acc["acc"][:, 2].sum() > 0.05 * acc["prop"][:, 2].sum()  # births are accepted often enough
