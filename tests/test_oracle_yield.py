"""Pins of the oracle's relative-light-yield machinery (section "Comparison of
relative light yield"; appendix "Relative light yield transformation").

The map T of paths ending on sensor 0 to paths ending on sensor 1 is pinned
by its round trip, by finite-difference Jacobians (volume for interior
vertices, area for the end vertex), and the geometric estimator
B = E_0[sqrt(p_1/p_0)] / E_1[sqrt(p_0/p_1)] by two known ratios: B = 1 for two
sensors placed symmetrically about an isotropic source, and B = I_1 / I_0 from
the independent single-scattering quadrature at vertex cap 3.
"""
import math

import numpy as np
import pytest

import quadrature as Q
from paper_1811_04156_gb300 import scenes as S


def _map_scene(O, R1=0.15):
    src = S.Source((0.1, -0.2, 0.05), S.EMIT_VMF, 8.0, (0.0, 0.0, 1.0))
    d0 = S.Sensor((0.1, -0.2, 12.0), 0.15)
    d1 = S.Sensor((6.0, 0.5, 10.5), R1)
    return O.source(src), O.sensor(d0), O.sensor(d1), src, d0, d1


def _paths_to_sensor0(src, d0, n, count, seed, lateral=0.8):
    xyz, nn = S.random_paths(src.pos, d0.centre, d0.radius, count, n, n, n, seed, lateral=lateral)
    out = []
    for i in range(count):
        p = xyz[:, i, :n].T.astype(np.float64)
        c = np.asarray(d0.centre, dtype=np.float64)
        p[-1] = c + d0.radius * (p[-1] - c) / np.linalg.norm(p[-1] - c)  # exactly on the sphere in FP64
        out.append(p)
    return out


def test_map_round_trip_and_geometry(oracle_lib):
    O = oracle_lib
    s, d0, d1, src, sen0, sen1 = _map_scene(O)
    T = O.ymap(s, d0, d1)
    # frame: orthonormal, k towards sensor 0, m away from sensor 1
    for a, b, v in (("k", "k", 1), ("m", "m", 1), ("n", "n", 1), ("k", "m", 0), ("k", "n", 0), ("m", "n", 0)):
        assert abs(np.dot(getattr(T, a), getattr(T, b)) - v) < 1e-12
    assert np.dot(T.m, np.asarray(sen1.centre) - np.asarray(src.pos)) < 0
    for path in _paths_to_sensor0(src, sen0, 9, 20, 3):
        y, lj = O.ymap_forward(T, path)
        assert np.isfinite(lj)
        assert np.allclose(y[0], src.pos)
        assert abs(np.linalg.norm(y[-1] - np.asarray(sen1.centre)) - sen1.radius) < 1e-12  # on sensor 1
        x, lj2 = O.ymap_inverse(T, y)
        assert np.allclose(x, path, atol=1e-9)
        assert abs(lj - lj2) < 1e-9
    # the straight path's sensor-0 point (w = 1 on the axis) lands about R1 from sensor 1's centre
    e0 = np.asarray(src.pos) + T.b0 * np.asarray(T.k)
    straight = np.stack([np.asarray(src.pos), 0.5 * (np.asarray(src.pos) + e0), e0])
    y, _ = O.ymap_forward(T, straight)
    dist = np.linalg.norm(y[1] - np.asarray(sen1.centre))
    mid_arc = np.asarray(src.pos) - T.rC * np.asarray(T.m) + T.rC * (
        np.asarray(T.m) * math.cos(0.5 * T.Omega) + np.asarray(T.k) * math.sin(0.5 * T.Omega))
    assert np.allclose(y[1], mid_arc, atol=1e-9)  # the axis bends onto the circle of radius rC
    chord = 2 * T.rC * math.sin(0.5 * (2 * math.atan2(
        np.linalg.norm(np.cross(T.k, np.asarray(sen1.centre) - np.asarray(src.pos))),
        np.dot(T.k, np.asarray(sen1.centre) - np.asarray(src.pos)))))
    assert abs(chord - np.linalg.norm(np.asarray(sen1.centre) - np.asarray(src.pos))) < 1e-9
    assert dist > 0


def test_map_interior_jacobian_by_finite_differences(oracle_lib):
    O = oracle_lib
    s, d0, d1, src, sen0, _ = _map_scene(O, R1=0.2)
    T = O.ymap(s, d0, d1)
    h = 1e-6
    for path in _paths_to_sensor0(src, sen0, 3, 12, 11, lateral=2.0):
        _, lj = O.ymap_forward(T, path)
        end_term = 2.0 * math.log(0.2 / 0.15)
        Jm = np.zeros((3, 3))
        for c in range(3):
            p, m_ = path.copy(), path.copy()
            p[1, c] += h
            m_[1, c] -= h
            Jm[:, c] = (O.ymap_forward(T, p)[0][1] - O.ymap_forward(T, m_)[0][1]) / (2 * h)
        assert abs(math.log(abs(np.linalg.det(Jm))) - (lj - end_term)) < 1e-6


def test_map_end_vertex_area_ratio(oracle_lib):
    O = oracle_lib
    s, d0, d1, src, sen0, sen1 = _map_scene(O, R1=0.2)
    T = O.ymap(s, d0, d1)
    c0, c1 = np.asarray(sen0.centre), np.asarray(sen1.centre)
    rng = np.random.default_rng(4)
    h = 1e-6
    for _ in range(10):
        th, ph = rng.uniform(0.3, 2.8), rng.uniform(0, 2 * math.pi)

        def pt(a, b):
            return c0 + 0.15 * np.array([math.sin(a) * math.cos(b), math.sin(a) * math.sin(b), math.cos(a)])

        def img(a, b):
            path = np.stack([np.asarray(src.pos), pt(a, b)])
            return O.ymap_forward(T, path)[0][1]
        ta = (pt(th + h, ph) - pt(th - h, ph)) / (2 * h)
        tb = (pt(th, ph + h) - pt(th, ph - h)) / (2 * h)
        ia = (img(th + h, ph) - img(th - h, ph)) / (2 * h)
        ib = (img(th, ph + h) - img(th, ph - h)) / (2 * h)
        ratio = np.linalg.norm(np.cross(ia, ib)) / np.linalg.norm(np.cross(ta, tb))
        assert abs(ratio - (0.2 / 0.15) ** 2) < 1e-6
        y = img(th, ph)
        assert abs(np.linalg.norm(y - c1) - 0.2) < 1e-12


def test_map_domain_outside_gives_zero_ratio(oracle_lib):
    """A vertex behind the cylinder axis (rC + xb b1 <= 0) has no one-to-one
    image: log p_1 = -inf, so the path adds 0 to E_0[sqrt(p_1/p_0)]."""
    O = oracle_lib
    s, d0, d1, src, sen0, _ = _map_scene(O)
    T = O.ymap(s, d0, d1)
    path = _paths_to_sensor0(src, sen0, 4, 1, 5)[0]
    path[1] = np.asarray(src.pos) + 1.5 * T.rC * T.b0 / T.b1 * np.asarray(T.m)  # xb b1 = 1.5 rC > 0: inside
    assert np.isfinite(O.ymap_forward(T, path)[1])
    path[1] = np.asarray(src.pos) - 1.5 * T.rC * T.b0 / T.b1 * np.asarray(T.m)  # rC + xb b1 < 0: outside
    assert O.ymap_forward(T, path)[1] == -math.inf


def _oracle_ratio(O, sc, n_chains, rounds, thin, burn_rounds, cap):
    m = O.medium(sc.medium)
    s = O.source(sc.sources[0])
    d0, d1 = O.sensor(sc.sensors[0]), O.sensor(sc.sensors[1])
    T = O.ymap(s, d0, d1)
    ch = [O.Chains(sc.medium, sc.sources[0], sc.sensors[k], sc.run, n_chains, cap, chain_offset=k * n_chains)
          for k in (0, 1)]
    sums = [np.zeros(n_chains), np.zeros(n_chains)]
    for r in range(rounds):
        for k in (0, 1):
            ch[k].run(thin)
        if r < burn_rounds:
            continue
        for k in (0, 1):
            for c in range(n_chains):
                lr = O.ymap_logratio(m, s, d0, d1, T, k, ch[k].xyz[c, : ch[k].n[c]])
                sums[k][c] += math.exp(0.5 * lr) if np.isfinite(lr) else 0.0
    return O.yield_ratio_estimate(sums[0], sums[1])


def test_geometric_estimator_symmetric_sensors(oracle_lib):
    """Two sensors at the same distance from an isotropic source in a
    homogeneous medium see the same light: B = 1 (the cylinder map is far
    from a rigid motion, so its Jacobian is exercised)."""
    O = oracle_lib
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.0)
    a = math.radians(70.0)
    sensors = [S.Sensor((0.0, 0.0, 1.2), 0.3), S.Sensor((1.2 * math.sin(a), 0.0, 1.2 * math.cos(a)), 0.3)]
    run = S.Run(seed=77, burn_in=0, sigma=0.1)
    sc = S.Scene("sym", med, [S.Source()], sensors, [S.Pair(0, 0, 96, 16), S.Pair(0, 1, 96, 16)], run)
    B, se = _oracle_ratio(O, sc, 96, 300, 20, 30, 16)
    assert abs(B - 1.0) < 3 * se, (B, se)
    assert se < 0.03


def test_geometric_estimator_single_scatter_quadrature(oracle_lib):
    """Cap 3 (n in {2, 3}): B equals (Z2 + Z3)(D1) / (Z2 + Z3)(D0) from the
    independent quadrature; sensors at 1.0 m and 1.4 m, 50 degrees apart."""
    O = oracle_lib
    ls, la, g, R = 0.5, 5.0, 0.9, 0.3
    med = S.Medium(lambda_s=ls, lambda_a=la, g=g)
    a = math.radians(50.0)
    sensors = [S.Sensor((0.0, 0.0, 1.0), R), S.Sensor((1.4 * math.sin(a), 0.0, 1.4 * math.cos(a)), R)]
    run = S.Run(seed=91, burn_in=0, sigma=0.05)
    sc = S.Scene("cap3", med, [S.Source()], sensors, [S.Pair(0, 0, 128, 3), S.Pair(0, 1, 128, 3)], run)
    B, se = _oracle_ratio(O, sc, 128, 400, 10, 40, 3)
    cext = 1.0 / ls + 1.0 / la
    I0 = Q.z2_closed(1.0, R, cext) + Q.z3(1.0, R, ls, la, g)
    I1 = Q.z2_closed(1.4, R, cext) + Q.z3(1.4, R, ls, la, g)
    assert abs(B - I1 / I0) < 3 * se, (B, se, I1 / I0)
    assert se / B < 0.03


def test_half_space_depths_brute_force(oracle_lib):
    """The paper's two-region medium (plane x = 0) built as two layers in the
    rotated frame: optical depths equal a midpoint brute force in the paper's
    frame."""
    O = oracle_lib
    sc = S.two_sensor(0.1)
    m = O.medium(sc.medium)
    rng = np.random.default_rng(2)
    for _ in range(20):
        P, Qp = rng.normal(scale=5.0, size=3), rng.normal(scale=5.0, size=3)
        ta, tb = O.segment_depths(m, S.to_device_frame(P), S.to_device_frame(Qp))
        N = 200_000
        t = (np.arange(N) + 0.5) / N
        x = P[0] + t * (Qp[0] - P[0])
        L = np.linalg.norm(Qp - P)
        b = np.where(x < 0.0, 0.3, 0.1)
        assert abs(tb - L * b.mean()) < 1e-4 * L
        assert abs(ta - 0.01 * L) < 1e-9 * L
    # frame maps are inverse rotations
    v = rng.normal(size=(5, 3))
    assert np.allclose(S.to_paper_frame(S.to_device_frame(v)), v)
    R = S.to_device_frame(np.eye(3))
    assert abs(np.linalg.det(R) - 1.0) < 1e-12


def test_tracer_length_histogram_sums_to_intensity(oracle_lib):
    O = oracle_lib
    m, s, d = O.medium(S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.5)), O.source(S.Source()), \
        O.sensor(S.Sensor((0.0, 0.0, 1.5), 0.5))
    res, h = O.trace_lengths(m, s, d, 3, 200_000, 0.0, 1e6, 50, max_scatter=30)
    assert abs(h.sum() - res["I"]) < 1e-12 * max(res["I"], 1)
    res2, h2 = O.trace_lengths(m, s, d, 3, 200_000, 1.0, 3.0, 8, max_scatter=30)
    assert h2.sum() < res["I"] and (h2 >= 0).all()


def _gauss_logratios(n_rows, n0, n1, seed, c=3.0, mu=0.5, sd=1.3):
    """q0 = exp(-x^2/2), q1 = c exp(-(x - mu)^2 / (2 sd^2)): c1/c0 = c sd."""
    rng = np.random.default_rng(seed)
    x0 = rng.normal(size=(n_rows, n0))
    x1 = mu + sd * rng.normal(size=(n_rows, n1))

    def lq0(x):
        return -0.5 * x * x

    def lq1(x):
        return math.log(c) - 0.5 * ((x - mu) / sd) ** 2
    return lq1(x0) - lq0(x0), lq0(x1) - lq1(x1), c * sd


def test_optimal_bridge_recovers_gaussian_ratio(oracle_lib):
    """Exact draws from two Gaussians of known normalising constants: over 40
    independent repetitions the estimates centre on c1/c0, their spread
    matches the reported group standard errors, and each estimate sits at the
    estimator's fixed point."""
    O = oracle_lib
    rs, ses = [], []
    for seed in range(40):
        L0, L1, ref = _gauss_logratios(50, 400, 300, 500 + seed)
        r, se, it, geo = O.optimal_bridge(L0, L1, groups=16)
        rs.append(r)
        ses.append(se)
    rs = np.array(rs)
    sd = rs.std(ddof=1)
    assert abs(rs.mean() - ref) < 4 * sd / math.sqrt(len(rs)), (rs.mean(), sd, ref)
    assert 0.6 < np.mean(ses) / sd < 1.6, (np.mean(ses), sd)
    s0, s1 = 400 / 700, 300 / 700
    a = (1.0 / (s1 + s0 * r / np.exp(L0))).mean()
    b = (1.0 / (s1 * np.exp(-L1) + s0 * r)).mean()
    assert abs(a / b / r - 1) < 1e-9
    assert abs(geo / ref - 1) < 0.05


def test_optimal_bridge_exact_for_proportional_densities(oracle_lib):
    """q1 = 2.5 q0: every l equals 2.5 and the estimator returns it exactly."""
    O = oracle_lib
    L0 = np.full((7, 5), math.log(2.5))
    L1 = np.full((7, 4), -math.log(2.5))
    r, se, it, geo = O.optimal_bridge(L0, L1, groups=2)
    assert abs(r - 2.5) < 1e-12 and abs(geo - 2.5) < 1e-12


def test_optimal_bridge_beats_geometric_on_poor_overlap(oracle_lib):
    """With little overlap the optimal bridge's spread over independent
    repetitions is smaller than the geometric estimator's."""
    O = oracle_lib
    opt, geo = [], []
    for seed in range(12):
        L0, L1, ref = _gauss_logratios(20, 200, 200, 100 + seed, mu=2.5, sd=0.7)
        r, se, it, g = O.optimal_bridge(L0, L1, groups=4)
        opt.append(r / ref)
        geo.append(g / ref)
    assert np.std(opt) < np.std(geo)
    assert abs(np.mean(opt) - 1) < 3 * np.std(opt) / math.sqrt(12) + 0.01
