"""Pins of the oracle's tree coordinates and tree-coordinate moves (appendix
"Path space coordinate system", Fig. tree_coords; section "Path proposal
distribution").

The coordinate map is pinned by its round trip, by a finite-difference
determinant against the product of the per-node volume factors
(d1 d2 / (2 gamma))^3 sin^2 s (the bispherical element in (zeta, t, phi),
reading Q14), by the tree of Fig. tree_coords, and by the paper's statement
that turning one vertex turns every vertex that depends on it: a change of
phi_m rotates the whole subtree of m rigidly about the axis of m's foci.  The
move built on it is pinned like the Cartesian moves: at vertex cap 3 the
chains' intensity equals Z2 + Z3 from the independent quadrature, and in a
well-mixing scene the intensity and the vertex-count split equal the forward
tracer's.
"""
import math

import numpy as np
import pytest

import quadrature as Q
from paper_1811_04156_gb300 import scenes as S


def _path(n, seed, D=3.0, lateral=0.4):
    xyz, nn = S.random_paths((0.1, -0.2, 0.0), (0.3, 0.1, D), 0.4, 1, n, n, n, seed, lateral=lateral)
    return xyz[:, 0, :n].T.astype(np.float64)


def test_tree_of_the_figure(oracle_lib):
    """Nine vertices (Fig. tree_coords): f4 in (f0, f8); f2 in (f0, f4) and f6
    in (f4, f8) below it; f1, f3, f5, f7 at the bottom."""
    O = oracle_lib
    expect = {4: (0, 8, -1), 2: (0, 4, 4), 6: (4, 8, 4), 1: (0, 2, 2), 3: (2, 4, 2), 5: (4, 6, 6), 7: (6, 8, 6)}
    for m, v in expect.items():
        assert O.tree_node(m, 9) == v


@pytest.mark.parametrize("n", [3, 4, 7, 12, 33])
def test_tree_round_trip(oracle_lib, n):
    O = oracle_lib
    v = O.tree_vref(O.source(S.Source((0.1, -0.2, 0.0))), O.sensor(S.Sensor((0.3, 0.1, 3.0), 0.4)))
    for seed in range(5):
        f = _path(n, 100 * n + seed)
        co, lj = O.tree_coords(v, f)
        g = O.tree_path(v, f[0], f[-1], co)
        assert np.abs(g - f).max() < 1e-10
        assert np.isfinite(lj)


@pytest.mark.parametrize("n", [3, 5, 6, 9])
def test_tree_jacobian_finite_differences(oracle_lib, n):
    """log |det d(interior vertices) / d(zeta, t, phi)| = the returned log J."""
    O = oracle_lib
    v = O.tree_vref(O.source(S.Source((0.1, -0.2, 0.0))), O.sensor(S.Sensor((0.3, 0.1, 3.0), 0.4)))
    for seed in range(3):
        f = _path(n, 7 * n + seed, lateral=0.6)
        co, lj = O.tree_coords(v, f)
        dim = 3 * (n - 2)
        Jm = np.zeros((dim, dim))
        h = 1e-6
        for a in range(dim):
            m, q = 1 + a // 3, a % 3
            cp, cm = co.copy(), co.copy()
            cp[m, q] += h
            cm[m, q] -= h
            gp = O.tree_path(v, f[0], f[-1], cp)[1:-1].ravel()
            gm = O.tree_path(v, f[0], f[-1], cm)[1:-1].ravel()
            Jm[:, a] = (gp - gm) / (2 * h)
        sign, logdet = np.linalg.slogdet(Jm)
        assert sign != 0
        assert abs(logdet - lj) < 1e-5 * max(1.0, abs(lj)), (n, seed, logdet, lj)


def _rotate(p, a, b, ang):
    """Rotate points p about the axis through a and b by ang (Rodrigues)."""
    k = (b - a) / np.linalg.norm(b - a)
    v = p - a
    c, s = math.cos(ang), math.sin(ang)
    return a + v * c + np.cross(k, v) * s + np.outer(v @ k, k) * (1 - c)


def test_turning_one_vertex_turns_its_subtree(oracle_lib):
    O = oracle_lib
    v = O.tree_vref(O.source(S.Source((0.1, -0.2, 0.0))), O.sensor(S.Sensor((0.3, 0.1, 3.0), 0.4)))
    n = 17
    f = _path(n, 5, lateral=0.5)
    co, _ = O.tree_coords(v, f)
    for m in (8, 4, 12, 2):
        k, l, _ = O.tree_node(m, n)
        c2 = co.copy()
        c2[m, 2] += 0.7
        g = O.tree_path(v, f[0], f[-1], c2)
        sub = np.arange(k + 1, l)
        rot = _rotate(f[sub], f[k], f[l], 0.7)
        assert np.abs(g[sub] - rot).max() < 1e-10, m
        rest = np.setdiff1d(np.arange(n), sub)
        assert np.abs(g[rest] - f[rest]).max() < 1e-12


def _tree_run(**kw):
    return S.Run(within=S.WITHIN_TREE, **kw)


def test_tree_chain_single_scatter_sector_matches_quadrature(oracle_lib):
    """Cap 3: I = Z2 + Z3 exactly, with tree moves as the within-dimension moves."""
    O = oracle_lib
    sc = S.plain()
    sc.run = _tree_run(seed=sc.run.seed, burn_in=2000, sigma=0.6)
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 3)
    ch.run(60000)
    m, s, d = O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[0])
    I, se, _ = O.direct_estimate(ch.accumulators(), O.z2(m, s, d))
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(I - ref) < 3 * se, (I, se, ref)
    assert se / I < 0.015
    acc = ch.accumulators()
    rate = acc["acc"][:, 0].sum() / acc["prop"][:, 0].sum()
    assert 0.05 < rate < 0.95


def test_tree_chain_matches_forward_tracer_all_orders(oracle_lib):
    """Well-mixing scene: intensity and vertex-count split agree with Algorithm 1."""
    O = oracle_lib
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.0)
    src, sen = S.Source(), S.Sensor((0.0, 0.0, 1.5), 0.5)
    run = _tree_run(seed=4321, burn_in=3000, sigma=0.8)
    cap = 24
    ch = O.Chains(med, src, sen, run, 96, cap)
    H = np.zeros((96, cap + 1))
    ch.run(60000, n_hist=H)
    m, s, d = O.medium(med), O.source(src), O.sensor(sen)
    z2 = O.z2(m, s, d)
    I, se, _ = O.direct_estimate(ch.accumulators(), z2)
    tr = O.trace(m, s, d, 77, 4_000_000, max_scatter=cap - 2, hist=True)
    assert abs(I - tr["I"]) < 3 * math.hypot(se, tr["se"]), (I, se, tr["I"], tr["se"])
    h = H.sum(0)
    zc = z2 * h / h[2]
    for k in (3, 4, 5):
        assert abs(zc[k] / tr["hist"][k - 2] - 1) < 0.04, (k, zc[k], tr["hist"][k - 2])


# ---------------------------------------------------------------------------
# Full-path gradient (HMC) moves (section "Discussion"), pinned the same way.
# ---------------------------------------------------------------------------
def _hmc_run(**kw):
    return S.Run(within=S.WITHIN_HMC, **kw)


def test_hmc_small_steps_conserve_energy(oracle_lib):
    """With a tiny leapfrog step the Hamiltonian is conserved to O(eps^2), so
    HMC proposals are almost always accepted: this ties the gradient the
    leapfrog follows to the density the acceptance uses (a dropped term or a
    wrong sign in either shows up as rejections)."""
    O = oracle_lib
    sc = S.general_small(n_chains=32, n_steps=400)
    sc.run = _hmc_run(seed=11, burn_in=0, mala_step=2e-4, hmc_steps=5, init=S.INIT_STRAIGHT, init_k=8,
                      init_jitter=0.02)
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 32, 64)
    ch.run(400)
    acc = ch.accumulators()
    rate = acc["acc"][:, 0].sum() / acc["prop"][:, 0].sum()
    assert rate > 0.98, rate


def test_hmc_chain_single_scatter_sector_matches_quadrature(oracle_lib):
    O = oracle_lib
    sc = S.plain()
    sc.run = _hmc_run(seed=sc.run.seed, burn_in=2000, mala_step=0.03, hmc_steps=4)
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, 3)
    ch.run(40000)
    m, s, d = O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[0])
    I, se, _ = O.direct_estimate(ch.accumulators(), O.z2(m, s, d))
    ref = Q.z2_closed(1.0, 0.1, 2.2) + Q.z3(1.0, 0.1, 0.5, 5.0, 0.9)
    assert abs(I - ref) < 3 * se, (I, se, ref)
    assert se / I < 0.015


def test_hmc_chain_matches_forward_tracer_all_orders(oracle_lib):
    O = oracle_lib
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.0)
    src, sen = S.Source(), S.Sensor((0.0, 0.0, 1.5), 0.5)
    run = _hmc_run(seed=2468, burn_in=3000, mala_step=0.08, hmc_steps=5, sigma=0.1)
    cap = 24
    ch = O.Chains(med, src, sen, run, 96, cap)
    H = np.zeros((96, cap + 1))
    ch.run(30000, n_hist=H)
    m, s, d = O.medium(med), O.source(src), O.sensor(sen)
    z2 = O.z2(m, s, d)
    I, se, _ = O.direct_estimate(ch.accumulators(), z2)
    tr = O.trace(m, s, d, 77, 4_000_000, max_scatter=cap - 2, hist=True)
    assert abs(I - tr["I"]) < 3 * math.hypot(se, tr["se"]), (I, se, tr["I"], tr["se"])
    h = H.sum(0)
    zc = z2 * h / h[2]
    for k in (3, 4, 5):
        assert abs(zc[k] / tr["hist"][k - 2] - 1) < 0.05, (k, zc[k], tr["hist"][k - 2])


def _hmc_path(n, seed):
    xyz, _ = S.random_paths((0.0, 0.0, 0.0), (0.0, 0.0, 1.5), 0.5, 1, n, n, n, seed, lateral=0.2)
    return xyz[:, 0, :n].T.astype(np.float64)


def test_leapfrog_is_reversible_and_volume_preserving(oracle_lib):
    """The HMC map (x, p) -> (x', p') of the oracle: running it from (x', -p')
    returns to (x, -p), and its Jacobian determinant over the interior
    coordinates and momenta is 1 (finite differences) -- the two properties
    that make the Hamiltonian acceptance ratio exact."""
    O = oracle_lib
    med = S.Medium(lambda_s=1.0, lambda_a=5.0, g=0.6)
    m, s, d = O.medium(med), O.source(S.Source()), O.sensor(S.Sensor((0.0, 0.0, 1.5), 0.5))
    rng = np.random.default_rng(3)
    n = 5
    for seed in range(4, 200):   # a start whose trajectory stays where the density is positive
        x = _hmc_path(n, seed)
        p = rng.normal(size=(n, 3))
        x1, p1, lp1 = O.hmc_leapfrog(m, s, d, x, p, 0.01, 6)
        if np.isfinite(O.logp(m, s, d, x)) and np.isfinite(lp1):
            break
    assert np.isfinite(lp1)
    x2, p2, _ = O.hmc_leapfrog(m, s, d, x1, -p1, 0.01, 6)
    assert np.abs(x2 - x).max() < 1e-10 and np.abs(-p2[1:-1] - p[1:-1]).max() < 1e-9
    # volume preservation over (interior x, interior p)
    dim = 3 * (n - 2)

    def flat(xx, pp):
        return np.concatenate([xx[1:-1].ravel(), pp[1:-1].ravel()])

    z0 = flat(x, p)
    Jm = np.zeros((2 * dim, 2 * dim))
    h = 1e-6
    for a in range(2 * dim):
        out = []
        for sgn in (1, -1):
            z = z0.copy()
            z[a] += sgn * h
            xx, pp = x.copy(), p.copy()
            xx[1:-1] = z[:dim].reshape(-1, 3)
            pp[1:-1] = z[dim:].reshape(-1, 3)
            xo, po, _ = O.hmc_leapfrog(m, s, d, xx, pp, 0.01, 6)
            out.append(flat(xo, po))
        Jm[:, a] = (out[0] - out[1]) / (2 * h)
    assert abs(np.linalg.det(Jm) - 1.0) < 1e-5


def test_tree_moves_balance_a_toy_target(oracle_lib):
    """Tree-coordinate moves with births and deaths on the toy product target
    (P(n) proportional to w_n, interior vertices Gaussian about the axis):
    the vertex-count distribution comes out right, which a wrong tree
    Jacobian would shift through the vertices' spread."""
    import ctypes as C
    O = oracle_lib
    cap = 6
    w = np.zeros(cap + 1)
    w[2:] = [1.0, 2.0, 1.5, 0.7, 0.3]
    sc = S.plain()
    sc.run = S.Run(seed=sc.run.seed, burn_in=2000, within=S.WITHIN_TREE, sigma=0.8)
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, 64, cap)
    ch.r.toy_s = 0.1
    ch.r.toy_w = w.ctypes.data_as(C.POINTER(C.c_double))
    H = np.zeros((64, cap + 1))
    ch.run(100_000, n_hist=H)
    P = H / H.sum(axis=1, keepdims=True)
    mean, se = P.mean(axis=0), P.std(axis=0, ddof=1) / math.sqrt(64)
    ref = w / w.sum()
    for k in range(2, cap + 1):
        assert abs(mean[k] - ref[k]) < 4 * se[k], (k, mean[k], ref[k], se[k])
    assert np.abs(mean - ref).max() < 0.015
