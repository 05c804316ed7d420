"""Independent numerical integrals used as pins for the oracle (numpy only).

Nothing here calls the oracle or the CUDA library.  Homogeneous medium,
isotropic point source at the origin, sensor of radius R centred at (0, 0, D),
detection probability 1, Henyey-Greenstein phase function (section
"Implementation" setting).  Z2 and Z3 are the zero- and single-scattering
parts of the path integral (paths with n = 2 and n = 3 vertices).
"""
from __future__ import annotations

import math

import numpy as np


def hg_per_sr(c, g):
    """Henyey-Greenstein density per steradian (Eq. angular_scattering with f_SL = 0) / (2 pi)."""
    return 0.5 * (1.0 - g * g) * (1.0 + g * g - 2.0 * g * c) ** -1.5 / (2.0 * math.pi)


def z2_closed(D, R, c_ext):
    """Direct part: 1/2 int_{cos th_max}^1 exp(-c r(w)) dw, r = first hit distance."""
    from scipy.integrate import quad
    wmin = math.sqrt(1.0 - (R / D) ** 2)

    def f(w):
        s2 = max(1.0 - w * w, 0.0)
        r = D * w - math.sqrt(max(R * R - D * D * s2, 0.0))
        return math.exp(-c_ext * r)
    # substitution w = wmin + (1 - wmin) v^2 removes the rim square root
    val, _ = quad(lambda v: f(wmin + (1 - wmin) * v * v) * 2 * (1 - wmin) * v, 0.0, 1.0, epsabs=0, epsrel=1e-12,
                  limit=200)
    return 0.5 * val


def _gl(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def z3(D, R, lam_s, lam_a, g, n_alpha=(64, 160), n_l=(64, 96), n_v=40, n_phi=48):
    """Single-scattering part: int d^3f1 int dA(f2) p(f0, f1, f2).

    Outer: direction alpha of f1 from the axis and distance l0 from the source
    (rays that hit the sensor stop at the hit: the first segment may not touch
    the ball); inner: directions from f1 over the visible cap, with the
    rim square root removed by theta = theta_c (1 - v^2).
    """
    b = 1.0 / lam_s
    cext = 1.0 / lam_s + 1.0 / lam_a
    a_hit = math.asin(R / D)
    total = 0.0
    for (lo, hi, na, nl_) in ((0.0, a_hit, n_alpha[0], n_l[0]), (a_hit, math.pi, n_alpha[1], n_l[1])):
        # cosine-graded nodes near the sensor direction
        al, wa = _gl(lo, hi, na)
        for alpha, w_alpha in zip(al, wa):
            sa, ca = math.sin(alpha), math.cos(alpha)
            if alpha < a_hit:
                lmax = D * ca - math.sqrt(max(R * R - D * D * sa * sa, 0.0))
                l0, wl = _gl(0.0, lmax, nl_)
            else:
                # exponential map of [0, inf): l = -log(1 - u)/cext
                u, wu = _gl(0.0, 1.0 - 1e-13, nl_)
                l0 = -np.log1p(-u) / cext
                wl = wu / (cext * (1.0 - u))
            om0 = np.array([sa, 0.0, ca])
            f1 = l0[:, None] * om0[None, :]                      # (L, 3)
            cvec = np.array([0.0, 0.0, D])
            dvec = cvec[None, :] - f1
            D1 = np.linalg.norm(dvec, axis=1)
            ok = D1 > R
            u1 = dvec / D1[:, None]
            thc = np.arcsin(np.clip(R / D1, 0, 1))
            # basis perpendicular to u1
            e1 = np.cross(u1, np.array([0.0, 1.0, 0.0]))
            e1 /= np.linalg.norm(e1, axis=1)[:, None]
            e2 = np.cross(u1, e1)
            v, wv = _gl(0.0, 1.0, n_v)
            phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
            th = thc[:, None] * (1.0 - v[None, :] ** 2)               # (L, V)
            jac = 2.0 * thc[:, None] * v[None, :]                      # d theta / dv
            st, ct = np.sin(th), np.cos(th)
            disc = np.maximum(R * R - (D1[:, None] * st) ** 2, 0.0)
            l1 = D1[:, None] * ct - np.sqrt(disc)                      # (L, V)
            cp, sp = np.cos(phi), np.sin(phi)
            # omega1 = ct u1 + st (cp e1 + sp e2); cos(scatter) = om0 . omega1
            c_u = u1 @ om0
            c_e1 = e1 @ om0
            c_e2 = e2 @ om0
            cs = ct[:, :, None] * c_u[:, None, None] + st[:, :, None] * (
                cp[None, None, :] * c_e1[:, None, None] + sp[None, None, :] * c_e2[:, None, None])
            inner = (hg_per_sr(cs, g) * (st * jac * np.exp(-cext * l1))[:, :, None]).sum(axis=2) * (2 * math.pi / n_phi)
            inner = (inner * wv[None, :]).sum(axis=1)                  # (L,)
            inner = np.where(ok, inner, 0.0)
            outer = (np.exp(-cext * l0) * b * inner * wl).sum()
            total += 2 * math.pi * math.sin(alpha) * w_alpha * outer / (4 * math.pi)
    return total


def spectrum_integral(spectrum_nm, spectrum, lambda_s, lambda_a, lambda0, k_s, k_a, fun, nodes=6):
    """int S(l) fun(lambda_s(l), lambda_a(l), l) dl: S the piecewise-linear
    spectrum normalised over its table, lambda_s(l) = lambda_s (l/lambda0)^k_s
    and lambda_a(l) = lambda_a (l/lambda0)^k_a (coefficients ~ l^-k);
    Gauss-Legendre with `nodes` points on every interval of the table."""
    nm, sp = np.asarray(spectrum_nm, float), np.asarray(spectrum, float)
    area = np.sum(0.5 * np.diff(nm) * (sp[:-1] + sp[1:]))
    x, w = np.polynomial.legendre.leggauss(nodes)
    tot = 0.0
    for i in range(len(nm) - 1):
        a, b = nm[i], nm[i + 1]
        for xi, wi in zip(x, w):
            lam = 0.5 * (a + b) + 0.5 * (b - a) * xi
            s_val = (sp[i] + (sp[i + 1] - sp[i]) * (lam - a) / (b - a)) / area
            tot += 0.5 * (b - a) * wi * s_val * fun(lambda_s * (lam / lambda0) ** k_s,
                                                    lambda_a * (lam / lambda0) ** k_a, lam)
    return tot
