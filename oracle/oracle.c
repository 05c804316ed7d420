/*
 * FP64 CPU oracle for path-integral RJMCMC light transport (arXiv:1811.04156).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * bench's CPU-baseline / reference legs.  The CUDA product path never uses it.
 *
 * Plain and slow on purpose: every proposal recomputes log p over the whole
 * path in double precision, directly from the paper's factor definitions.
 *
 * Readings of passages that the paper leaves silent, ambiguous or garbled:
 *   Q1  acceptance of a birth is Green's form p(y)/p(x) * P(death)/P(birth) * J/q;
 *       a death uses the reciprocal of the birth factor of the reverse move.
 *   Q2  tau is the optical depth: segment length times the mean coefficient.
 *   Q3  the phase density per steradian is sigma(cos theta) / (2 pi).
 *   Q4  the final segment also carries its survival exp(-tau).
 *   Q5  the bispherical insertion map is centred on the segment midpoint.
 *   Q7  the insertion concentration beta uses b at the segment midpoint.
 *   Q9  birth at the vertex cap and death at n = 2 are proposed and rejected.
 *   Q11 end-vertex moves are vMF steps on the sensor sphere.
 *   Q12 interior segments may not touch the sensor ball; the final segment must
 *       arrive from outside (cos Phi > 0).
 *   Q13 the tracer's initial log-weight is 0 (w = 1).
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define NEG_INF (-INFINITY)

/* ------------------------------------------------------------------------ */
/* Small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static void copy3(const double* a, double* o) { o[0] = a[0]; o[1] = a[1]; o[2] = a[2]; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 Philox S-box with a Weyl  */
/* key schedule.                                                             */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0, 1) from the top 23 bits: ((x >> 9) + 1/2) * 2^-23. */
double or_u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* floor of the 23-bit fraction times m, computed in integers. */
static uint32_t index_draw(uint32_t x, uint32_t m) { return (uint32_t)(((uint64_t)(x >> 9) * m) >> 23); }

static void draw_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* Orthonormal basis completing a unit vector n (Duff et al., "Building an
 * Orthonormal Basis, Revisited", JCGT 2017). */
void or_onb(const double n[3], double e1[3], double e2[3]) {
  double sign = copysign(1.0, n[2]);
  double a = -1.0 / (sign + n[2]);
  double b = n[0] * n[1] * a;
  e1[0] = 1.0 + sign * n[0] * n[0] * a; e1[1] = sign * b; e1[2] = -sign * n[0];
  e2[0] = b; e2[1] = sign + n[1] * n[1] * a; e2[2] = -n[1];
}

/* ------------------------------------------------------------------------ */
/* Medium: a(x), b(x) and optical depths (Eq. b_depth_def)                    */
/* ------------------------------------------------------------------------ */
static int layer_index(const or_medium* m, double z) {
  double f = floor((z - m->z0) / m->dz);
  if (f < 0.0) return 0;
  if (f > (double)(m->n_layers - 1)) return m->n_layers - 1;
  return (int)f;
}

double or_b_at(const or_medium* m, const double x[3]) {
  if (m->kind == OR_HOMOGENEOUS) return 1.0 / m->lambda_s;
  return 1.0 / m->lambda_s_layers[layer_index(m, x[2])];
}

double or_a_at(const or_medium* m, const double x[3]) {
  if (m->kind == OR_HOMOGENEOUS) return 1.0 / m->lambda_a;
  return 1.0 / m->lambda_a_layers[layer_index(m, x[2])];
}

/* tau_a, tau_b of the straight segment P -> Q: the line integrals of a and b
 * along it (Eq. b_depth_def with the segment length restored, reading Q2).
 * Layered media: sum over the pieces between horizontal layer boundaries. */
void or_segment_depths(const or_medium* m, const double P[3], const double Q[3],
                       double* tau_a, double* tau_b) {
  double r[3];
  sub3(Q, P, r);
  double ell = norm3(r);
  if (m->kind == OR_HOMOGENEOUS) {
    *tau_a = ell / m->lambda_a;
    *tau_b = ell / m->lambda_s;
    return;
  }
  /* fractions u in [0,1] where the segment crosses layer boundaries */
  double cuts[2048];
  int nc = 0;
  cuts[nc++] = 0.0;
  double zP = P[2], zQ = Q[2];
  if (zQ != zP) {
    if (zQ > zP) {
      for (int j = 1; j < m->n_layers && nc < 2046; ++j) {
        double zb = m->z0 + j * m->dz;
        if (zb > zP && zb < zQ) cuts[nc++] = (zb - zP) / (zQ - zP);
      }
    } else {
      for (int j = m->n_layers - 1; j >= 1 && nc < 2046; --j) {
        double zb = m->z0 + j * m->dz;
        if (zb < zP && zb > zQ) cuts[nc++] = (zb - zP) / (zQ - zP);
      }
    }
  }
  cuts[nc++] = 1.0;
  double ta = 0.0, tb = 0.0;
  for (int i = 0; i + 1 < nc; ++i) {
    double um = 0.5 * (cuts[i] + cuts[i + 1]);
    double x[3] = {P[0] + um * r[0], P[1] + um * r[1], P[2] + um * r[2]};
    double len = ell * (cuts[i + 1] - cuts[i]);
    ta += or_a_at(m, x) * len;
    tb += or_b_at(m, x) * len;
  }
  *tau_a = ta;
  *tau_b = tb;
}

/* Does the closed segment P -> Q touch the closed ball (c, R)? */
int or_segment_hits_ball(const double P[3], const double Q[3], const double c[3], double R) {
  double r[3], w[3];
  sub3(Q, P, r);
  sub3(c, P, w);
  double rr = dot3(r, r);
  double t = rr > 0.0 ? dot3(w, r) / rr : 0.0;
  if (t < 0.0) t = 0.0;
  if (t > 1.0) t = 1.0;
  double p[3] = {P[0] + t * r[0] - c[0], P[1] + t * r[1] - c[1], P[2] + t * r[2] - c[2]};
  return dot3(p, p) <= R * R;
}

/* ------------------------------------------------------------------------ */
/* Angular factors                                                          */
/* ------------------------------------------------------------------------ */

/* kappa_eq solves coth(k) - 1/k = Gamma (appendix, dimension matching
 * transformation): Newton iteration on the Langevin function. */
double or_kappa_eq(double G) {
  if (G <= 0.0) return 0.0;
  double k = 3.0 * G / (1.0 - G * G); /* starting point */
  if (k < 1e-3) k = 1e-3;
  for (int it = 0; it < 200; ++it) {
    double f = 1.0 / tanh(k) - 1.0 / k - G;
    double sh = sinh(k);
    double df = -1.0 / (sh * sh) + 1.0 / (k * k);
    if (k > 300.0) df = 1.0 / (k * k);
    double step = f / df;
    double kn = k - step;
    if (kn <= 0.0) kn = 0.5 * k;
    if (fabs(kn - k) < 1e-15 * k) { k = kn; break; }
    k = kn;
  }
  return k;
}

/* sigma(cos theta), normalised over cos theta in [-1, 1]
 * (Eq. angular_scattering with the simplified-Liu and Henyey-Greenstein components). */
static double sigma_cos(const or_medium* m, double c) {
  double G = m->g;
  double hg = 0.5 * (1.0 - G * G) * pow(1.0 + G * G - 2.0 * G * c, -1.5);
  double val = (1.0 - m->f_sl) * hg;
  if (m->f_sl > 0.0) {
    double alpha = 2.0 / (1.0 / G - 1.0);
    double sl = 0.5 * ((1.0 + G) / (1.0 - G)) * pow(0.5 * (1.0 + c), alpha);
    val += m->f_sl * sl;
  }
  return val;
}

double or_log_sigma_cos(const or_medium* m, double c) { return log(sigma_cos(m, c)); }

/* Density per steradian of the scattered direction (reading Q3). */
double or_log_sigma(const or_medium* m, double c) { return log(sigma_cos(m, c)) - log(2.0 * M_PI); }

/* d sigma / d cos theta divided by sigma. */
static double dlog_sigma_dc(const or_medium* m, double c) {
  double G = m->g;
  double den = 1.0 + G * G - 2.0 * G * c;
  double hg = 0.5 * (1.0 - G * G) * pow(den, -1.5);
  double dhg = hg * 3.0 * G / den;
  double val = (1.0 - m->f_sl) * hg, dval = (1.0 - m->f_sl) * dhg;
  if (m->f_sl > 0.0) {
    double alpha = 2.0 / (1.0 / G - 1.0);
    double v = 0.5 * (1.0 + c);
    double sl = 0.5 * ((1.0 + G) / (1.0 - G)) * pow(v, alpha);
    val += m->f_sl * sl;
    dval += m->f_sl * sl * alpha / (2.0 * v);
  }
  return dval / val;
}

/* d log sigma / d Gamma at fixed cos theta. */
static double dlog_sigma_dG(const or_medium* m, double c) {
  double G = m->g;
  double den = 1.0 + G * G - 2.0 * G * c;
  double hg = 0.5 * (1.0 - G * G) * pow(den, -1.5);
  double dl_hg = -2.0 * G / (1.0 - G * G) - 3.0 * (G - c) / den;
  double val = (1.0 - m->f_sl) * hg, dval = (1.0 - m->f_sl) * hg * dl_hg;
  if (m->f_sl > 0.0) {
    double alpha = 2.0 / (1.0 / G - 1.0);
    double v = 0.5 * (1.0 + c);
    double sl = 0.5 * ((1.0 + G) / (1.0 - G)) * pow(v, alpha);
    double dl_sl = 2.0 / (1.0 - G * G) + 2.0 * log(v) / ((1.0 - G) * (1.0 - G));
    val += m->f_sl * sl;
    dval += m->f_sl * sl * dl_sl;
  }
  return dval / val;
}

/* Emission density per steradian (Eq. emission_dist; isotropic when kappa = 0). */
double or_log_emission(const or_source* s, const double rhat[3]) {
  if (s->emission == OR_EMIT_ISOTROPIC || s->kappa <= 0.0) return -log(4.0 * M_PI);
  double k = s->kappa;
  return log(k) - log(4.0 * M_PI * sinh(k)) + k * dot3(rhat, s->dir);
}

/* Detection probability rho (Eq. detection_prob), or 1. */
double or_log_rho(const or_sensor* d, const double nu[3]) {
  if (d->rho == OR_RHO_ONE) return 0.0;
  double x = dot3(nu, d->rho_hat);
  return log(exp(3.0 * x - 1.0) / cosh(2.0 * x + 0.7));
}

/* ------------------------------------------------------------------------ */
/* Path density: p = p_i * prod p_v * p_f (appendix, path probability         */
/* distribution; Eqs. emission_dist, intervtx, b_depth_def, detection_prob).  */
/* ------------------------------------------------------------------------ */
double or_logp(const or_medium* m, const or_source* s, const or_sensor* d,
               int n, const double* f) {
  if (n < 2) return NEG_INF;
  double lp = 0.0;
  double rhat_prev[3] = {0, 0, 0};
  for (int k = 0; k <= n - 2; ++k) {
    double r[3];
    sub3(f + 3 * (k + 1), f + 3 * k, r);
    double ell = norm3(r);
    if (!(ell > 0.0)) return NEG_INF;
    double rhat[3] = {r[0] / ell, r[1] / ell, r[2] / ell};
    /* segment survival and the 1/|r|^2 of the next vertex's factor */
    double ta, tb;
    or_segment_depths(m, f + 3 * k, f + 3 * (k + 1), &ta, &tb);
    lp += -ta - tb - 2.0 * log(ell);
    /* non-final segments may not touch the sensor (reading Q12) */
    if (k <= n - 3 && or_segment_hits_ball(f + 3 * k, f + 3 * (k + 1), d->c, d->R)) return NEG_INF;
    if (k == 0) {
      lp += or_log_emission(s, rhat);                 /* p_i */
    } else {
      lp += log(or_b_at(m, f + 3 * k));               /* p_v at vertex k */
      lp += or_log_sigma(m, dot3(rhat_prev, rhat));
    }
    copy3(rhat, rhat_prev);
  }
  /* p_f: max(0, -rhat . nu) rho(f) (the 1/|r|^2 is in the segment term) */
  double nu[3];
  sub3(f + 3 * (n - 1), d->c, nu);
  double nn = norm3(nu);
  nu[0] /= nn; nu[1] /= nn; nu[2] /= nn;
  double cphi = -dot3(rhat_prev, nu);
  if (!(cphi > 0.0)) return NEG_INF;
  lp += log(cphi) + or_log_rho(d, nu);
  return lp;
}

/* d (r_hat . v) / d(end point of r), with r_hat = r/|r|. */
static void drhat_dot(const double rhat[3], double ell, const double v[3], double out[3]) {
  double rv = dot3(rhat, v);
  for (int i = 0; i < 3; ++i) out[i] = (v[i] - rv * rhat[i]) / ell;
}

/* Analytic gradient of or_logp with respect to every vertex coordinate. */
double or_grad_logp(const or_medium* m, const or_source* s, const or_sensor* d,
                    int n, const double* f, double* grad) {
  double lp = or_logp(m, s, d, n, f);
  for (int i = 0; i < 3 * n; ++i) grad[i] = 0.0;
  if (!isfinite(lp)) return lp;
  size_t nseg = (size_t)(n > 1 ? n - 1 : 1);
  double* rh = (double*)malloc(sizeof(double) * 3 * nseg);
  double* el = (double*)malloc(sizeof(double) * nseg);
  for (int k = 0; k <= n - 2; ++k) {
    double r[3];
    sub3(f + 3 * (k + 1), f + 3 * k, r);
    el[k] = norm3(r);
    for (int i = 0; i < 3; ++i) rh[3 * k + i] = r[i] / el[k];
  }
  /* segment terms -tau - 2 log ell */
  for (int k = 0; k <= n - 2; ++k) {
    const double* P = f + 3 * k;
    const double* Q = f + 3 * (k + 1);
    const double* rhat = rh + 3 * k;
    double dQ[3], dP[3];
    if (m->kind == OR_HOMOGENEOUS) {
      double c = 1.0 / m->lambda_a + 1.0 / m->lambda_s;
      for (int i = 0; i < 3; ++i) { dQ[i] = c * rhat[i]; dP[i] = -c * rhat[i]; }
    } else {
      /* tau = ell * cbar, cbar = mean of c(z) over [zP, zQ] */
      double ta, tb;
      or_segment_depths(m, P, Q, &ta, &tb);
      double cbar = (ta + tb) / el[k];
      for (int i = 0; i < 3; ++i) { dQ[i] = cbar * rhat[i]; dP[i] = -cbar * rhat[i]; }
      int lP = layer_index(m, P[2]), lQ = layer_index(m, Q[2]);
      if (lP != lQ) {
        double cP = or_a_at(m, P) + or_b_at(m, P);
        double cQ = or_a_at(m, Q) + or_b_at(m, Q);
        double dz = Q[2] - P[2];
        dQ[2] += el[k] * (cQ - cbar) / dz;
        dP[2] += el[k] * (cbar - cP) / dz;
      }
    }
    for (int i = 0; i < 3; ++i) {
      grad[3 * (k + 1) + i] += -dQ[i] - 2.0 * rhat[i] / el[k];
      grad[3 * k + i] += -dP[i] + 2.0 * rhat[i] / el[k];
    }
  }
  /* emission */
  if (s->emission == OR_EMIT_VMF && s->kappa > 0.0) {
    double t[3];
    drhat_dot(rh, el[0], s->dir, t);
    for (int i = 0; i < 3; ++i) { grad[3 + i] += s->kappa * t[i]; grad[i] -= s->kappa * t[i]; }
  }
  /* interior angle factors */
  for (int k = 1; k <= n - 2; ++k) {
    const double* a = rh + 3 * (k - 1);
    const double* b = rh + 3 * k;
    double c = dot3(a, b);
    double w = dlog_sigma_dc(m, c);
    double ta[3], tb[3];
    drhat_dot(a, el[k - 1], b, ta); /* d c / d f_k through a (a's end) */
    drhat_dot(b, el[k], a, tb);     /* d c / d f_{k+1} through b (b's end) */
    for (int i = 0; i < 3; ++i) {
      grad[3 * (k - 1) + i] -= w * ta[i];
      grad[3 * k + i] += w * (ta[i] - tb[i]);
      grad[3 * (k + 1) + i] += w * tb[i];
    }
  }
  /* sensor term log(-rhat . nu) + log rho(nu) */
  {
    int k = n - 2;
    const double* rhat = rh + 3 * k;
    double nu[3];
    sub3(f + 3 * (n - 1), d->c, nu);
    double dn = norm3(nu);
    for (int i = 0; i < 3; ++i) nu[i] /= dn;
    double u = -dot3(rhat, nu);
    double t1[3], t2[3];
    drhat_dot(rhat, el[k], nu, t1); /* d(rhat.nu)/d f_{n-1} via rhat */
    drhat_dot(nu, dn, rhat, t2);    /* d(rhat.nu)/d f_{n-1} via nu */
    for (int i = 0; i < 3; ++i) {
      grad[3 * (n - 1) + i] += -(t1[i] + t2[i]) / u;
      grad[3 * k + i] += t1[i] / u;
    }
    if (d->rho == OR_RHO_PAPER) {
      double x = dot3(nu, d->rho_hat);
      double dl = 3.0 - 2.0 * tanh(2.0 * x + 0.7);
      double t3[3];
      drhat_dot(nu, dn, d->rho_hat, t3);
      for (int i = 0; i < 3; ++i) grad[3 * (n - 1) + i] += dl * t3[i];
    }
  }
  free(rh);
  free(el);
  return lp;
}

/* Score d log p / d theta (calibration gradients).  Homogeneous:
 * theta = (lambda_s, lambda_a, Gamma); layered: (lambda_s[l], lambda_a[l]). */
int or_score(const or_medium* m, const or_source* s, const or_sensor* d,
             int n, const double* f, double* score) {
  (void)s; (void)d;
  if (m->kind == OR_HOMOGENEOUS) {
    double L = 0.0, sg = 0.0;
    double rprev[3] = {0, 0, 0};
    for (int k = 0; k <= n - 2; ++k) {
      double r[3];
      sub3(f + 3 * (k + 1), f + 3 * k, r);
      double ell = norm3(r);
      L += ell;
      double rhat[3] = {r[0] / ell, r[1] / ell, r[2] / ell};
      if (k >= 1) sg += dlog_sigma_dG(m, dot3(rprev, rhat));
      copy3(rhat, rprev);
    }
    double ls = m->lambda_s, la = m->lambda_a;
    score[0] = L / (ls * ls) - (double)(n - 2) / ls;
    score[1] = L / (la * la);
    score[2] = sg;
    return 3;
  }
  int nl = m->n_layers;
  for (int i = 0; i < 2 * nl; ++i) score[i] = 0.0;
  /* segment lengths per layer */
  for (int k = 0; k <= n - 2; ++k) {
    const double* P = f + 3 * k;
    const double* Q = f + 3 * (k + 1);
    /* per-layer length: evaluate the depth integral with unit coefficient of a
     * single layer at a time (plain, slow) */
    double r[3];
    sub3(Q, P, r);
    double ell = norm3(r);
    double zP = P[2], zQ = Q[2];
    for (int l = 0; l < nl; ++l) {
      double lo = (l == 0) ? -INFINITY : m->z0 + l * m->dz;
      double hi = (l == nl - 1) ? INFINITY : m->z0 + (l + 1) * m->dz;
      double len;
      if (zQ == zP) {
        len = (zP >= lo && zP < hi) ? ell : 0.0;
      } else {
        double z1 = fmin(zP, zQ), z2 = fmax(zP, zQ);
        double a = fmax(z1, lo), b = fmin(z2, hi);
        len = (b > a) ? ell * (b - a) / (z2 - z1) : 0.0;
      }
      double lsl = m->lambda_s_layers[l], lal = m->lambda_a_layers[l];
      score[l] += len / (lsl * lsl);
      score[nl + l] += len / (lal * lal);
    }
  }
  for (int k = 1; k <= n - 2; ++k) {
    int l = layer_index(m, f[3 * k + 2]);
    score[l] -= 1.0 / m->lambda_s_layers[l];
  }
  return 2 * nl;
}

/* ------------------------------------------------------------------------ */
/* Dimension matching transformation (appendix): bispherical coordinates     */
/* (s, t, phi) about the foci f_k, f_{k+1}, centred at their midpoint (Q5).   */
/* ------------------------------------------------------------------------ */
void or_bisph_point(const double fk[3], const double fk1[3], double s, double t, double phi,
                    double out[3]) {
  double r[3];
  sub3(fk1, fk, r);
  double ell = norm3(r);
  double gamma = 0.5 * ell;
  double rhat[3] = {r[0] / ell, r[1] / ell, r[2] / ell};
  double xi[3], ze[3];
  or_onb(rhat, xi, ze);
  double den = cosh(t) - cos(s);
  for (int i = 0; i < 3; ++i) {
    double mid = 0.5 * (fk[i] + fk1[i]);
    out[i] = mid + gamma * (rhat[i] * sinh(t) + (xi[i] * cos(phi) + ze[i] * sin(phi)) * sin(s)) / den;
  }
}

/* Inverse map: t = ln(d1/d2), s = angle at f between the two foci. */
void or_bisph_coords(const double fk[3], const double fk1[3], const double f[3],
                     double* s, double* t, double* phi) {
  double a[3], b[3];
  sub3(fk, f, a);
  sub3(fk1, f, b);
  double d1 = norm3(a), d2 = norm3(b);
  double cs = dot3(a, b) / (d1 * d2);
  if (cs > 1.0) cs = 1.0;
  if (cs < -1.0) cs = -1.0;
  *s = acos(cs);
  *t = log(d1 / d2);
  double r[3];
  sub3(fk1, fk, r);
  double ell = norm3(r);
  double rhat[3] = {r[0] / ell, r[1] / ell, r[2] / ell};
  double xi[3], ze[3];
  or_onb(rhat, xi, ze);
  double v[3];
  for (int i = 0; i < 3; ++i) v[i] = f[i] - 0.5 * (fk[i] + fk1[i]);
  *phi = atan2(dot3(v, ze), dot3(v, xi));
  if (*phi < 0.0) *phi += 2.0 * M_PI;
}

/* log J(s, t, phi) = 3 log(gamma / (cosh t - cos s)) + log sin s. */
double or_log_bisph_jacobian(double gamma, double s, double t) {
  return 3.0 * log(gamma / (cosh(t) - cos(s))) + log(sin(s));
}

/* log q(s) = log(beta e^{-beta cos s} sin s / (2 sinh beta)). */
double or_log_q_s(double beta, double s) {
  return log(beta) - beta * cos(s) + log(sin(s)) - log(2.0 * sinh(beta));
}

/* log q(t) = -log(2 + 2 cosh t). */
double or_log_q_t(double t) { return -log(2.0 + 2.0 * cosh(t)); }

/* Insertion concentration beta (appendix; reading Q7: b at the midpoint). */
static double insertion_beta(const or_medium* m, const or_run* r, double kappa_eq,
                             const double fk[3], const double fk1[3]) {
  double mid[3] = {0.5 * (fk[0] + fk1[0]), 0.5 * (fk[1] + fk1[1]), 0.5 * (fk[2] + fk1[2])};
  double diff[3];
  sub3(fk1, fk, diff);
  double gamma = 0.5 * norm3(diff);
  double beta = kappa_eq + 0.5 * (gamma * or_b_at(m, mid) - 1.0);
  return beta < r->beta_min ? r->beta_min : beta;
}

/* log of q(s) q(t) q(phi) / J for the vertex f placed between fk and fk1:
 * the density of the inserted vertex per unit volume. */
static double log_insert_density(const or_medium* m, const or_run* r, double kappa_eq,
                                 const double fk[3], const double fk1[3], const double f[3]) {
  double s, t, phi;
  or_bisph_coords(fk, fk1, f, &s, &t, &phi);
  double diff[3];
  sub3(fk1, fk, diff);
  double gamma = 0.5 * norm3(diff);
  double beta = insertion_beta(m, r, kappa_eq, fk, fk1);
  return or_log_q_s(beta, s) + or_log_q_t(t) - log(2.0 * M_PI) - or_log_bisph_jacobian(gamma, s, t);
}

/* ------------------------------------------------------------------------ */
/* Tree coordinates (appendix "Path space coordinate system"; the frames     */
/* follow the inherited-axes rule: a child's eta is its parent's eta turned  */
/* by the parent's phi, i.e. the normal of the parent's triangle).           */
/* ------------------------------------------------------------------------ */
void or_tree_node(int m, int n, int* k, int* l, int* parent) {
  int kk = 0, ll = n - 1, p = -1;
  for (;;) {
    int mid = (kk + ll) / 2;
    if (mid == m) break;
    p = mid;
    if (m < mid) ll = mid; else kk = mid;
  }
  *k = kk;
  *l = ll;
  *parent = p;
}

void or_tree_vref(const or_source* s, const or_sensor* d, double v_ref[3]) {
  double a[3], e2[3];
  sub3(d->c, s->pos, a);
  double la = norm3(a);
  for (int i = 0; i < 3; ++i) a[i] /= la;
  or_onb(a, v_ref, e2);
}

static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Unit axis e, half focal distance gamma and frame (xi, eta) of node m. */
static void tree_frame(const double v_ref[3], int m, int n, const double* f, double e[3], double* gamma,
                       double xi[3], double eta[3]) {
  int k, l, p;
  or_tree_node(m, n, &k, &l, &p);
  double r[3];
  sub3(f + 3 * l, f + 3 * k, r);
  double ell = norm3(r);
  *gamma = 0.5 * ell;
  for (int i = 0; i < 3; ++i) e[i] = r[i] / ell;
  int have = 0;
  if (p >= 0) {
    int kp, lp, pp;
    or_tree_node(p, n, &kp, &lp, &pp);
    double ep[3], rho[3], nrm[3];
    sub3(f + 3 * lp, f + 3 * kp, ep);
    double lep = norm3(ep);
    for (int i = 0; i < 3; ++i) {
      ep[i] /= lep;
      rho[i] = f[3 * p + i] - 0.5 * (f[3 * kp + i] + f[3 * lp + i]);
    }
    cross3(ep, rho, nrm);
    double nn = norm3(nrm), nr = norm3(rho);
    if (nn > 1e-9 * nr && nn > 0.0) {
      /* remove the rounding component along e, then normalise */
      double de = dot3(nrm, e);
      for (int i = 0; i < 3; ++i) nrm[i] -= de * e[i];
      nn = norm3(nrm);
      for (int i = 0; i < 3; ++i) eta[i] = nrm[i] / nn;
      cross3(eta, e, xi);
      have = 1;
    }
  }
  if (!have) {
    /* root, or a parent on its own axis: xi from v_ref */
    double dv = dot3(v_ref, e), x[3];
    for (int i = 0; i < 3; ++i) x[i] = v_ref[i] - dv * e[i];
    double nx = norm3(x);
    for (int i = 0; i < 3; ++i) xi[i] = x[i] / nx;
    cross3(e, xi, eta);
  }
}

double or_tree_coords(const double v_ref[3], int n, const double* f, double* coords) {
  double lj = 0.0;
  for (int m = 1; m <= n - 2; ++m) {
    int k, l, p;
    or_tree_node(m, n, &k, &l, &p);
    double e[3], xi[3], eta[3], gamma;
    tree_frame(v_ref, m, n, f, e, &gamma, xi, eta);
    double a[3], b[3];
    sub3(f + 3 * k, f + 3 * m, a);
    sub3(f + 3 * l, f + 3 * m, b);
    double d1 = norm3(a), d2 = norm3(b);
    /* 1 +- cos s from |a/d1 +- b/d2|^2 / 2: accurate near s = 0 and s = pi */
    double sp = 0.0, sm = 0.0;
    for (int i = 0; i < 3; ++i) {
      double u = a[i] / d1, v = b[i] / d2;
      sp += (u + v) * (u + v);
      sm += (u - v) * (u - v);
    }
    double opc = 0.5 * sp, omc = 0.5 * sm;
    double zeta = 0.5 * log(opc / omc);
    double t = log(d1 / d2);
    double rho[3];
    for (int i = 0; i < 3; ++i) rho[i] = f[3 * m + i] - 0.5 * (f[3 * k + i] + f[3 * l + i]);
    double phi = atan2(dot3(rho, eta), dot3(rho, xi));
    coords[3 * m + 0] = zeta;
    coords[3 * m + 1] = t;
    coords[3 * m + 2] = phi;
    double sins = sqrt(opc * omc);  /* sin s = sqrt((1 + cos s)(1 - cos s)) */
    lj += 3.0 * log(d1 * d2 / (2.0 * gamma)) + 2.0 * log(sins);
  }
  return lj;
}

void or_tree_path(const double v_ref[3], int n, const double* coords, double* f) {
  /* nodes by depth: a node's foci and parent are shallower */
  int maxd = 0;
  for (int m = 1; m <= n - 2; ++m) {
    int k = 0, l = n - 1, d = 0;
    for (;;) {
      int mid = (k + l) / 2;
      if (mid == m) break;
      if (m < mid) l = mid; else k = mid;
      ++d;
    }
    if (d > maxd) maxd = d;
  }
  for (int depth = 0; depth <= maxd; ++depth) {
    for (int m = 1; m <= n - 2; ++m) {
      int k = 0, l = n - 1, d = 0;
      for (;;) {
        int mid = (k + l) / 2;
        if (mid == m) break;
        if (m < mid) l = mid; else k = mid;
        ++d;
      }
      if (d != depth) continue;
      double e[3], xi[3], eta[3], gamma;
      tree_frame(v_ref, m, n, f, e, &gamma, xi, eta);
      double zeta = coords[3 * m], t = coords[3 * m + 1], phi = coords[3 * m + 2];
      double cs = tanh(zeta), sn = 1.0 / cosh(zeta);
      double den = cosh(t) - cs;
      for (int i = 0; i < 3; ++i) {
        double mid = 0.5 * (f[3 * k + i] + f[3 * l + i]);
        f[3 * m + i] = mid + gamma * (e[i] * sinh(t) + (xi[i] * cos(phi) + eta[i] * sin(phi)) * sn) / den;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Chains                                                                    */
/* ------------------------------------------------------------------------ */
#define PURPOSE_STEP_A 0u
#define PURPOSE_STEP_B 1u
#define PURPOSE_INIT 2u
#define PURPOSE_QREF 3u
#define PURPOSE_TRACE 4u
#define PURPOSE_TREE 5u   /* | (vertex << 8): the normals of one tree node */
#define PURPOSE_HMC 6u    /* | (vertex << 8): the momentum of one interior vertex */

static void normals3(const uint32_t w[4], double z[3]) {
  double r1 = sqrt(-2.0 * log(or_u01(w[0])));
  double a1 = 2.0 * M_PI * or_u01(w[1]);
  double r2 = sqrt(-2.0 * log(or_u01(w[2])));
  double a2 = 2.0 * M_PI * or_u01(w[3]);
  z[0] = r1 * cos(a1);
  z[1] = r1 * sin(a1);
  z[2] = r2 * cos(a2);
}

static void near_point(const or_source* s, const or_sensor* d, double e[3]) {
  double u[3];
  sub3(s->pos, d->c, u);
  double D = norm3(u);
  for (int i = 0; i < 3; ++i) e[i] = d->c[i] + d->R * u[i] / D;
}

int or_init_chains(const or_medium* m, const or_source* s, const or_sensor* d,
                   const or_run* r, int init_kind, int init_k, double jitter,
                   int n_chains, int cap, uint32_t chain_offset, double* xyz, int* n) {
  (void)m;
  double e[3];
  near_point(s, d, e);
  for (int c = 0; c < n_chains; ++c) {
    double* f = xyz + (size_t)c * cap * 3;
    if (init_kind == OR_INIT_USER) continue;
    int k = (init_kind == OR_INIT_DIRECT) ? 0 : init_k;
    if (k + 2 > cap) return -1;
    copy3(s->pos, f);
    for (int i = 1; i <= k; ++i) {
      double fr = (double)i / (double)(k + 1);
      uint32_t w[4];
      draw_block(r->seed, (uint32_t)i, 0u, chain_offset + (uint32_t)c, PURPOSE_INIT, w);
      double z[3];
      normals3(w, z);
      for (int j = 0; j < 3; ++j) f[3 * i + j] = s->pos[j] + fr * (e[j] - s->pos[j]) + jitter * z[j];
    }
    copy3(e, f + 3 * (k + 1));
    n[c] = k + 2;
  }
  return 0;
}

typedef struct {
  const or_medium* m;
  const or_source* s;
  const or_sensor* d;
  const or_run* r;
  int cap;
  uint32_t chain_offset;
  uint64_t step0, n_steps;
  double* xyz;
  int* n;
  or_acc* acc;
  double* min_margin;
  double* n_hist;
  double* min_hmc_seg;
  double* lam;       /* wavelength per chain (NULL: wavelength not sampled) */
  int c_begin, c_end;
  double kappa_eq;
  uint32_t thr_within, thr_birth;
  double v_ref[3];   /* tree coordinates: root reference vector */
  double* coords;    /* tree coordinates: scratch of 3 cap doubles per worker */
} chain_job;

static double log_sum_tb(const or_medium* m, int n, const double* f, double* tbs) {
  double T = 0.0;
  for (int k = 0; k <= n - 2; ++k) {
    double ta, tb;
    or_segment_depths(m, f + 3 * k, f + 3 * (k + 1), &ta, &tb);
    tbs[k] = tb;
    T += tb;
  }
  return T;
}

static double path_length(int n, const double* f) {
  double L = 0.0;
  for (int k = 0; k <= n - 2; ++k) {
    double r[3];
    sub3(f + 3 * (k + 1), f + 3 * k, r);
    L += norm3(r);
  }
  return L;
}

static void record_state(const chain_job* J, or_acc* a, int n, const double* f, double lp,
                         uint64_t t) {
  a->n_rec += 1.0;
  if (n == 2) a->n_direct += 1.0;
  double L = path_length(n, f);
  a->sum_n += n;
  a->sum_L += L;
  a->sum_L2 += L * L;
  if (J->r->gradients && J->m->kind == OR_HOMOGENEOUS) {
    double sc[3];
    or_score(J->m, J->s, J->d, n, f, sc);
    for (int i = 0; i < 3; ++i) a->sum_score[i] += sc[i];
  }
  if (J->r->thin_bridge > 0 && (t % J->r->thin_bridge) == 0) {
    double lq = or_qref_logdensity(J->m, J->s, J->d, J->cap, n, f);
    a->sum_bridge += isfinite(lq) ? exp(0.5 * (lq - lp)) : 0.0;
    a->n_bridge += 1.0;
  }
}

/* One HMC trajectory of the path density (the move's deterministic part):
 * from positions x (n x 3, source and end vertex held) and momenta p (n x 3,
 * interior rows used), L leapfrog steps of size eps with the force
 * d log p / d f (zero where the density is zero); x and p are updated in
 * place.  Returns log p at the end point. */
double or_hmc_leapfrog(const or_medium* m, const or_source* s, const or_sensor* d, int n, double* x, double* p,
                       double eps, int L) {
  double* g = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  or_grad_logp(m, s, d, n, x, g);
  for (int i = 1; i <= n - 2; ++i)
    for (int q = 0; q < 3; ++q) p[3 * i + q] += 0.5 * eps * g[3 * i + q];
  for (int st = 1; st <= L; ++st) {
    for (int i = 1; i <= n - 2; ++i)
      for (int q = 0; q < 3; ++q) x[3 * i + q] += eps * p[3 * i + q];
    or_grad_logp(m, s, d, n, x, g);
    double h = (st == L) ? 0.5 * eps : eps;
    for (int i = 1; i <= n - 2; ++i)
      for (int q = 0; q < 3; ++q) p[3 * i + q] += h * g[3 * i + q];
  }
  free(g);
  return or_logp(m, s, d, n, x);
}

/* The chains' target: the path density, or (toy_s > 0, pins only) a product
 * density with known sector weights: P(n) proportional to toy_w[n], interior
 * vertex k of an n-vertex path ~ N(mu_k, toy_s^2 I) with mu_k on the segment
 * from the source to the sensor centre at fraction k/(n-1), and the end
 * vertex uniform on the sensor sphere. */
static double target_logp(const chain_job* J, const or_medium* m, double lam, int n, const double* f) {
  const or_run* r = J->r;
  if (!(r->toy_s > 0.0)) {
    /* the joint density S(lam) p_lam(path) when the wavelength is sampled */
    double lp = or_logp(m, J->s, J->d, n, f);
    return r->n_lambda >= 2 ? lp + or_log_spectrum(r, lam) : lp;
  }
  double lp = log(r->toy_w[n]) - log(4.0 * M_PI * J->d->R * J->d->R);
  double s2 = r->toy_s * r->toy_s;
  for (int k = 1; k <= n - 2; ++k) {
    double fr = (double)k / (double)(n - 1);
    for (int i = 0; i < 3; ++i) {
      double mu = J->s->pos[i] + fr * (J->d->c[i] - J->s->pos[i]);
      double dlt = f[3 * k + i] - mu;
      lp += -0.5 * dlt * dlt / s2 - 0.5 * log(2.0 * M_PI * s2);
    }
  }
  return lp;
}

/* Length of the shortest segment of an n-vertex path (a diagnostic of
 * leapfrog stiffness: the curvature of log p grows like 1 / length^2). */
static double shortest_segment(int n, const double* f) {
  double lo = INFINITY;
  for (int k = 0; k + 1 < n; ++k) {
    double r[3];
    sub3(f + 3 * (k + 1), f + 3 * k, r);
    lo = fmin(lo, norm3(r));
  }
  return lo;
}

/* ------------------------------------------------------------------------ */
/* Wavelength as a sampled coordinate (section "Discussion": a wavelength   */
/* parameter added to the probability distribution and sampled along with  */
/* the path vertices).  The paper gives no medium model; the reading here:  */
/* power laws of the coefficients about a reference wavelength, and the    */
/* emission-times-detection spectrum S(l) as a normalised piecewise-linear  */
/* table.                                                                   */
/* ------------------------------------------------------------------------ */
void or_medium_at(const or_medium* m, double lam, or_medium* out) {
  *out = *m;
  if (!(m->lambda0 > 0.0) || !(lam > 0.0)) return;
  /* b = 1 / lambda_s scales as (l / l0)^(-k_s): the length as (l / l0)^(+k_s) */
  out->lambda_s = m->lambda_s * pow(lam / m->lambda0, m->k_s);
  out->lambda_a = m->lambda_a * pow(lam / m->lambda0, m->k_a);
}

static double spectrum_area(const or_run* r) {
  double A = 0.0;
  for (int i = 0; i + 1 < r->n_lambda; ++i)
    A += 0.5 * (r->lambda_nm[i + 1] - r->lambda_nm[i]) * (r->spectrum[i] + r->spectrum[i + 1]);
  return A;
}

double or_log_spectrum(const or_run* r, double lam) {
  const int K = r->n_lambda;
  if (K < 2 || !(lam >= r->lambda_nm[0]) || !(lam <= r->lambda_nm[K - 1])) return NEG_INF;
  int i = 0;
  while (i + 2 < K && lam > r->lambda_nm[i + 1]) ++i;
  const double h = r->lambda_nm[i + 1] - r->lambda_nm[i];
  const double v = r->spectrum[i] + (r->spectrum[i + 1] - r->spectrum[i]) * (lam - r->lambda_nm[i]) / h;
  return v > 0.0 ? log(v / spectrum_area(r)) : NEG_INF;
}

double or_spectrum_quantile(const or_run* r, double u) {
  const int K = r->n_lambda;
  double t = u * spectrum_area(r);
  for (int i = 0; i + 1 < K; ++i) {
    const double h = r->lambda_nm[i + 1] - r->lambda_nm[i];
    const double y0 = r->spectrum[i], y1 = r->spectrum[i + 1];
    const double area = 0.5 * h * (y0 + y1);
    if (t <= area || i + 2 == K) {
      /* y0 s + k s^2 / 2 = t with k = (y1 - y0) / h, in the form that stays
       * accurate for k of either sign and k -> 0 */
      const double k = (y1 - y0) / h;
      const double disc = fmax(y0 * y0 + 2.0 * k * t, 0.0);
      const double den = y0 + sqrt(disc);
      const double s_ = den > 0.0 ? 2.0 * t / den : 0.0;
      return r->lambda_nm[i] + fmin(fmax(s_, 0.0), h);
    }
    t -= area;
  }
  return r->lambda_nm[K - 1];
}

void or_init_lambda(const or_run* r, int n_chains, uint32_t chain_offset, double* lam) {
  for (int c = 0; c < n_chains; ++c) {
    uint32_t w[4];
    draw_block(r->seed, 0u, 1u, chain_offset + (uint32_t)c, PURPOSE_INIT, w);
    lam[c] = or_spectrum_quantile(r, or_u01(w[0]));
  }
}

static void* chain_worker(void* arg) {
  chain_job* J = (chain_job*)arg;
  const or_medium* m = J->m;
  const or_run* r = J->r;
  const int lam_on = r->n_lambda >= 2 && J->lam != NULL;
  or_medium mc;      /* the medium at the chain's wavelength */
  int cap = J->cap;
  double* y = (double*)malloc(sizeof(double) * 3 * (cap + 1));
  double* tbs = (double*)malloc(sizeof(double) * (cap + 1));
  double* gx = (double*)malloc(sizeof(double) * 3 * (cap + 1));
  double* gy = (double*)malloc(sizeof(double) * 3 * (cap + 1));
  for (int c = J->c_begin; c < J->c_end; ++c) {
    double* x = J->xyz + (size_t)c * cap * 3;
    int n = J->n[c];
    uint32_t chain = J->chain_offset + (uint32_t)c;
    or_acc* a = J->acc ? &J->acc[c] : NULL;
    double lam = lam_on ? J->lam[c] : 0.0;
    if (lam_on) {
      or_medium_at(J->m, lam, &mc);
      m = &mc;
    }
    double lpx = target_logp(J, m, lam, n, x);
    double margin = INFINITY;
    double hmc_seg = INFINITY;
    for (uint64_t t = J->step0; t < J->step0 + J->n_steps; ++t) {
      uint32_t A[4], B[4];
      draw_block(r->seed, (uint32_t)t, (uint32_t)(t >> 32), chain, PURPOSE_STEP_A, A);
      draw_block(r->seed, (uint32_t)t, (uint32_t)(t >> 32), chain, PURPOSE_STEP_B, B);
      uint32_t u_move = A[0] >> 9;
      double log_u = log(or_u01(A[2]));
      int kind;
      int ny = n;
      int lam_move = 0;
      double lam_y = lam;
      or_medium mc_y;
      double logA = NEG_INF, lpy = NEG_INF;
      int proposed = 0;
      if (u_move < J->thr_within && r->within == OR_WITHIN_TREE) {
        /* the paper's within-dimension move in tree coordinates: the end
         * vertex takes a vMF step on the sensor, then every interior vertex's
         * (zeta, t, phi) a normal step of scale sigma / sqrt(n); the path is
         * rebuilt top-down, and the acceptance carries the coordinates'
         * Jacobian p(y) J(y) / (p(x) J(x)) */
        kind = OR_MOVE_INTERIOR;
        double ljx = or_tree_coords(J->v_ref, n, x, J->coords);
        double nu[3];
        sub3(x + 3 * (n - 1), J->d->c, nu);
        double dn = norm3(nu);
        for (int i = 0; i < 3; ++i) nu[i] /= dn;
        double ke = r->kappa_end;
        double u0 = or_u01(B[0]);
        double w = 1.0 + log(u0 + (1.0 - u0) * exp(-2.0 * ke)) / ke;
        double ph = 2.0 * M_PI * or_u01(B[1]);
        double sw = sqrt(fmax(0.0, 1.0 - w * w));
        double e1[3], e2[3];
        or_onb(nu, e1, e2);
        copy3(x, y);
        for (int i = 0; i < 3; ++i) {
          double nn = w * nu[i] + sw * (cos(ph) * e1[i] + sin(ph) * e2[i]);
          y[3 * (n - 1) + i] = J->d->c[i] + J->d->R * nn;
        }
        double step = r->sigma / sqrt((double)n);
        for (int mm = 1; mm <= n - 2; ++mm) {
          uint32_t Wn[4];
          draw_block(r->seed, (uint32_t)t, (uint32_t)(t >> 32), chain, PURPOSE_TREE | ((uint32_t)mm << 8), Wn);
          double z[3];
          normals3(Wn, z);
          for (int q = 0; q < 3; ++q) J->coords[3 * mm + q] += step * z[q];
        }
        or_tree_path(J->v_ref, n, J->coords, y);
        lpy = target_logp(J, m, lam, n, y);
        if (isfinite(lpy)) {
          double ljy = or_tree_coords(J->v_ref, n, y, J->coords);
          logA = lpy + ljy - lpx - ljx;
        }
        proposed = 1;
      } else if (u_move < J->thr_within && r->within == OR_WITHIN_HMC &&
                 1 + (int)index_draw(A[1], (uint32_t)(n - 1)) != n - 1) {
        /* full-path gradient move (section "Discussion": Hamiltonian Monte
         * Carlo): every interior vertex gets a standard normal momentum, L
         * leapfrog steps of size eps follow the gradient of log p with the
         * source and the end vertex fixed, and the move is accepted with
         * exp(-H(x', p') + H(x, p)), H = -log p + |p|^2 / 2.  Picking the end
         * vertex (probability 1/(n-1)) still makes a vMF end move. */
        kind = OR_MOVE_INTERIOR;
        double eps = r->mala_step;
        int L = r->hmc_steps;
        double* pm = J->coords;  /* momentum, 3 doubles per vertex */
        double k0 = 0.0;
        for (int i = 1; i <= n - 2; ++i) {
          uint32_t Wn[4];
          draw_block(r->seed, (uint32_t)t, (uint32_t)(t >> 32), chain, PURPOSE_HMC | ((uint32_t)i << 8), Wn);
          normals3(Wn, pm + 3 * i);
          k0 += dot3(pm + 3 * i, pm + 3 * i);
        }
        memcpy(y, x, sizeof(double) * 3 * n);
        if (J->min_hmc_seg) hmc_seg = fmin(hmc_seg, shortest_segment(n, y));
        or_grad_logp(m, J->s, J->d, n, y, gy);
        for (int i = 1; i <= n - 2; ++i)
          for (int q = 0; q < 3; ++q) pm[3 * i + q] += 0.5 * eps * gy[3 * i + q];
        for (int st = 1; st <= L; ++st) {
          for (int i = 1; i <= n - 2; ++i)
            for (int q = 0; q < 3; ++q) y[3 * i + q] += eps * pm[3 * i + q];
          if (J->min_hmc_seg) hmc_seg = fmin(hmc_seg, shortest_segment(n, y));
          or_grad_logp(m, J->s, J->d, n, y, gy);
          double h = (st == L) ? 0.5 * eps : eps;
          for (int i = 1; i <= n - 2; ++i)
            for (int q = 0; q < 3; ++q) pm[3 * i + q] += h * gy[3 * i + q];
        }
        double k1 = 0.0;
        for (int i = 1; i <= n - 2; ++i) k1 += dot3(pm + 3 * i, pm + 3 * i);
        lpy = or_logp(m, J->s, J->d, n, y);
        if (isfinite(lpy)) logA = lpy - lpx - 0.5 * k1 + 0.5 * k0;
        proposed = 1;
      } else if (u_move < J->thr_within && lam_on && 1 + (int)index_draw(A[1], (uint32_t)n) == n) {
        /* wavelength move (section "Discussion": the wavelength sampled along
         * with the path vertices, one more coordinate picked with them): a
         * Gaussian step of the wavelength with the path held, accepted with
         * S(l') p_l'(x) / (S(l) p_l(x)) */
        kind = OR_MOVE_INTERIOR;
        double z[3];
        normals3(B, z);
        lam_y = lam + r->sigma_lambda * z[0];
        or_medium_at(J->m, lam_y, &mc_y);
        lpy = target_logp(J, &mc_y, lam_y, n, x);
        memcpy(y, x, sizeof(double) * 3 * n);
        logA = lpy - lpx;
        lam_move = 1;
        proposed = 1;
      } else if (u_move < J->thr_within) {
        /* within-dimension move of one of the n-1 movable vertices (of the n
         * movable coordinates, the last being the wavelength, when it is sampled) */
        int j = 1 + (int)index_draw(A[1], (uint32_t)(n - 1 + lam_on));
        memcpy(y, x, sizeof(double) * 3 * n);
        if (j == n - 1) {
          kind = OR_MOVE_END;
          double nu[3];
          sub3(x + 3 * j, J->d->c, nu);
          double dn = norm3(nu);
          for (int i = 0; i < 3; ++i) nu[i] /= dn;
          double ke = r->kappa_end;
          double u0 = or_u01(B[0]);
          double w = 1.0 + log(u0 + (1.0 - u0) * exp(-2.0 * ke)) / ke;
          double ph = 2.0 * M_PI * or_u01(B[1]);
          double sw = sqrt(fmax(0.0, 1.0 - w * w));
          double e1[3], e2[3];
          or_onb(nu, e1, e2);
          for (int i = 0; i < 3; ++i) {
            double nn = w * nu[i] + sw * (cos(ph) * e1[i] + sin(ph) * e2[i]);
            y[3 * j + i] = J->d->c[i] + J->d->R * nn;
          }
          lpy = target_logp(J, m, lam, n, y);
          logA = lpy - lpx;
        } else {
          kind = OR_MOVE_INTERIOR;
          double z[3];
          normals3(B, z);
          if (r->within == OR_WITHIN_MALA) {
            double eps = r->mala_step;
            or_grad_logp(m, J->s, J->d, n, x, gx);
            double mean_f[3];
            for (int i = 0; i < 3; ++i) {
              mean_f[i] = x[3 * j + i] + 0.5 * eps * eps * gx[3 * j + i];
              y[3 * j + i] = mean_f[i] + eps * z[i];
            }
            lpy = or_grad_logp(m, J->s, J->d, n, y, gy);
            if (isfinite(lpy)) {
              double fw = 0.0, bw = 0.0;
              for (int i = 0; i < 3; ++i) {
                double dfw = y[3 * j + i] - mean_f[i];
                double dbw = x[3 * j + i] - y[3 * j + i] - 0.5 * eps * eps * gy[3 * j + i];
                fw += dfw * dfw;
                bw += dbw * dbw;
              }
              logA = lpy - lpx - bw / (2.0 * eps * eps) + fw / (2.0 * eps * eps);
            }
          } else {
            for (int i = 0; i < 3; ++i) y[3 * j + i] = x[3 * j + i] + r->sigma * z[i];
            lpy = target_logp(J, m, lam, n, y);
            logA = lpy - lpx;
          }
        }
        proposed = 1;
      } else if (u_move < J->thr_birth) {
        kind = OR_MOVE_BIRTH;
        if (n < cap) {
          double T = log_sum_tb(m, n, x, tbs);
          if (T > 0.0) {
            double target = or_u01(A[1]) * T;
            int k = n - 2;
            double cum = 0.0;
            for (int i = 0; i <= n - 2; ++i) {
              cum += tbs[i];
              if (cum > target) { k = i; break; }
            }
            const double* fk = x + 3 * k;
            const double* fk1 = x + 3 * (k + 1);
            double beta = insertion_beta(m, r, J->kappa_eq, fk, fk1);
            double ub = or_u01(B[0]);
            double cs = -1.0 - log(1.0 - ub * (1.0 - exp(-2.0 * beta))) / beta;
            if (cs > 1.0) cs = 1.0;
            if (cs < -1.0) cs = -1.0;
            double sv = acos(cs);
            double ut = or_u01(B[1]);
            double tv = log(ut / (1.0 - ut));
            double ph = 2.0 * M_PI * or_u01(B[2]);
            double fnew[3];
            or_bisph_point(fk, fk1, sv, tv, ph, fnew);
            /* y = x with fnew inserted at index k+1 */
            memcpy(y, x, sizeof(double) * 3 * (k + 1));
            copy3(fnew, y + 3 * (k + 1));
            memcpy(y + 3 * (k + 2), x + 3 * (k + 1), sizeof(double) * 3 * (n - k - 1));
            ny = n + 1;
            lpy = target_logp(J, m, lam, ny, y);
            double lq = log_insert_density(m, r, J->kappa_eq, fk, fk1, fnew);
            logA = lpy - lpx + log(r->p_death) - log((double)(ny - 2)) - log(r->p_birth) -
                   log(tbs[k] / T) - lq;
            proposed = 1;
          }
        }
      } else {
        kind = OR_MOVE_DEATH;
        if (n > 2) {
          int j = 1 + (int)index_draw(A[1], (uint32_t)(n - 2));
          memcpy(y, x, sizeof(double) * 3 * j);
          memcpy(y + 3 * j, x + 3 * (j + 1), sizeof(double) * 3 * (n - j - 1));
          ny = n - 1;
          lpy = target_logp(J, m, lam, ny, y);
          double T = log_sum_tb(m, ny, y, tbs);
          double lq = log_insert_density(m, r, J->kappa_eq, x + 3 * (j - 1), x + 3 * (j + 1), x + 3 * j);
          /* reverse birth y -> x selects segment j-1 of y and inserts x_j */
          double logA_birth = lpx - lpy + log(r->p_death) - log((double)(n - 2)) - log(r->p_birth) -
                              log(tbs[j - 1] / T) - lq;
          logA = -logA_birth;
          proposed = 1;
        }
      }
      if (a) a->prop[kind] += 1.0;
      int accept = 0;
      if (proposed && isfinite(lpy)) {
        if (isfinite(logA)) {
          double mg = fabs(logA - log_u);
          if (mg < margin) margin = mg;
        }
        accept = log_u < logA;
      }
      if (accept) {
        memcpy(x, y, sizeof(double) * 3 * ny);
        n = ny;
        lpx = lpy;
        if (lam_move) {
          lam = lam_y;
          mc = mc_y;
        }
        if (a) a->acc[kind] += 1.0;
      }
      if (a && t >= r->burn_in) record_state(J, a, n, x, lpx, t);
      if (J->n_hist && t >= r->burn_in) J->n_hist[(size_t)c * (cap + 1) + n] += 1.0;
    }
    J->n[c] = n;
    if (lam_on) J->lam[c] = lam;
    if (J->min_margin) J->min_margin[c] = margin;
    if (J->min_hmc_seg) J->min_hmc_seg[c] = hmc_seg;
  }
  free(y);
  free(tbs);
  free(gx);
  free(gy);
  return NULL;
}

int or_run_chains(const or_medium* m, const or_source* s, const or_sensor* d,
                  const or_run* r, int n_chains, int cap, uint32_t chain_offset,
                  uint64_t step0, uint64_t n_steps, double* xyz, int* n,
                  or_acc* acc, double* min_margin, int n_threads) {
  return or_run_chains_hist(m, s, d, r, n_chains, cap, chain_offset, step0, n_steps, xyz, n, acc,
                            min_margin, NULL, n_threads);
}

int or_run_chains_hist(const or_medium* m, const or_source* s, const or_sensor* d,
                       const or_run* r, int n_chains, int cap, uint32_t chain_offset,
                       uint64_t step0, uint64_t n_steps, double* xyz, int* n,
                       or_acc* acc, double* min_margin, double* n_hist, int n_threads) {
  return or_run_chains_diag(m, s, d, r, n_chains, cap, chain_offset, step0, n_steps, xyz, n, acc, min_margin,
                            n_hist, NULL, n_threads);
}

int or_run_chains_diag(const or_medium* m, const or_source* s, const or_sensor* d,
                       const or_run* r, int n_chains, int cap, uint32_t chain_offset,
                       uint64_t step0, uint64_t n_steps, double* xyz, int* n,
                       or_acc* acc, double* min_margin, double* n_hist, double* min_hmc_seg, int n_threads) {
  return or_run_chains_lam(m, s, d, r, n_chains, cap, chain_offset, step0, n_steps, xyz, n, NULL, acc, min_margin,
                           n_hist, min_hmc_seg, n_threads);
}

int or_run_chains_lam(const or_medium* m, const or_source* s, const or_sensor* d,
                      const or_run* r, int n_chains, int cap, uint32_t chain_offset,
                      uint64_t step0, uint64_t n_steps, double* xyz, int* n, double* lam,
                      or_acc* acc, double* min_margin, double* n_hist, double* min_hmc_seg, int n_threads) {
  /* the wavelength is sampled with Gaussian vertex moves in homogeneous media */
  if (r->n_lambda >= 2 && (lam == NULL || m->kind != OR_HOMOGENEOUS || r->within != OR_WITHIN_PERTURB))
    return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_chains) n_threads = n_chains > 0 ? n_chains : 1;
  double keq = or_kappa_eq(m->g);
  uint32_t thr_w = (uint32_t)floor(r->p_within * 8388608.0 + 0.5);
  uint32_t thr_b = (uint32_t)floor((r->p_within + r->p_birth) * 8388608.0 + 0.5);
  chain_job* jobs = (chain_job*)calloc((size_t)n_threads, sizeof(chain_job));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int i = 0; i < n_threads; ++i) {
    chain_job* J = &jobs[i];
    J->m = m; J->s = s; J->d = d; J->r = r; J->cap = cap; J->chain_offset = chain_offset;
    J->step0 = step0; J->n_steps = n_steps; J->xyz = xyz; J->n = n; J->acc = acc;
    J->min_margin = min_margin; J->n_hist = n_hist; J->min_hmc_seg = min_hmc_seg; J->lam = lam; J->kappa_eq = keq; J->thr_within = thr_w; J->thr_birth = thr_b;
    or_tree_vref(s, d, J->v_ref);
    J->coords = (double*)calloc((size_t)3 * (size_t)(cap + 1), sizeof(double));
    J->c_begin = (int)((long)n_chains * i / n_threads);
    J->c_end = (int)((long)n_chains * (i + 1) / n_threads);
    pthread_create(&th[i], NULL, chain_worker, J);
  }
  for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
  for (int i = 0; i < n_threads; ++i) free(jobs[i].coords);
  free(jobs);
  free(th);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Direct-sector integral Z2: the n = 2 part of the path integral,           */
/* integral over the sensor area of p(f_0, f_1) (paper: the path integral    */
/* restricted to paths without scattering).  Over the solid angle seen from  */
/* the source: Z2 = int dOmega eps(omega) exp(-tau(s -> hit)) rho(hit).       */
/* The rim singularity is removed by w = w_min + (1 - w_min) v^2.             */
/* ------------------------------------------------------------------------ */
double or_z2(const or_medium* m, const or_source* s, const or_sensor* d, int n_v, int n_phi) {
  double ax[3];
  sub3(d->c, s->pos, ax);
  double D = norm3(ax);
  for (int i = 0; i < 3; ++i) ax[i] /= D;
  double R = d->R;
  double wmin = sqrt(1.0 - (R / D) * (R / D));
  double e1[3], e2[3];
  or_onb(ax, e1, e2);
  double sum = 0.0;
  for (int iv = 0; iv < n_v; ++iv) {
    double v = (iv + 0.5) / n_v;
    double w = wmin + (1.0 - wmin) * v * v;
    double dw = 2.0 * (1.0 - wmin) * v / n_v;
    double sw = sqrt(fmax(0.0, 1.0 - w * w));
    double disc = R * R - D * D * (1.0 - w * w);
    if (disc < 0.0) disc = 0.0;
    double rr = D * w - sqrt(disc);
    for (int ip = 0; ip < n_phi; ++ip) {
      double ph = 2.0 * M_PI * (ip + 0.5) / n_phi;
      double om[3], h[3], nu[3];
      for (int i = 0; i < 3; ++i) {
        om[i] = w * ax[i] + sw * (cos(ph) * e1[i] + sin(ph) * e2[i]);
        h[i] = s->pos[i] + rr * om[i];
        nu[i] = (h[i] - d->c[i]) / R;
      }
      double ta, tb;
      or_segment_depths(m, s->pos, h, &ta, &tb);
      double val = exp(or_log_emission(s, om) - ta - tb + or_log_rho(d, nu));
      sum += val * dw * (2.0 * M_PI / n_phi);
    }
  }
  return sum;
}

/* ------------------------------------------------------------------------ */
/* Normalised reference density q_ref for the geometric bridge estimator    */
/* (section "Comparison of relative light yield", with p_0 := q_ref).  It is */
/* the paper's recursive tree of bispherical coordinates (appendix, path     */
/* space coordinate system): vertex m = floor((k+l)/2) is placed about the   */
/* foci f_k, f_l with q(s) q(t) q(phi), recursively; the vertex count is a    */
/* truncated Poisson in the straight-line scattering depth, and the end      */
/* vertex is uniform over the sensor cap visible from the source.            */
/* parity unpinned: the paper fixes no reference density; its normalisation  */
/* and sampling are pinned only by the tests' importance-sampling checks.    */
/* ------------------------------------------------------------------------ */
static double qref_mu(const or_medium* m, const or_source* s, const or_sensor* d) {
  double e[3];
  near_point(s, d, e);
  double ta, tb;
  or_segment_depths(m, s->pos, e, &ta, &tb);
  return tb;
}

static double qref_log_pn(double mu, int cap, int n) {
  /* truncated Poisson over k = n-2 in [0, cap-2] */
  double norm = 0.0;
  for (int k = 0; k <= cap - 2; ++k) norm += exp(k * log(mu) - mu - lgamma(k + 1.0));
  int k = n - 2;
  return k * log(mu) - mu - lgamma(k + 1.0) - log(norm);
}

static double qref_tree_logdensity(const or_medium* m, double keq, double beta_min,
                                   const double* f, int k, int l) {
  if (l - k < 2) return 0.0;
  int mm = (k + l) / 2;
  const double* fk = f + 3 * k;
  const double* fl = f + 3 * l;
  double s, t, phi;
  or_bisph_coords(fk, fl, f + 3 * mm, &s, &t, &phi);
  double diff[3];
  sub3(fl, fk, diff);
  double gamma = 0.5 * norm3(diff);
  or_run rr;
  memset(&rr, 0, sizeof rr);
  rr.beta_min = beta_min;
  double beta = insertion_beta(m, &rr, keq, fk, fl);
  double lq = or_log_q_s(beta, s) + or_log_q_t(t) - log(2.0 * M_PI) - or_log_bisph_jacobian(gamma, s, t);
  return lq + qref_tree_logdensity(m, keq, beta_min, f, k, mm) + qref_tree_logdensity(m, keq, beta_min, f, mm, l);
}

#define QREF_BETA_MIN 0.01

double or_qref_logdensity(const or_medium* m, const or_source* s, const or_sensor* d,
                          int cap, int n, const double* f) {
  double u[3];
  sub3(s->pos, d->c, u);
  double D = norm3(u);
  for (int i = 0; i < 3; ++i) u[i] /= D;
  double nu[3];
  sub3(f + 3 * (n - 1), d->c, nu);
  double dn = norm3(nu);
  for (int i = 0; i < 3; ++i) nu[i] /= dn;
  double R = d->R;
  if (dot3(nu, u) <= R / D) return NEG_INF;
  double lq = qref_log_pn(qref_mu(m, s, d), cap, n) - log(2.0 * M_PI * R * R * (1.0 - R / D));
  lq += qref_tree_logdensity(m, or_kappa_eq(m->g), QREF_BETA_MIN, f, 0, n - 1);
  return lq;
}

static void qref_tree_sample(const or_medium* m, double keq, uint64_t seed, uint32_t stream,
                             uint64_t draw, double* f, int k, int l) {
  if (l - k < 2) return;
  int mm = (k + l) / 2;
  uint32_t w[4];
  draw_block(seed, (uint32_t)draw, (uint32_t)(draw >> 32), (uint32_t)mm, PURPOSE_QREF | (stream << 8), w);
  or_run rr;
  memset(&rr, 0, sizeof rr);
  rr.beta_min = QREF_BETA_MIN;
  double beta = insertion_beta(m, &rr, keq, f + 3 * k, f + 3 * l);
  double ub = or_u01(w[0]);
  double cs = -1.0 - log(1.0 - ub * (1.0 - exp(-2.0 * beta))) / beta;
  if (cs > 1.0) cs = 1.0;
  if (cs < -1.0) cs = -1.0;
  double ut = or_u01(w[1]);
  double t = log(ut / (1.0 - ut));
  double ph = 2.0 * M_PI * or_u01(w[2]);
  or_bisph_point(f + 3 * k, f + 3 * l, acos(cs), t, ph, f + 3 * mm);
  qref_tree_sample(m, keq, seed, stream, draw, f, k, mm);
  qref_tree_sample(m, keq, seed, stream, draw, f, mm, l);
}

int or_qref_sample(const or_medium* m, const or_source* s, const or_sensor* d, int cap,
                   uint64_t seed, uint32_t stream, uint64_t draw, double* f) {
  uint32_t w[4];
  draw_block(seed, (uint32_t)draw, (uint32_t)(draw >> 32), 0u, PURPOSE_QREF | (stream << 8), w);
  double mu = qref_mu(m, s, d);
  /* vertex count by inverse CDF of the truncated Poisson */
  double un = or_u01(w[0]);
  int n = cap;
  double cum = 0.0;
  for (int nn = 2; nn <= cap; ++nn) {
    cum += exp(qref_log_pn(mu, cap, nn));
    if (cum > un) { n = nn; break; }
  }
  /* end vertex uniform on the visible cap */
  double u[3];
  sub3(s->pos, d->c, u);
  double D = norm3(u);
  for (int i = 0; i < 3; ++i) u[i] /= D;
  double R = d->R;
  double wv = R / D + (1.0 - R / D) * or_u01(w[1]);
  double ph = 2.0 * M_PI * or_u01(w[2]);
  double e1[3], e2[3];
  or_onb(u, e1, e2);
  double sw = sqrt(fmax(0.0, 1.0 - wv * wv));
  copy3(s->pos, f);
  for (int i = 0; i < 3; ++i)
    f[3 * (n - 1) + i] = d->c[i] + R * (wv * u[i] + sw * (cos(ph) * e1[i] + sin(ph) * e2[i]));
  qref_tree_sample(m, or_kappa_eq(m->g), seed, stream, draw, f, 0, n - 1);
  return n;
}

typedef struct {
  const or_medium* m; const or_source* s; const or_sensor* d; int cap;
  uint64_t seed; uint32_t stream; uint64_t d0, d1; double out[4];
} qref_job;

static void* qref_worker(void* arg) {
  qref_job* J = (qref_job*)arg;
  double* f = (double*)malloc(sizeof(double) * 3 * J->cap);
  for (uint64_t i = J->d0; i < J->d1; ++i) {
    int n = or_qref_sample(J->m, J->s, J->d, J->cap, J->seed, J->stream, i, f);
    double lp = or_logp(J->m, J->s, J->d, n, f);
    double lq = or_qref_logdensity(J->m, J->s, J->d, J->cap, n, f);
    double ratio = isfinite(lp) ? exp(lp - lq) : 0.0;
    J->out[0] += sqrt(ratio);
    J->out[1] += ratio;
    J->out[2] += ratio * ratio;
    J->out[3] += 1.0;
  }
  free(f);
  return NULL;
}

int or_qref_bridge_sums(const or_medium* m, const or_source* s, const or_sensor* d, int cap,
                        uint64_t seed, uint32_t stream, uint64_t n_draws, double* out,
                        int n_threads) {
  if (n_threads < 1) n_threads = 1;
  qref_job* jobs = (qref_job*)calloc((size_t)n_threads, sizeof(qref_job));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int i = 0; i < n_threads; ++i) {
    qref_job* J = &jobs[i];
    J->m = m; J->s = s; J->d = d; J->cap = cap; J->seed = seed; J->stream = stream;
    J->d0 = n_draws * (uint64_t)i / (uint64_t)n_threads;
    J->d1 = n_draws * (uint64_t)(i + 1) / (uint64_t)n_threads;
    pthread_create(&th[i], NULL, qref_worker, J);
  }
  for (int k = 0; k < 4; ++k) out[k] = 0.0;
  for (int i = 0; i < n_threads; ++i) {
    pthread_join(th[i], NULL);
    for (int k = 0; k < 4; ++k) out[k] += jobs[i].out[k];
  }
  free(jobs);
  free(th);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Forward ray tracer (appendix, Algorithm 1)                               */
/* ------------------------------------------------------------------------ */

/* Distance along the ray x + s n to the first intersection with the sphere,
 * or +inf if the ray misses it ahead. */
static double ray_sphere(const double x[3], const double nh[3], const double c[3], double R) {
  double w[3];
  sub3(x, c, w);
  double b = dot3(w, nh);
  double cc = dot3(w, w) - R * R;
  double disc = b * b - cc;
  if (disc < 0.0) return INFINITY;
  double sq = sqrt(disc);
  double s1 = -b - sq;
  if (s1 > 0.0) return s1;
  double s2 = -b + sq;
  if (s2 > 0.0 && cc < 0.0) return s2; /* starting inside: not expected */
  return INFINITY;
}

/* Solve int_0^dL b(x + s n) ds = tau for dL (Algorithm 1, free-path step). */
static double free_path(const or_medium* m, const double x[3], const double nh[3], double tau) {
  if (m->kind == OR_HOMOGENEOUS) return tau * m->lambda_s;
  double dL = 0.0;
  double z = x[2];
  int l = layer_index(m, z);
  for (int guard = 0; guard < 100000; ++guard) {
    double b = 1.0 / m->lambda_s_layers[l];
    double dist = INFINITY;
    int next = l;
    if (nh[2] > 0.0 && l < m->n_layers - 1) {
      double zb = m->z0 + (l + 1) * m->dz;
      dist = (zb - z) / nh[2];
      next = l + 1;
    } else if (nh[2] < 0.0 && l > 0) {
      double zb = m->z0 + l * m->dz;
      dist = (zb - z) / nh[2];
      next = l - 1;
    }
    if (dist < 0.0) dist = 0.0;
    if (tau <= b * dist) return dL + tau / b;
    tau -= b * dist;
    dL += dist;
    z += dist * nh[2];
    l = next;
  }
  return dL;
}

static double sample_cos_theta(const or_medium* m, double u_cos, double u_mix) {
  double G = m->g;
  if (m->f_sl > 0.0 && u_mix < m->f_sl) {
    double alpha = 2.0 / (1.0 / G - 1.0);
    double v = pow(u_cos, 1.0 / (alpha + 1.0));
    return 2.0 * v - 1.0;
  }
  if (fabs(G) < 1e-9) return 2.0 * u_cos - 1.0;
  double q = (1.0 - G * G) / (1.0 - G + 2.0 * G * u_cos);
  double c = (1.0 + G * G - q * q) / (2.0 * G);
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  return c;
}

typedef struct {
  const or_medium* m; const or_source* s; const or_sensor* d;
  uint64_t seed, p0, p1; double r_reject; int max_scatter; double out[5];
  double* hist;
  double* lhist; double l_lo, l_hi; int l_bins;   /* path-length histogram (may be NULL) */
} trace_job;

static void* trace_worker(void* arg) {
  trace_job* J = (trace_job*)arg;
  const or_medium* m = J->m;
  const or_sensor* d = J->d;
  for (uint64_t p = J->p0; p < J->p1; ++p) {
    uint32_t w[4];
    draw_block(J->seed, (uint32_t)p, (uint32_t)(p >> 32), 0u, PURPOSE_TRACE, w);
    double x[3], nh[3];
    copy3(J->s->pos, x);
    double ph = 2.0 * M_PI * or_u01(w[1]);
    double e1[3], e2[3];
    if (J->s->emission == OR_EMIT_VMF && J->s->kappa > 0.0) {
      double k = J->s->kappa;
      double u0 = or_u01(w[0]);
      double ww = 1.0 + log(u0 + (1.0 - u0) * exp(-2.0 * k)) / k;
      double sw = sqrt(fmax(0.0, 1.0 - ww * ww));
      or_onb(J->s->dir, e1, e2);
      for (int i = 0; i < 3; ++i) nh[i] = ww * J->s->dir[i] + sw * (cos(ph) * e1[i] + sin(ph) * e2[i]);
    } else {
      double ww = 2.0 * or_u01(w[0]) - 1.0;
      double sw = sqrt(fmax(0.0, 1.0 - ww * ww));
      nh[0] = sw * cos(ph); nh[1] = sw * sin(ph); nh[2] = ww;
    }
    double lnw = 0.0; /* reading Q13 */
    double L = 0.0;
    J->out[3] += 1.0;
    for (int i = 0; i <= J->max_scatter; ++i) {
      draw_block(J->seed, (uint32_t)p, (uint32_t)(p >> 32), (uint32_t)(i + 1), PURPOSE_TRACE, w);
      double tau_b = -log(or_u01(w[0]));
      double dL = free_path(m, x, nh, tau_b);
      double dist = ray_sphere(x, nh, d->c, d->R);
      double go = dist < dL ? dist : dL;
      double end[3] = {x[0] + go * nh[0], x[1] + go * nh[1], x[2] + go * nh[2]};
      double ta, tb;
      or_segment_depths(m, x, end, &ta, &tb);
      lnw -= ta;
      if (dist < dL) {
        double nu[3];
        for (int k = 0; k < 3; ++k) nu[k] = (end[k] - d->c[k]) / d->R;
        double W = exp(lnw + or_log_rho(d, nu));
        L += dist;
        J->out[0] += W;
        J->out[1] += W * W;
        J->out[2] += 1.0;
        J->out[4] += W * L;
        if (J->hist) J->hist[i] += W;
        if (J->lhist && L >= J->l_lo && L < J->l_hi) {
          int bin = (int)floor((L - J->l_lo) / (J->l_hi - J->l_lo) * J->l_bins);
          if (bin >= 0 && bin < J->l_bins) J->lhist[bin] += W;
        }
        break;
      }
      double rel[3];
      sub3(x, d->c, rel);
      if (norm3(rel) > J->r_reject) break;
      if (i == J->max_scatter) break;
      copy3(end, x);
      L += dL;
      double c = sample_cos_theta(m, or_u01(w[1]), or_u01(w[3]));
      double phs = 2.0 * M_PI * or_u01(w[2]);
      double sc = sqrt(fmax(0.0, 1.0 - c * c));
      or_onb(nh, e1, e2);
      double nn[3];
      for (int k = 0; k < 3; ++k) nn[k] = c * nh[k] + sc * (cos(phs) * e1[k] + sin(phs) * e2[k]);
      double nl = norm3(nn);
      for (int k = 0; k < 3; ++k) nh[k] = nn[k] / nl;
    }
  }
  return NULL;
}

int or_trace(const or_medium* m, const or_source* s, const or_sensor* d,
             uint64_t seed, uint64_t photon0, uint64_t n_photons, double r_reject,
             int max_scatter, double* out, int n_threads) {
  return or_trace_hist(m, s, d, seed, photon0, n_photons, r_reject, max_scatter, out, NULL, n_threads);
}

static int trace_run(const or_medium* m, const or_source* s, const or_sensor* d,
                     uint64_t seed, uint64_t photon0, uint64_t n_photons, double r_reject,
                     int max_scatter, double* out, double* hist, double l_lo, double l_hi, int l_bins,
                     double* lhist, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  trace_job* jobs = (trace_job*)calloc((size_t)n_threads, sizeof(trace_job));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int i = 0; i < n_threads; ++i) {
    trace_job* J = &jobs[i];
    J->m = m; J->s = s; J->d = d; J->seed = seed; J->r_reject = r_reject; J->max_scatter = max_scatter;
    J->hist = hist ? (double*)calloc((size_t)max_scatter + 1, sizeof(double)) : NULL;
    J->lhist = lhist ? (double*)calloc((size_t)l_bins, sizeof(double)) : NULL;
    J->l_lo = l_lo; J->l_hi = l_hi; J->l_bins = l_bins;
    J->p0 = photon0 + n_photons * (uint64_t)i / (uint64_t)n_threads;
    J->p1 = photon0 + n_photons * (uint64_t)(i + 1) / (uint64_t)n_threads;
    pthread_create(&th[i], NULL, trace_worker, J);
  }
  for (int k = 0; k < 5; ++k) out[k] = 0.0;
  if (hist) for (int k = 0; k <= max_scatter; ++k) hist[k] = 0.0;
  if (lhist) for (int k = 0; k < l_bins; ++k) lhist[k] = 0.0;
  for (int i = 0; i < n_threads; ++i) {
    pthread_join(th[i], NULL);
    for (int k = 0; k < 5; ++k) out[k] += jobs[i].out[k];
    if (hist) {
      for (int k = 0; k <= max_scatter; ++k) hist[k] += jobs[i].hist[k];
      free(jobs[i].hist);
    }
    if (lhist) {
      for (int k = 0; k < l_bins; ++k) lhist[k] += jobs[i].lhist[k];
      free(jobs[i].lhist);
    }
  }
  free(jobs);
  free(th);
  return 0;
}

int or_trace_hist(const or_medium* m, const or_source* s, const or_sensor* d,
                  uint64_t seed, uint64_t photon0, uint64_t n_photons, double r_reject,
                  int max_scatter, double* out, double* hist, int n_threads) {
  return trace_run(m, s, d, seed, photon0, n_photons, r_reject, max_scatter, out, hist, 0.0, 0.0, 0, NULL,
                   n_threads);
}

int or_trace_lhist(const or_medium* m, const or_source* s, const or_sensor* d,
                   uint64_t seed, uint64_t photon0, uint64_t n_photons, double r_reject,
                   int max_scatter, double l_lo, double l_hi, int l_bins, double* out, double* lhist,
                   int n_threads) {
  if (!(l_hi > l_lo) || l_bins < 1) return -1;
  return trace_run(m, s, d, seed, photon0, n_photons, r_reject, max_scatter, out, NULL, l_lo, l_hi, l_bins, lhist,
                   n_threads);
}

/* ------------------------------------------------------------------------
 * Relative light yield of two sensors (section "Comparison of relative light
 * yield": B = E_0[sqrt(p_1/p_0)] / E_1[sqrt(p_0/p_1)]; appendix "Relative
 * light yield transformation": the map T of paths ending on sensor 0 to
 * paths ending on sensor 1 by bending them along a cylinder through the
 * source, p_1(x) = p(T x) |dT/dx|).
 *
 * Interior vertices: intermediate coordinates xb = (f - f0).m / b0,
 * yb = (f - f0).n / b0, w = (f - f0).k / b0, then
 *   T f = f0 - rC m + (rC + xb b1)(m cos(w Omega) + k sin(w Omega)) + n yb b1,
 * a cylindrical-coordinate map with volume ratio b1^2 Omega (rC + xb b1) / b0^3.
 * The map is one-to-one where rC + xb b1 > 0 and |w Omega| < pi; outside that
 * domain p_1 is taken as 0, which keeps B = I_1 / I_0 exact (every sensor-1
 * path has its preimage inside the domain).
 * End vertex: the unit offset from sensor 0's centre, rotated in the (m, k) plane
 * by Omega (the turn of the bent path) and scaled by R1/R0, placed about
 * sensor 1's centre: a bijection of the spheres with area ratio (R1/R0)^2.
 * Frame: k = unit vector from the source to sensor 0, m = unit vector normal
 * to k in the plane of k and B = eta1 - f0, pointing away from B, n = k x m;
 * cos Psi = k.B/|B|, rC = |B| / (2 sin Psi), Omega = 2 Psi - R1/rC, b1 = rC Omega,
 * b0 = |eta0 - f0| - R0.
 * ---------------------------------------------------------------------- */
int or_ymap_init(const or_source* s, const or_sensor* d0, const or_sensor* d1, or_ymap* T) {
  double a[3], B[3];
  sub3(d0->c, s->pos, a);
  sub3(d1->c, s->pos, B);
  const double la = norm3(a), lB = norm3(B);
  if (!(la > d0->R) || !(lB > d1->R)) return -1;
  copy3(s->pos, T->f0);
  copy3(d0->c, T->eta0);
  copy3(d1->c, T->eta1);
  T->R0 = d0->R;
  T->R1 = d1->R;
  for (int i = 0; i < 3; ++i) T->k[i] = a[i] / la;
  const double cpsi = dot3(T->k, B) / lB;
  double perp[3];
  for (int i = 0; i < 3; ++i) perp[i] = B[i] / lB - cpsi * T->k[i];
  const double spsi = norm3(perp);
  if (!(spsi > 1e-9)) return -1;
  for (int i = 0; i < 3; ++i) T->m[i] = -perp[i] / spsi;
  T->n[0] = T->k[1] * T->m[2] - T->k[2] * T->m[1];
  T->n[1] = T->k[2] * T->m[0] - T->k[0] * T->m[2];
  T->n[2] = T->k[0] * T->m[1] - T->k[1] * T->m[0];
  const double psi = atan2(spsi, cpsi);
  T->b0 = la - d0->R;
  T->rC = lB / (2.0 * spsi);
  T->Omega = 2.0 * psi - d1->R / T->rC;
  T->b1 = T->rC * T->Omega;
  if (!(T->Omega > 0.0)) return -1;
  return 0;
}

double or_ymap_forward(const or_ymap* T, int n, const double* x, double* y) {
  double lj = 0.0;
  int inside = 1;
  copy3(T->f0, y);
  for (int i = 1; i <= n - 2; ++i) {
    double d[3];
    sub3(&x[3 * i], T->f0, d);
    const double xb = dot3(d, T->m) / T->b0, yb = dot3(d, T->n) / T->b0, w = dot3(d, T->k) / T->b0;
    const double ang = w * T->Omega, rad = T->rC + xb * T->b1;
    if (!(rad > 0.0) || !(fabs(ang) < M_PI)) inside = 0;
    for (int c = 0; c < 3; ++c)
      y[3 * i + c] = T->f0[c] - T->rC * T->m[c] + rad * (T->m[c] * cos(ang) + T->k[c] * sin(ang)) +
                     T->n[c] * yb * T->b1;
    lj += log(T->b1 * T->b1 * T->Omega * fabs(rad) / (T->b0 * T->b0 * T->b0));
  }
  if (n >= 2) {
    double u[3];
    sub3(&x[3 * (n - 1)], T->eta0, u);
    const double lu = norm3(u);  /* the end vertex lies on sensor 0: its unit offset */
    const double um = dot3(u, T->m) / lu, uk = dot3(u, T->k) / lu, un = dot3(u, T->n) / lu;
    const double co = cos(T->Omega), si = sin(T->Omega);
    const double vm = um * co - uk * si, vk = um * si + uk * co;
    for (int c = 0; c < 3; ++c)
      y[3 * (n - 1) + c] = T->eta1[c] + T->R1 * (vm * T->m[c] + vk * T->k[c] + un * T->n[c]);
    lj += 2.0 * log(T->R1 / T->R0);
  }
  return inside ? lj : -INFINITY;
}

double or_ymap_inverse(const or_ymap* T, int n, const double* y, double* x) {
  double lj = 0.0;
  int inside = 1;
  copy3(T->f0, x);
  for (int i = 1; i <= n - 2; ++i) {
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = y[3 * i + c] - (T->f0[c] - T->rC * T->m[c]);
    const double h = dot3(d, T->n), pm = dot3(d, T->m), pk = dot3(d, T->k);
    const double rad = sqrt(pm * pm + pk * pk), ang = atan2(pk, pm);
    if (!(rad > 0.0) || !(fabs(ang) < M_PI)) inside = 0;
    const double xb = (rad - T->rC) / T->b1, yb = h / T->b1, w = ang / T->Omega;
    for (int c = 0; c < 3; ++c) x[3 * i + c] = T->f0[c] + T->b0 * (xb * T->m[c] + yb * T->n[c] + w * T->k[c]);
    lj += log(T->b1 * T->b1 * T->Omega * rad / (T->b0 * T->b0 * T->b0));
  }
  if (n >= 2) {
    double v[3];
    sub3(&y[3 * (n - 1)], T->eta1, v);
    const double lv = norm3(v);
    const double vm = dot3(v, T->m) / lv, vk = dot3(v, T->k) / lv, vn = dot3(v, T->n) / lv;
    const double co = cos(T->Omega), si = sin(T->Omega);
    const double um = vm * co + vk * si, uk = -vm * si + vk * co;
    for (int c = 0; c < 3; ++c)
      x[3 * (n - 1) + c] = T->eta0[c] + T->R0 * (um * T->m[c] + uk * T->k[c] + vn * T->n[c]);
    lj += 2.0 * log(T->R1 / T->R0);
  }
  return inside ? lj : -INFINITY;
}

double or_ymap_logratio(const or_medium* m, const or_source* s, const or_sensor* d0, const or_sensor* d1,
                        const or_ymap* T, int side, int n, const double* path) {
  double* other = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double r;
  if (side == 0) {
    const double lj = or_ymap_forward(T, n, path, other);
    const double lo = isfinite(lj) ? or_logp(m, s, d1, n, other) : -INFINITY;
    r = lo + lj - or_logp(m, s, d0, n, path);
  } else {
    const double lj = or_ymap_inverse(T, n, path, other);
    const double lo = isfinite(lj) ? or_logp(m, s, d0, n, other) : -INFINITY;
    r = lo - lj - or_logp(m, s, d1, n, path);
  }
  free(other);
  return isnan(r) ? -INFINITY : r;
}
