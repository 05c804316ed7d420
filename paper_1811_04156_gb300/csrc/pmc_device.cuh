// Device-side data structures and FP32 factor arithmetic of the path density
// (Collin, arXiv:1811.04156, appendix "Path probability distribution").
//
// All positions on the device are relative to the pair's source (f_0 = 0);
// the absolute height z_abs = z + zoff is only needed by layered media.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pmc {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kLog2Pi = 1.83787706640934548356f;
constexpr float kLog4Pi = 2.53102424696929079f;
constexpr float kNegInf = -__builtin_huge_valf();

// ---------------------------------------------------------------------------
// Scene constants (built on the host, passed by value)
// ---------------------------------------------------------------------------
struct DMedium {
  int kind;            // 0 homogeneous, 1 layered
  float a, b;          // homogeneous coefficients (1/m)
  float log_b;         // log b (homogeneous)
  float g, f_sl;
  float hg_lognorm;    // log(0.5 (1 - g^2)) - log(2 pi): HG per steradian
  float omg2;          // (1 - g)^2
  float two_g;         // 2 g
  float hg_dg0;        // -2 g / (1 - g^2)
  float sl_alpha;      // 2 g / (1 - g)
  float sl_lognorm;    // log(0.5 (1 + g)/(1 - g)) - log(2 pi)
  float sl_dg0;        // 2 / (1 - g^2)
  float sl_dg1;        // 2 / (1 - g)^2
  float kappa_eq;      // solves coth k - 1/k = g
  int n_layers;
  float z0, dz, inv_dz;
  const float* la;     // [n_layers] absorption coefficient per layer
  const float* lb;     // [n_layers] scattering coefficient per layer
  const float* llogb;  // [n_layers] log of lb
  float lam0, ks, ka;  // wavelength dependence: b ~ (l / lam0)^-ks, a ~ (l / lam0)^-ka (homogeneous)
};

struct DPair {
  float org[3];        // absolute position of the frame origin (the source, or 0)
  float src[3];        // source position in the frame of this struct
  float c[3];          // sensor centre in the frame (high part)
  float c_lo[3];       // low part: centre = c + c_lo to ~2^-48 relative
  float zoff;          // absolute height of the frame origin (layered media)
  float R, R2;
  int emission;        // 0 isotropic, 1 vMF
  float kappa, vmf_lognorm;
  float dir[3];
  int rho;             // 0 one, 1 paper
  float rho_hat[3];
  int cap, n_chains, chain0;
  float kappa_end, exp_m2ke;   // vMF end moves: kappa and exp(-2 kappa)
  float e_near[3];     // sensor point nearest the source (relative)
};

struct DRun {
  unsigned long long seed;
  uint32_t thr_within, thr_birth;  // 23-bit thresholds of the move draw
  float log_pb, log_pd;            // log p_birth, log p_death
  float sigma, mala_eps;
  int within;                      // 0 perturb, 1 MALA, 2 tree, 3 HMC
  int hmc_steps;                   // HMC: leapfrog steps of size mala_eps
  unsigned long long burn_in;
  float beta_min;
  int gradients;
  // wavelength sampled with the path: n_spec >= 2 nodes of the normalised
  // piecewise-linear spectrum (spec_x increasing, nm; spec_y densities per nm), 0 = off
  int n_spec;
  const float* spec_x;
  const float* spec_y;
  float sigma_lam;                 // Gaussian step of a wavelength move (nm)
};

// ---------------------------------------------------------------------------
// Small vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 ld3(const float* p) { return f3(p[0], p[1], p[2]); }

// ---------------------------------------------------------------------------
// Math policy: F = false uses the accurate CUDA functions (density kernels on
// caller batches, compared with the FP64 oracle to 1e-5); F = true uses the
// SFU approximations (chain kernel: a few ulp, far below the Monte-Carlo
// error, and every decision stays a function of the stored FP32 state).
// ---------------------------------------------------------------------------
template <bool F>
__device__ __forceinline__ float m_log(float x) {
  if constexpr (F) return __logf(x);
  else return logf(x);
}
template <bool F>
__device__ __forceinline__ float m_exp(float x) {
  if constexpr (F) return __expf(x);
  else return expf(x);
}
template <bool F>
__device__ __forceinline__ float m_sqrt(float x) {
  if constexpr (F) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  } else {
    return sqrtf(x);
  }
}
template <bool F>
__device__ __forceinline__ float m_div(float a, float b) {
  if constexpr (F) return __fdividef(a, b);
  else return a / b;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), counter (c0..c3), key (k0, k1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ((x >> 9) + 1/2) * 2^-23: exact in FP32, in (0, 1).
__device__ __forceinline__ float u01(uint32_t x) {
  return __fmaf_rn(static_cast<float>(x >> 9), 1.1920928955078125e-7f, 5.9604644775390625e-8f);
}
// floor(23-bit fraction * m), in integers.
__device__ __forceinline__ uint32_t index_draw(uint32_t x, uint32_t m) {
  return static_cast<uint32_t>((static_cast<unsigned long long>(x >> 9) * m) >> 23);
}

// Orthonormal completion of a unit vector (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb(float3 n, float3& e1, float3& e2) {
  const float sign = copysignf(1.0f, n.z);
  const float a = -1.0f / (sign + n.z);
  const float b = n.x * n.y * a;
  e1 = f3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  e2 = f3(b, sign + n.y * n.y * a, -n.y);
}

// ---------------------------------------------------------------------------
// Medium
// ---------------------------------------------------------------------------
__device__ __forceinline__ int layer_of(const DMedium& M, float z_abs) {
  const float f = floorf((z_abs - M.z0) * M.inv_dz);
  int l = static_cast<int>(fminf(fmaxf(f, 0.0f), static_cast<float>(M.n_layers - 1)));
  return l;
}

__device__ __forceinline__ float log_b_at(const DMedium& M, float z_abs) {
  if (M.kind == 0) return M.log_b;
  return __ldg(M.llogb + layer_of(M, z_abs));
}

__device__ __forceinline__ float b_at(const DMedium& M, float z_abs) {
  if (M.kind == 0) return M.b;
  return __ldg(M.lb + layer_of(M, z_abs));
}

// Optical depths of the segment from height zP to zQ (absolute) with length
// ell: tau = ell * (mean coefficient over [zP, zQ]).  Layered media add the
// coefficient of each crossed layer weighted by its share of the height span.
__device__ __forceinline__ void seg_tau(const DMedium& M, float zP, float zQ, float ell,
                                        float& ta, float& tb) {
  if (M.kind == 0) {
    ta = M.a * ell;
    tb = M.b * ell;
    return;
  }
  const int lP = layer_of(M, zP), lQ = layer_of(M, zQ);
  if (lP == lQ) {
    ta = __ldg(M.la + lP) * ell;
    tb = __ldg(M.lb + lP) * ell;
    return;
  }
  const float zlo = fminf(zP, zQ), zhi = fmaxf(zP, zQ);
  const int l0 = min(lP, lQ), l1 = max(lP, lQ);
  const float inv_span = 1.0f / (zhi - zlo);
  float sa = 0.0f, sb = 0.0f;
  for (int l = l0; l <= l1; ++l) {
    const float lo = (l == l0) ? zlo : M.z0 + l * M.dz;
    const float hi = (l == l1) ? zhi : M.z0 + (l + 1) * M.dz;
    const float w = fmaxf(hi - lo, 0.0f) * inv_span;
    sa = fmaf(__ldg(M.la + l), w, sa);
    sb = fmaf(__ldg(M.lb + l), w, sb);
  }
  ta = sa * ell;
  tb = sb * ell;
}

// ---------------------------------------------------------------------------
// Factors of the path density
// ---------------------------------------------------------------------------

// log of the phase density per steradian at the angle between unit
// directions a (incoming) and b (outgoing), and its derivative in g.
// 1 - cos and 1 + cos come from |a - b|^2 / 2 and |a + b|^2 / 2, which stay
// accurate for the forward-peaked angles that dominate at g ~ 0.9.
template <bool F = false, bool kMix = true>
__device__ __forceinline__ float phase_term(const DMedium& M, float3 a, float3 b, float& gterm) {
  const float3 dm = a - b;
  const float omc = 0.5f * dot(dm, dm);
  const float den = fmaf(M.two_g, omc, M.omg2);
  const float lhg = fmaf(-1.5f, m_log<F>(den), M.hg_lognorm);
  const float ghg = M.hg_dg0 - 3.0f * m_div<F>(M.g - 1.0f + omc, den);
  if (!kMix || M.f_sl <= 0.0f) {
    gterm = ghg;
    return lhg;
  }
  const float3 dp = a + b;
  const float opc = 0.5f * dot(dp, dp);
  const float lv = m_log<F>(0.5f * opc);
  const float lsl = fmaf(M.sl_alpha, lv, M.sl_lognorm);
  const float gsl = fmaf(M.sl_dg1, lv, M.sl_dg0);
  const float mx = fmaxf(lhg, lsl);
  const float wh = (1.0f - M.f_sl) * m_exp<F>(lhg - mx);
  const float ws = M.f_sl * m_exp<F>(lsl - mx);
  gterm = m_div<F>(wh * ghg + ws * gsl, wh + ws);
  return mx + m_log<F>(wh + ws);
}

// d log sigma / d cos(theta) for unit directions a, b.
__device__ __forceinline__ float phase_dlogdc(const DMedium& M, float3 a, float3 b) {
  const float3 dm = a - b, dp = a + b;
  const float omc = 0.5f * dot(dm, dm);
  const float opc = 0.5f * dot(dp, dp);
  const float den = fmaf(M.two_g, omc, M.omg2);
  const float dhg = 3.0f * M.g / den;
  if (M.f_sl <= 0.0f) return dhg;
  const float lv = logf(0.5f * opc);
  const float lhg = fmaf(-1.5f, logf(den), M.hg_lognorm);
  const float lsl = fmaf(M.sl_alpha, lv, M.sl_lognorm);
  const float mx = fmaxf(lhg, lsl);
  const float wh = (1.0f - M.f_sl) * expf(lhg - mx);
  const float ws = M.f_sl * expf(lsl - mx);
  return (wh * dhg + ws * (M.sl_alpha / opc)) / (wh + ws);
}

// Emission factor p_i (Eq. emission_dist) for the first direction b.
__device__ __forceinline__ float emission_term(const DPair& P, float3 b) {
  if (P.emission == 0) return -kLog4Pi;
  return fmaf(P.kappa, dot(b, f3(P.dir[0], P.dir[1], P.dir[2])), P.vmf_lognorm);
}

// Outward unit normal of the sensor at e.  e - c_hi is exact when e lies near
// the sphere (Sterbenz), so the normal keeps full FP32 accuracy however far
// the sensor is from the frame origin.
__device__ __forceinline__ float3 sensor_normal(const DPair& P, float3 e) {
  float3 nu = (e - f3(P.c[0], P.c[1], P.c[2])) - f3(P.c_lo[0], P.c_lo[1], P.c_lo[2]);
  return rsqrtf(dot(nu, nu)) * nu;
}

// Detection factor of p_f without its 1/|r|^2: log max(0, -a . nu) + log rho(nu)
// (Eq. detection_prob), for the last direction a and end vertex e.
template <bool F = false>
__device__ __forceinline__ float sensor_term(const DPair& P, float3 a, float3 e) {
  const float3 nu = sensor_normal(P, e);
  const float cphi = -dot(a, nu);
  if (!(cphi > 0.0f)) return kNegInf;
  float t = m_log<F>(cphi);
  if (P.rho != 0) {
    const float x = dot(nu, f3(P.rho_hat[0], P.rho_hat[1], P.rho_hat[2]));
    t += fmaf(3.0f, x, -1.0f) - logf(coshf(fmaf(2.0f, x, 0.7f)));
  }
  return t;
}

// Does the segment P -> P + r touch the sensor ball?
template <bool F = false>
__device__ __forceinline__ bool hits_ball(const DPair& S, float3 P, float3 r) {
  const float3 c = f3(S.c[0], S.c[1], S.c[2]);
  const float rr = dot(r, r);
  float t = m_div<F>(dot(c - P, r), rr);
  t = fminf(fmaxf(t, 0.0f), 1.0f);
  const float3 d = P + t * r - c;
  return dot(d, d) <= S.R2;
}

// Segment factor -tau_a - tau_b - 2 log ell (the 1/|r|^2 of Eq. intervtx and
// of p_f, with the survival of Eq. b_depth_def), plus tau_b and ell.
struct SegOut {
  float seg, tb, len;
};

__device__ __forceinline__ SegOut segment_term(const DMedium& M, const DPair& S, float zoff, float3 P,
                                               float3 Q, bool non_final) {
  const float3 r = Q - P;
  const float l2 = dot(r, r);
  const float ell = sqrtf(l2);
  float ta, tb;
  seg_tau(M, P.z + zoff, Q.z + zoff, ell, ta, tb);
  SegOut o;
  o.seg = -(ta + tb) - logf(l2);
  o.tb = tb;
  o.len = ell;
  if (!(l2 > 0.0f)) o.seg = kNegInf;
  if (non_final && hits_ball(S, P, r)) o.seg = kNegInf;
  return o;
}

// Vertex factor of vertex v of an n-vertex path from its neighbours:
// emission at v = 0, detection at v = n-1, else log b + log sigma/(2 pi).
// gterm receives d log sigma / d g for interior vertices (0 otherwise).
__device__ __forceinline__ float vertex_term(const DMedium& M, const DPair& S, float zoff, float3 Pp,
                                             float3 P, float3 Pn, int v, int n, float& gterm) {
  gterm = 0.0f;
  if (v == 0) {
    const float3 b = Pn - P;
    return emission_term(S, rsqrtf(dot(b, b)) * b);
  }
  const float3 a0 = P - Pp;
  const float3 a = rsqrtf(dot(a0, a0)) * a0;
  if (v == n - 1) return sensor_term(S, a, P);
  const float3 b0 = Pn - P;
  const float3 b = rsqrtf(dot(b0, b0)) * b0;
  return log_b_at(M, P.z + zoff) + phase_term(M, a, b, gterm);
}

// ---------------------------------------------------------------------------
// Gradient of log p with respect to vertex v (adjoint and MALA)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dtau_dends(const DMedium& M, float zoff, float3 P, float3 Q, float ell,
                                           float3 rhat, float3& dP, float3& dQ) {
  float ta, tb;
  seg_tau(M, P.z + zoff, Q.z + zoff, ell, ta, tb);
  const float cbar = (ta + tb) / ell;
  dQ = cbar * rhat;
  dP = -cbar * rhat;
  if (M.kind != 0) {
    const int lP = layer_of(M, P.z + zoff), lQ = layer_of(M, Q.z + zoff);
    if (lP != lQ) {
      const float cP = __ldg(M.la + lP) + __ldg(M.lb + lP);
      const float cQ = __ldg(M.la + lQ) + __ldg(M.lb + lQ);
      const float dz = Q.z - P.z;
      dQ.z += ell * (cQ - cbar) / dz;
      dP.z += ell * (cbar - cP) / dz;
    }
  }
}

// d(rhat . w)/d(end point) for a segment of length ell and direction rhat.
__device__ __forceinline__ float3 drdot(float3 rhat, float ell, float3 w) {
  return (1.0f / ell) * (w - dot(rhat, w) * rhat);
}

template <class PosF>
__device__ float3 grad_vertex(const DMedium& M, const DPair& S, float zoff, PosF pos, int n, int v) {
  float3 rh[4];
  float el[4];
  bool ex[4];
  float3 pv[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int k = v - 2 + i;
    pv[i] = (k >= 0 && k <= n - 1) ? pos(k) : f3(0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = v - 2 + i;  // segment k: vertex k -> k+1
    ex[i] = (k >= 0 && k <= n - 2);
    const float3 r = pv[i + 1] - pv[i];
    el[i] = ex[i] ? sqrtf(dot(r, r)) : 1.0f;
    rh[i] = (1.0f / el[i]) * r;
  }
  float3 g = f3(0.f, 0.f, 0.f);
  // segment v-1 ends at v, segment v starts at v
  if (ex[1]) {
    float3 dP, dQ;
    dtau_dends(M, zoff, pv[1], pv[2], el[1], rh[1], dP, dQ);
    g = g - dQ - (2.0f / el[1]) * rh[1];
  }
  if (ex[2]) {
    float3 dP, dQ;
    dtau_dends(M, zoff, pv[2], pv[3], el[2], rh[2], dP, dQ);
    g = g - dP + (2.0f / el[2]) * rh[2];
  }
  // emission
  if (S.emission != 0) {
    const float3 ed = f3(S.dir[0], S.dir[1], S.dir[2]);
    if (v == 1) g = g + S.kappa * drdot(rh[1], el[1], ed);
    if (v == 0 && ex[2]) g = g - S.kappa * drdot(rh[2], el[2], ed);
  }
  // interior angles at v-1, v, v+1
  if (v - 1 >= 1 && v - 1 <= n - 2) {
    const float w = phase_dlogdc(M, rh[0], rh[1]);
    g = g + w * drdot(rh[1], el[1], rh[0]);
  }
  if (v >= 1 && v <= n - 2) {
    const float w = phase_dlogdc(M, rh[1], rh[2]);
    g = g + w * (drdot(rh[1], el[1], rh[2]) - drdot(rh[2], el[2], rh[1]));
  }
  if (v + 1 >= 1 && v + 1 <= n - 2) {
    const float w = phase_dlogdc(M, rh[2], rh[3]);
    g = g - w * drdot(rh[2], el[2], rh[3]);
  }
  // detection term log(-rhat_{n-2} . nu) + log rho(nu)
  if (v == n - 2 || v == n - 1) {
    const float3 e = (v == n - 1) ? pv[2] : pv[3];
    const float3 rhat = (v == n - 1) ? rh[1] : rh[2];
    const float ell = (v == n - 1) ? el[1] : el[2];
    float3 nu = (e - f3(S.c[0], S.c[1], S.c[2])) - f3(S.c_lo[0], S.c_lo[1], S.c_lo[2]);
    const float dn = sqrtf(dot(nu, nu));
    nu = (1.0f / dn) * nu;
    const float u = -dot(rhat, nu);
    const float3 t1 = drdot(rhat, ell, nu);
    if (v == n - 2) {
      g = g + (1.0f / u) * t1;
    } else {
      const float3 t2 = drdot(nu, dn, rhat);
      g = g - (1.0f / u) * (t1 + t2);
      if (S.rho != 0) {
        const float3 rh_ = f3(S.rho_hat[0], S.rho_hat[1], S.rho_hat[2]);
        const float x = dot(nu, rh_);
        const float dl = 3.0f - 2.0f * tanhf(fmaf(2.0f, x, 0.7f));
        g = g + dl * drdot(nu, dn, rh_);
      }
    }
  }
  return g;
}

// ---------------------------------------------------------------------------
// Insertion density of a vertex f between foci A and B (appendix, dimension
// matching transformation): q(s) q(t) q(phi) / J, written with the distances
// d1 = |f - A|, d2 = |f - B| and 2 gamma = |B - A|, using
//   cosh t - cos s = 2 gamma^2 / (d1 d2),  q(t) = d1 d2 / (d1 + d2)^2,
// so that log density = log q_c(cos s) + 3 log(2 gamma) - 2 log(d1 d2 (d1 + d2)) - log 2pi,
// with q_c(c) = beta exp(-beta c) / (2 sinh beta).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float insertion_beta(const DMedium& M, const DRun& R, float zoff, float3 A,
                                                float3 B, float gamma) {
  const float zmid = 0.5f * (A.z + B.z) + zoff;
  const float beta = M.kappa_eq + 0.5f * (gamma * b_at(M, zmid) - 1.0f);
  return fmaxf(beta, R.beta_min);
}

template <bool F = false>
__device__ __forceinline__ float log_insert_density(const DMedium& M, const DRun& R, float zoff, float3 A,
                                                    float3 B, float3 f) {
  const float3 ab = B - A;
  const float gamma = 0.5f * m_sqrt<F>(dot(ab, ab));
  const float3 u = A - f, w = B - f;
  const float d1 = m_sqrt<F>(dot(u, u)), d2 = m_sqrt<F>(dot(w, w));
  const float cs = m_div<F>(dot(u, w), d1 * d2);
  const float beta = insertion_beta(M, R, zoff, A, B, gamma);
  const float log2sinh = beta + m_log<F>(1.0f - m_exp<F>(-2.0f * beta));
  return m_log<F>(beta) - beta * cs - log2sinh + 3.0f * m_log<F>(2.0f * gamma) -
         2.0f * m_log<F>(d1 * d2 * (d1 + d2)) - kLog2Pi;
}

// ---------------------------------------------------------------------------
// Wavelength as a sampled coordinate (section "Discussion": a wavelength
// parameter in the path density, sampled along with the vertices).  The
// chains sample S(l) p_l(path): S the normalised piecewise-linear spectrum,
// p_l the path density of the homogeneous medium whose coefficients follow
// power laws in l / lam0.
// ---------------------------------------------------------------------------
__device__ inline float spectrum_log(const DRun& R, float lam) {
  const int K = R.n_spec;
  if (!(lam >= R.spec_x[0]) || !(lam <= R.spec_x[K - 1])) return kNegInf;
  int i = 0;
  while (i + 2 < K && lam > R.spec_x[i + 1]) ++i;
  const float x0 = R.spec_x[i], x1 = R.spec_x[i + 1], y0 = R.spec_y[i], y1 = R.spec_y[i + 1];
  const float v = fmaf(y1 - y0, (lam - x0) / (x1 - x0), y0);
  return v > 0.f ? logf(v) : kNegInf;
}

// Wavelength at which the spectrum's CDF equals u: walk the intervals'
// trapezoid areas, then solve y0 s + k s^2 / 2 = t (k the slope) as
// s = 2 t / (y0 + sqrt(y0^2 + 2 k t)).
__device__ inline float spectrum_quantile(const DRun& R, float u) {
  const int K = R.n_spec;
  float t = u;
  for (int i = 0; i + 1 < K; ++i) {
    const float h = R.spec_x[i + 1] - R.spec_x[i];
    const float y0 = R.spec_y[i], y1 = R.spec_y[i + 1];
    const float area = 0.5f * h * (y0 + y1);
    if (t <= area || i + 2 == K) {
      const float k = (y1 - y0) / h;
      const float den = y0 + sqrtf(fmaxf(fmaf(2.0f * k, t, y0 * y0), 0.f));
      const float sv = den > 0.f ? 2.0f * t / den : 0.f;
      return R.spec_x[i] + fminf(fmaxf(sv, 0.f), h);
    }
    t -= area;
  }
  return R.spec_x[K - 1];
}

// The homogeneous medium at wavelength lam (coefficients scaled, log b with them).
__device__ __forceinline__ void medium_at(const DMedium& M0, float lam, DMedium& out) {
  out = M0;
  const float r = logf(lam / M0.lam0);
  out.b = M0.b * expf(-M0.ks * r);
  out.a = M0.a * expf(-M0.ka * r);
  out.log_b = M0.log_b - M0.ks * r;
}

// ---------------------------------------------------------------------------
// Chain kernels (warp per chain and lane per chain)
// ---------------------------------------------------------------------------
// Factors attached to vertex v of an n-vertex path: its vertex factor (and
// d log sigma / d g) and, when v <= n-2, the factor of the segment v -> v+1.
template <bool kGen>
__device__ __forceinline__ void vertex_and_segment(const DMedium& M, const DPair& S, float zoff, float3 Pp, float3 Pc,
                                                   float3 Pn, int v, int n, float& vt, float& gt, float& seg,
                                                   float& tb, float& len) {
  constexpr bool F = true;  // SFU forms
  gt = 0.f;
  seg = 0.f;
  tb = 0.f;
  len = 0.f;
  const float3 b0 = Pn - Pc;
  const float bb = dot(b0, b0);
  const float ib = rsqrtf(bb);
  const float3 b = ib * b0;
  if (v <= n - 2) {
    const float ell = bb * ib;
    float ta, tbv;
    if constexpr (kGen) {
      seg_tau(M, Pc.z + zoff, Pn.z + zoff, ell, ta, tbv);
    } else {
      ta = M.a * ell;
      tbv = M.b * ell;
    }
    seg = -(ta + tbv) - m_log<F>(bb);
    tb = tbv;
    len = ell;
    if (!(bb > 0.0f)) seg = kNegInf;
    if (v <= n - 3 && hits_ball<F>(S, Pc, b0)) seg = kNegInf;
  }
  if (v == 0) {
    if constexpr (kGen) vt = emission_term(S, b);
    else vt = -kLog4Pi;
    return;
  }
  const float3 a0 = Pc - Pp;
  const float3 a = rsqrtf(dot(a0, a0)) * a0;
  if (v == n - 1) {
    vt = sensor_term<F>(S, a, Pc);
    return;
  }
  const float lb = kGen ? log_b_at(M, Pc.z + zoff) : M.log_b;
  vt = lb + phase_term<F, kGen>(M, a, b, gt);
}

}  // namespace pmc
