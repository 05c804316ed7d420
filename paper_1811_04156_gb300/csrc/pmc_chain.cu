// Persistent RJMCMC chain kernel: one warp per chain, the chain's path staged
// in shared memory as SoA arrays with per-segment and per-vertex caches of the
// log-density factors (Collin, arXiv:1811.04156: section "Numerical path
// integration", Eq. acceptFact; appendix "Jump proposal" and "Dimension
// matching transformation").
//
// Per warp and per step:
//   * random numbers: every 32 steps each lane draws the two Philox4x32-10
//     blocks of one future step, pre-transforms them (Box-Muller normals, vMF
//     cosine, logistic t, log u) and stores 8 words in the warp's shared
//     staging row; each step then reads its row with two broadcast loads;
//   * delta evaluator: a move changes at most 3 vertex factors and 2 segment
//     factors; lane i evaluates vertex factor i and segment factor i of the
//     changed window in parallel, the old values come from the caches, and
//     two shuffles give the change of log p;
//   * accept / commit: births and deaths shift the SoA arrays with the whole
//     warp; caches of the changed window are written back.
// Two instantiations: kGen = false is the lean kernel for a homogeneous
// medium, isotropic emission, detection probability 1, pure Henyey-Greenstein
// phase function and Gaussian perturbations; kGen = true handles layered
// media, vMF emission, the paper's detection probability, the simplified-Liu
// mixture and MALA moves.
// Estimators: observables (n, length L, sum of d log sigma/dg) change only on
// acceptance, so each state's values are added once with its dwell time into
// FP32 partials that are flushed into lane-distributed FP64 accumulators.
// kTree adds the paper's within-dimension move in tree coordinates (section
// "Path proposal distribution"; appendix "Path space coordinate system"): the
// whole path is re-expressed node by node in recursive bispherical systems,
// every node's (zeta, t, phi) takes a normal step, and the new path is built
// level by level into three extra shared arrays.
#include <climits>

#include "pmc_internal.h"
#include "pmc_tree.cuh"

namespace pmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRefreshSteps = 256;  // recompute the running sums from the caches
constexpr int kFlushAccepts = 64;   // FP32 partials -> FP64 accumulators
constexpr int kRngWords = 8;        // staged words per step
constexpr int kPairWords = 64;      // shared slot for the pair constants (floats)
static_assert(sizeof(DPair) <= kPairWords * sizeof(float), "pair slot too small");
constexpr int kMedWords = 48;       // wavelength sampling: the medium at the chain's wavelength (floats)
static_assert(sizeof(DMedium) <= kMedWords * sizeof(float), "medium slot too small");

enum Move { MV_INTERIOR = 0, MV_END = 1, MV_BIRTH = 2, MV_DEATH = 3 };

// View of one chain's path: entries [0, S) of every array live in the warp's
// shared memory, entries [S, cap) in the chain's global block (same layout:
// array a at offset a * stride).  kTb: tau_b per segment is cached (layered
// media); otherwise it is b * length.  kGt: d log sigma / dg per vertex is
// cached (gradients requested).  kSpill = false: the whole cap fits (S >= cap)
// and every access goes to shared memory.
template <bool kTb, bool kGt, bool kSpill>
struct WarpPath {
  static constexpr int kArrays = 6 + (kTb ? 1 : 0) + (kGt ? 1 : 0);
  static constexpr int kX = 0, kY = 1, kZ = 2, kSeg = 3, kLen = 4, kVt = 5, kTbA = 6, kGtA = 6 + (kTb ? 1 : 0);
  float* sm;   // shared arrays, stride S
  float* gm;   // global block of the chain, stride cap
  int S, cap;
  float b;
  template <int a>
  __device__ __forceinline__ float ld(int i) const {
    if (kSpill && i >= S) return gm[a * cap + i];
    return sm[a * S + i];
  }
  template <int a>
  __device__ __forceinline__ void st(int i, float v) const {
    if (kSpill && i >= S) gm[a * cap + i] = v;
    else sm[a * S + i] = v;
  }
  __device__ float3 pos(int i) const { return f3(ld<kX>(i), ld<kY>(i), ld<kZ>(i)); }
  __device__ void set_pos(int i, float3 p) const {
    st<kX>(i, p.x);
    st<kY>(i, p.y);
    st<kZ>(i, p.z);
  }
  __device__ float seg(int i) const { return ld<kSeg>(i); }
  __device__ float len(int i) const { return ld<kLen>(i); }
  __device__ float vt(int i) const { return ld<kVt>(i); }
  __device__ void set_seg(int i, float v) const { st<kSeg>(i, v); }
  __device__ void set_len(int i, float v) const { st<kLen>(i, v); }
  __device__ void set_vt(int i, float v) const { st<kVt>(i, v); }
  __device__ float tb(int i) const {
    if constexpr (kTb) return ld<kTbA>(i);
    else return b * ld<kLen>(i);
  }
  __device__ float gt(int i) const {
    if constexpr (kGt) return ld<kGtA>(i);
    else return 0.f;
  }
  __device__ void set_tb(int i, float v) const {
    if constexpr (kTb) st<kTbA>(i, v);
  }
  __device__ void set_gt(int i, float v) const {
    if constexpr (kGt) st<kGtA>(i, v);
  }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// d log p / d f_v with the terms spread over lanes: lanes 0-1 the two segment
// factors that end / start at v, lanes 2-4 the scattering angles at v-1, v,
// v+1, lane 5 the emission and detection factors; a shuffle tree sums them
// and every lane returns the total.  Same formulas as grad_vertex.
template <class PosF>
__device__ float3 grad_vertex_warp(const DMedium& M, const DPair& S, float zoff, PosF pos, int n, int v, int lane) {
  float3 pv[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int k = min(max(v - 2 + i, 0), n - 1);
    pv[i] = pos(k);
  }
  float3 rh[4];
  float el[4];
  bool ex[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = v - 2 + i;
    ex[i] = (k >= 0 && k <= n - 2);
    const float3 r = pv[i + 1] - pv[i];
    const float rr = dot(r, r);
    const float ir = ex[i] ? rsqrtf(rr) : 1.0f;
    el[i] = ex[i] ? rr * ir : 1.0f;
    rh[i] = ir * r;
  }
  float3 g = f3(0.f, 0.f, 0.f);
  if (lane < 2) {
    const bool e = (lane == 0) ? ex[1] : ex[2];
    const float3 P = (lane == 0) ? pv[1] : pv[2];
    const float3 Q = (lane == 0) ? pv[2] : pv[3];
    const float3 r = (lane == 0) ? rh[1] : rh[2];
    const float l = (lane == 0) ? el[1] : el[2];
    if (e) {
      float3 dP, dQ;
      dtau_dends(M, zoff, P, Q, l, r, dP, dQ);
      g = (lane == 0) ? (f3(0.f, 0.f, 0.f) - dQ - (2.0f / l) * r) : ((2.0f / l) * r - dP);
    }
  } else if (lane < 5) {
    const int k = v - 3 + lane;
    if (k >= 1 && k <= n - 2) {
      const float3 A = (lane == 2) ? rh[0] : ((lane == 3) ? rh[1] : rh[2]);
      const float3 B = (lane == 2) ? rh[1] : ((lane == 3) ? rh[2] : rh[3]);
      const float lA = (lane == 2) ? el[0] : ((lane == 3) ? el[1] : el[2]);
      const float lB = (lane == 2) ? el[1] : ((lane == 3) ? el[2] : el[3]);
      const float alpha = (lane == 2) ? 0.f : ((lane == 3) ? 1.f : -1.f);
      const float beta = (lane == 2) ? 1.f : ((lane == 3) ? -1.f : 0.f);
      const float w = phase_dlogdc(M, A, B);
      g = w * (alpha * drdot(A, lA, B) + beta * drdot(B, lB, A));
    }
  } else if (lane == 5) {
    if (S.emission != 0) {
      const float3 ed = f3(S.dir[0], S.dir[1], S.dir[2]);
      if (v == 1) g = g + S.kappa * drdot(rh[1], el[1], ed);
      if (v == 0 && ex[2]) g = g - S.kappa * drdot(rh[2], el[2], ed);
    }
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
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    g.x += __shfl_xor_sync(kFull, g.x, o);
    g.y += __shfl_xor_sync(kFull, g.y, o);
    g.z += __shfl_xor_sync(kFull, g.z, o);
  }
  return f3(__shfl_sync(kFull, g.x, 0), __shfl_sync(kFull, g.y, 0), __shfl_sync(kFull, g.z, 0));
}

struct Sums {
  float L, G;
};

template <class WP>
__device__ Sums path_sums(const WP& w, int n, int lane) {
  float L = 0.f, G = 0.f;
  for (int i = lane; i < n; i += 32) {
    G += w.gt(i);
    if (i <= n - 2) L += w.len(i);
  }
  Sums s;
  s.L = warp_sum(L);
  s.G = warp_sum(G);
  return s;
}

// The general density's vertex and segment factors.  kCall: as one
// out-of-line function, so that the kernel holds a single copy of them.  The
// general tree-move kernel takes it: its warps sit in different phases of a
// long step (tree levels, births, deaths) and instruction fetch limits it
// (8 % faster on the paper's two-sensor scene); the general Cartesian kernel,
// whose step is short, runs a third slower with the call and keeps them
// inline.
struct VsOut {
  float vt, gt, seg, tb, len;
};
__device__ __noinline__ VsOut vs_general(const DMedium& M, const DPair& S, float zoff, float3 Pp, float3 Pc, float3 Pn,
                                        int v, int n) {
  VsOut o;
  vertex_and_segment<true>(M, S, zoff, Pp, Pc, Pn, v, n, o.vt, o.gt, o.seg, o.tb, o.len);
  return o;
}
template <bool kGen, bool kCall>
__device__ __forceinline__ void vs_factors(const DMedium& M, const DPair& S, float zoff, float3 Pp, float3 Pc,
                                           float3 Pn, int v, int n, float& vt, float& gt, float& seg, float& tb,
                                           float& len) {
  if constexpr (kGen && kCall) {
    const VsOut o = vs_general(M, S, zoff, Pp, Pc, Pn, v, n);
    vt = o.vt;
    gt = o.gt;
    seg = o.seg;
    tb = o.tb;
    len = o.len;
  } else {
    vertex_and_segment<kGen>(M, S, zoff, Pp, Pc, Pn, v, n, vt, gt, seg, tb, len);
  }
}

// Recompute every cached factor of the path from its vertices; returns log p.
template <bool kGen, bool kCall, class WP>
__device__ float refresh_caches(const DMedium& M, const DPair& S, float zoff, const WP& w, int n, int lane) {
  float lp = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float3 P = w.pos(i);
    const float3 Pp = (i >= 1) ? w.pos(i - 1) : P;
    const float3 Pn = (i <= n - 2) ? w.pos(i + 1) : P;
    float vt, gt, seg, tb, len;
    vs_factors<kGen, kCall>(M, S, zoff, Pp, P, Pn, i, n, vt, gt, seg, tb, len);
    w.set_vt(i, vt);
    w.set_gt(i, gt);
    lp += vt;
    if (i <= n - 2) {
      w.set_seg(i, seg);
      w.set_tb(i, tb);
      w.set_len(i, len);
      lp += seg;
    }
  }
  __syncwarp();
  return warp_sum(lp);
}

// Shift entries [a, e) of the vertex-indexed and segment-indexed arrays.
template <class WP>
__device__ void shift_right(const WP& w, int a, int e_vtx, int e_seg, int lane) {
  for (int base = e_vtx - 1; base >= a; base -= 32) {
    const int i = base - lane;
    const bool ok = i >= a;
    const bool oks = ok && i < e_seg;
    float x = 0, y = 0, z = 0, vt = 0, gt = 0, tb = 0, sg = 0, ln = 0;
    if (ok) { x = w.template ld<WP::kX>(i); y = w.template ld<WP::kY>(i); z = w.template ld<WP::kZ>(i); vt = w.vt(i); gt = w.gt(i); }
    if (oks) { tb = w.tb(i); sg = w.seg(i); ln = w.len(i); }
    __syncwarp();
    if (ok) { w.set_pos(i + 1, f3(x, y, z)); w.set_vt(i + 1, vt); w.set_gt(i + 1, gt); }
    if (oks) { w.set_tb(i + 1, tb); w.set_seg(i + 1, sg); w.set_len(i + 1, ln); }
    __syncwarp();
  }
}

template <class WP>
__device__ void shift_left(const WP& w, int a, int e_vtx, int e_seg, int lane) {
  for (int base = a; base < e_vtx; base += 32) {
    const int i = base + lane;
    const bool ok = i < e_vtx;
    const bool oks = i < e_seg;
    float x = 0, y = 0, z = 0, vt = 0, gt = 0, tb = 0, sg = 0, ln = 0;
    if (ok) { x = w.template ld<WP::kX>(i); y = w.template ld<WP::kY>(i); z = w.template ld<WP::kZ>(i); vt = w.vt(i); gt = w.gt(i); }
    if (oks) { tb = w.tb(i); sg = w.seg(i); ln = w.len(i); }
    __syncwarp();
    if (ok) { w.set_pos(i - 1, f3(x, y, z)); w.set_vt(i - 1, vt); w.set_gt(i - 1, gt); }
    if (oks) { w.set_tb(i - 1, tb); w.set_seg(i - 1, sg); w.set_len(i - 1, ln); }
    __syncwarp();
  }
}

// Segment chosen for a birth: smallest k with cumsum_k(tau_b) > u * T_b.
template <class WP>
__device__ int select_segment(const WP& w, int nseg, float u, float& total, int lane) {
  if (nseg <= 32) {
    // one segment per lane: inclusive scan, then the first lane past the target
    float incl = (lane < nseg) ? w.tb(lane) : 0.f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    total = __shfl_sync(kFull, incl, 31);
    const unsigned over = __ballot_sync(kFull, lane < nseg && incl > u * total);
    return over ? (__ffs(over) - 1) : (nseg - 1);
  }
  const int m = (nseg + 31) >> 5;
  const int lo = lane * m;
  const int hi = min(lo + m, nseg);
  float local = 0.f;
  for (int i = lo; i < hi; ++i) local += w.tb(i);
  float incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  total = __shfl_sync(kFull, incl, 31);
  const float target = u * total;
  const unsigned has = __ballot_sync(kFull, lo < nseg);
  const unsigned over = __ballot_sync(kFull, lo < nseg && incl > target);
  const int owner = over ? (__ffs(over) - 1) : (31 - __clz(has));
  int k = nseg - 1;
  if (lane == owner) {
    float cum = incl - local;
    k = hi - 1;
    for (int i = lo; i < hi; ++i) {
      cum += w.tb(i);
      if (cum > target) { k = i; break; }
    }
  }
  return __shfl_sync(kFull, k, owner);
}

// One whole-path tree proposal (tree coordinates: pmc_tree.cuh): the end vertex goes to `end`, every node's
// coordinates step by `step` times its normals; the new path is built level
// by level into nx/ny/nz.  Returns log p(x') + log J(x') - log J(x)
// (-inf if x' has zero density).  Pass 1 (all lanes over all nodes): the old
// coordinates and their Jacobian, the normal steps, and the new coordinates
// parked in nx/ny/nz[m]; pass 2 (level by level): each node reads its new
// coordinates and overwrites them with its new position, whose frame comes
// from the already-built shallower nodes.
template <bool kGen, class WP>
__device__ float tree_propose(const DMedium& M, const DPair& S, float zoff, const WP& w, float* nx, float* ny,
                              float* nz, int n, float3 end, float step, float3 vref, unsigned long long t, int c,
                              uint32_t key0, uint32_t key1, int lane) {
  constexpr unsigned kAll = 0xffffffffu;
  auto opos = [&](int i) { return w.pos(i); };
  auto npos = [&](int i) { return f3(nx[i], ny[i], nz[i]); };
  float lj = 0.f;  // log J(x') - log J(x), lane partials
  for (int m = 1 + lane; m <= n - 2; m += 32) {
    const float3 zc = tree_step_node(opos, m, n, vref, step, t, static_cast<uint32_t>(c), key0, key1, lj);
    nx[m] = zc.x;
    ny[m] = zc.y;
    nz[m] = zc.z;
  }
  if (lane == 0) {
    nx[0] = ny[0] = nz[0] = 0.f;
    nx[n - 1] = end.x;
    ny[n - 1] = end.y;
    nz[n - 1] = end.z;
  }
  __syncwarp();
  for (int d = 0;; ++d) {
    bool any = false;
    for (int j0 = 0; j0 < (1 << d); j0 += 32) {
      const int j = j0 + lane;
      int k = 0, l = 0, kp = -1, lp = -1;
      const bool valid = j < (1 << d) && tree_interval(n, d, j, k, l, kp, lp);
      any = any || __any_sync(kAll, valid);
      if (valid) {
        const int m = (k + l) >> 1;
        const float3 fnew = tree_place_node(npos, k, l, kp, lp, vref, f3(nx[m], ny[m], nz[m]), lj);
        nx[m] = fnew.x;
        ny[m] = fnew.y;
        nz[m] = fnew.z;
      }
    }
    __syncwarp();
    if (!any) break;
  }
  // log p of the new path
  float lp = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float3 Pc = npos(i);
    const float3 Pp = (i >= 1) ? npos(i - 1) : Pc;
    const float3 Pn = (i <= n - 2) ? npos(i + 1) : Pc;
    float vt, gt, seg, tb, len;
    vs_factors<kGen, true>(M, S, zoff, Pp, Pc, Pn, i, n, vt, gt, seg, tb, len);
    lp += vt + ((i <= n - 2) ? seg : 0.f);
  }
  return warp_sum(lp) + warp_sum(lj);
}

// ---------------------------------------------------------------------------
// Full-path HMC (section "Discussion": gradient-based moves).  Every interior
// vertex gets a standard normal momentum; L leapfrog steps of size eps
// follow d log p / d f (the adjoint of the density, grad_vertex) with the
// source and the end vertex fixed; where the path has zero density (a
// non-final segment touching the sensor, the last one arriving from
// behind, or a zero-length segment) the gradient is taken as zero.
// ---------------------------------------------------------------------------
// 1 if the path in (nx, ny, nz) has positive density, on every lane.
__device__ __forceinline__ bool hmc_path_valid(const DPair& S, const float* nx, const float* ny, const float* nz,
                                               int n, int lane) {
  bool ok = true;
  for (int k = lane; k <= n - 2; k += 32) {
    const float3 P = f3(nx[k], ny[k], nz[k]);
    const float3 Q = f3(nx[k + 1], ny[k + 1], nz[k + 1]);
    const float3 r = Q - P;
    if (!(dot(r, r) > 0.f)) ok = false;
    else if (k <= n - 3) ok = ok && !hits_ball<true>(S, P, r);
    else ok = ok && (-dot(r, sensor_normal(S, Q)) > 0.f);
  }
  return __all_sync(0xffffffffu, ok);
}

// p += h * grad log p(x') for the interior vertices (0 where the density is 0).
__device__ __forceinline__ void hmc_kick(const DMedium& M, const DPair& S, float zoff, const float* nx,
                                         const float* ny, const float* nz, float* mx, float* my, float* mz, int n,
                                         float h, int lane) {
  if (!hmc_path_valid(S, nx, ny, nz, n, lane)) return;
  auto npos = [&](int i) { return f3(nx[i], ny[i], nz[i]); };
  for (int i = 1 + lane; i <= n - 2; i += 32) {
    const float3 g = grad_vertex(M, S, zoff, npos, n, i);
    mx[i] = fmaf(h, g.x, mx[i]);
    my[i] = fmaf(h, g.y, my[i]);
    mz[i] = fmaf(h, g.z, mz[i]);
  }
}

// One HMC proposal: returns log p(x') - |p'|^2/2 + |p|^2/2 (without log p(x)),
// the proposed path left in nx/ny/nz.
template <bool kGen, class WP>
__device__ float hmc_propose(const DMedium& M, const DPair& S, float zoff, const WP& w, float* nx, float* ny,
                             float* nz, float* mx, float* my, float* mz, int n, float eps, int L,
                             unsigned long long t, int c, uint32_t key0, uint32_t key1, int lane) {
  float k0 = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float3 P = w.pos(i);
    nx[i] = P.x;
    ny[i] = P.y;
    nz[i] = P.z;
    if (i >= 1 && i <= n - 2) {
      // the oracle's draw: Box-Muller on one Philox block per vertex
      const uint4 rn = philox4x32_10(make_uint4(static_cast<uint32_t>(t), static_cast<uint32_t>(t >> 32),
                                                static_cast<uint32_t>(c), PUR_HMC | (static_cast<uint32_t>(i) << 8)),
                                     key0, key1);
      float s1, c1, s2, c2;
      const float r1 = sqrtf(-2.0f * __logf(u01(rn.x)));
      sincospif(2.0f * u01(rn.y), &s1, &c1);
      const float r2 = sqrtf(-2.0f * __logf(u01(rn.z)));
      sincospif(2.0f * u01(rn.w), &s2, &c2);
      mx[i] = r1 * c1;
      my[i] = r1 * s1;
      mz[i] = r2 * c2;
      k0 += mx[i] * mx[i] + my[i] * my[i] + mz[i] * mz[i];
    }
  }
  __syncwarp();
  hmc_kick(M, S, zoff, nx, ny, nz, mx, my, mz, n, 0.5f * eps, lane);
  for (int st = 1; st <= L; ++st) {
    __syncwarp();
    for (int i = 1 + lane; i <= n - 2; i += 32) {
      nx[i] = fmaf(eps, mx[i], nx[i]);
      ny[i] = fmaf(eps, my[i], ny[i]);
      nz[i] = fmaf(eps, mz[i], nz[i]);
    }
    __syncwarp();
    hmc_kick(M, S, zoff, nx, ny, nz, mx, my, mz, n, st == L ? 0.5f * eps : eps, lane);
  }
  __syncwarp();
  float k1 = 0.f, lp = 0.f;
  for (int i = lane; i < n; i += 32) {
    if (i >= 1 && i <= n - 2) k1 += mx[i] * mx[i] + my[i] * my[i] + mz[i] * mz[i];
    const float3 Pc = f3(nx[i], ny[i], nz[i]);
    const float3 Pp = (i >= 1) ? f3(nx[i - 1], ny[i - 1], nz[i - 1]) : Pc;
    const float3 Pn = (i <= n - 2) ? f3(nx[i + 1], ny[i + 1], nz[i + 1]) : Pc;
    float vt, gt, seg, tb, len;
    vertex_and_segment<kGen>(M, S, zoff, Pp, Pc, Pn, i, n, vt, gt, seg, tb, len);
    lp += vt + ((i <= n - 2) ? seg : 0.f);
  }
  return warp_sum(lp) - 0.5f * (warp_sum(k1) - warp_sum(k0));
}

struct Accum {
  unsigned long long pn2, pn;  // integer partials of the current flush interval
  float pL, pL2, pG;           // FP32 partials of the current flush interval
  unsigned long long t_a;      // step from which the current state is recorded
  unsigned int nflush;
  unsigned int prop_w, prop_end, prop_b, prop_d;  // proposals: within (all), end, birth, death
  unsigned int acc_i, acc_e, acc_b, acc_d;        // acceptances per move kind
  double my;                   // lane-distributed FP64 accumulator word `lane` (lanes 0..15)
};

// The state that became current at step t_a is recorded at every step in
// [t_a, t_b) at or after burn-in, t_b being the step that replaces it; its
// observables enter the sums once, weighted by that count.
__device__ __forceinline__ void close_state(Accum& a, unsigned long long t_b, unsigned long long burn_in, int n,
                                            float L, float G) {
  const unsigned long long from = a.t_a > burn_in ? a.t_a : burn_in;
  a.t_a = t_b;
  if (t_b <= from) return;
  const unsigned long long d = t_b - from;
  const float dw = static_cast<float>(d);
  a.pn2 += (n == 2) ? d : 0ull;
  a.pn += static_cast<unsigned long long>(n) * d;
  a.pL = fmaf(L, dw, a.pL);
  a.pL2 = fmaf(L * L, dw, a.pL2);
  a.pG = fmaf(G, dw, a.pG);
  a.nflush++;
}

__device__ __forceinline__ void flush64(Accum& a, int lane) {
  double v = 0.0;
  if (lane == ACC_NDIRECT) v = static_cast<double>(a.pn2);
  if (lane == ACC_SUMN) v = static_cast<double>(a.pn);
  if (lane == ACC_SUML) v = static_cast<double>(a.pL);
  if (lane == ACC_SUML2) v = static_cast<double>(a.pL2);
  if (lane == ACC_SUMG) v = static_cast<double>(a.pG);
  a.my += v;
  a.pn2 = 0;
  a.pn = 0;
  a.pL = a.pL2 = a.pG = 0.f;
  a.nflush = 0;
}

// Pre-transformed random numbers of one step (8 staged words):
//   lo.x = 23-bit index draw | move type << 24, lo.y = log u (accept),
//   within: lo.z, lo.w, hi.x = standard normals, hi.y = vMF cosine,
//           hi.z, hi.w = cos, sin of the vMF azimuth
//   birth:  lo.z = u for cos s, lo.w = sinh t, hi.x = cosh t, hi.y, hi.z = cos, sin of phi
// Launch bounds: the general tree-move kernel takes up to 128 registers (4
// CTAs of 128 threads per SM), which holds its out-of-line density call
// without spills (+2 % on the two-sensor scene); the general Cartesian
// kernel runs faster at 96 (-1 % at 128 on the layered workload).
template <bool kGen, bool kGrad, bool kSpill, int kX>
__global__ void __launch_bounds__(128, (kGen && kX == 1) ? 4 : ((kGen || kX != 0) ? 5 : 6))
    chain_kernel(const ChainParams P) {
  using WP = WarpPath<kGen, kGrad, kSpill>;
  constexpr bool kTree = kX == 1, kHmc = kX == 2, kLam = kX == 3;
  static_assert(kX == 0 || !kSpill, "tree, HMC and wavelength moves keep the whole cap in shared memory");
  static_assert(kX == 0 || kX == 1 || kGen, "HMC and wavelength moves use the general kernel");
  constexpr int kArraysAll = WP::kArrays + (kTree ? 3 : 0) + (kHmc ? 6 : 0);
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int cap_s = P.smem_cap;
  const size_t per_warp = static_cast<size_t>(kArraysAll) * cap_s + 32 * kRngWords + kPairWords + (kLam ? kMedWords : 0);
  WP w;
  w.sm = smem + static_cast<size_t>(wib) * per_warp;
  w.S = cap_s;
  w.b = P.M.b;
  float* tnx = w.sm + static_cast<size_t>(WP::kArrays) * cap_s;  // tree / HMC moves: the proposed path
  float* tny = tnx + cap_s;
  float* tnz = tny + cap_s;
  float* hmx = tnz + cap_s;                                        // HMC moves: the momenta
  float* hmy = hmx + cap_s;
  float* hmz = hmy + cap_s;
  uint4* rng = reinterpret_cast<uint4*>(w.sm + static_cast<size_t>(kArraysAll) * cap_s);  // [32][2] uint4
  DPair* spair = reinterpret_cast<DPair*>(rng + 64);
  // wavelength sampling: the medium at the chain's current wavelength, in the warp's shared slot
  DMedium* smed = reinterpret_cast<DMedium*>(reinterpret_cast<float*>(spair) + kPairWords);
  const DMedium& M = kLam ? *smed : P.M;
  const DRun& R = P.R;
  const uint32_t key0 = static_cast<uint32_t>(R.seed), key1 = static_cast<uint32_t>(R.seed >> 32);

  for (;;) {
    int item = 0;
    if (lane == 0) item = static_cast<int>(atomicAdd(P.queue, 1u));
    item = __shfl_sync(kFull, item, 0);
    if (P.chain_lo + item >= P.chain_hi) break;
    const int c = P.order[P.chain_lo + item];

    // pair constants, staged in the warp's shared slot
    {
      const int* src = reinterpret_cast<const int*>(P.pairs + P.chain_pair[c]);
      int* dst = reinterpret_cast<int*>(spair);
      for (int q = lane; q < static_cast<int>(sizeof(DPair) / sizeof(int)); q += 32) dst[q] = src[q];
      __syncwarp();
    }
    const DPair& S = *spair;
    const float zoff = S.zoff;
    const int cap = S.cap;
    const int cid = static_cast<int>(static_cast<uint32_t>(c) + P.chain_id0);  // global chain index
    int n = P.n[c];
    const unsigned long long step0 = P.step[c];
    if (n < 2 || n > cap || (!kSpill && cap > cap_s)) {
      if (lane == 0) { P.status[c] |= ST_BAD_N; atomicOr(P.any_status, ST_BAD_N); }
      continue;
    }
    float* gx = P.xyz + P.chain_base[c];
    float* gy = gx + cap;
    float* gz = gy + cap;
    w.gm = gx;
    w.cap = cap;
    float lam = 0.f;
    if constexpr (kLam) {
      lam = P.lam[c];
      if (lane == 0) medium_at(P.M, lam, *smed);
      __syncwarp();
    }
    // the shared window holds entries [0, min(n, S)); the rest stays in the global block
    for (int i = lane; i < min(n, cap_s); i += 32) {
      w.sm[WP::kX * cap_s + i] = gx[i];
      w.sm[WP::kY * cap_s + i] = gy[i];
      w.sm[WP::kZ * cap_s + i] = gz[i];
    }
    __syncwarp();
    const float lp0 = refresh_caches<kGen, kGen && kTree>(M, S, zoff, w, n, lane);
    if (!isfinite(lp0)) {
      if (lane == 0) { P.status[c] |= ST_NONFINITE; atomicOr(P.any_status, ST_NONFINITE); }
      continue;
    }
    Sums sm = path_sums(w, n, lane);
    float L = sm.L, G = sm.G;

    Accum A;
    A.pn2 = A.pn = 0;
    A.pL = A.pL2 = A.pG = 0.f;
    A.t_a = step0;
    A.nflush = 0;
    A.prop_w = A.prop_end = A.prop_b = A.prop_d = 0;
    A.acc_i = A.acc_e = A.acc_b = A.acc_d = 0;
    A.my = (lane < ACC_WORDS) ? P.acc[static_cast<size_t>(c) * ACC_WORDS + lane] : 0.0;

    const float3 cS = f3(S.c[0], S.c[1], S.c[2]);
    float3 vref = f3(1.f, 0.f, 0.f);
    if constexpr (kTree) vref = tree_vref(S);  // the root frame's reference direction
    unsigned long long done = 0;
    bool aborted = false;
    for (unsigned long long s0 = 0; s0 < P.n_steps; s0 += 32) {
      if ((s0 & 1023ull) == 0 && P.abort_flag != nullptr && *P.abort_flag) { aborted = true; break; }
      // ---- lane-parallel random numbers of steps step0+s0 .. +31 ----
      {
        const unsigned long long tl = step0 + s0 + lane;
        const uint4 ra = philox4x32_10(make_uint4(static_cast<uint32_t>(tl), static_cast<uint32_t>(tl >> 32),
                                                  static_cast<uint32_t>(c) + P.chain_id0, PUR_STEP_A), key0, key1);
        const uint4 rb = philox4x32_10(make_uint4(static_cast<uint32_t>(tl), static_cast<uint32_t>(tl >> 32),
                                                  static_cast<uint32_t>(c) + P.chain_id0, PUR_STEP_B), key0, key1);
        const uint32_t um = ra.x >> 9;
        const uint32_t type = um < R.thr_within ? 0u : (um < R.thr_birth ? 2u : 3u);
        uint4 lo = make_uint4((ra.y >> 9) | (type << 24), __float_as_uint(__logf(u01(ra.z))), 0u, 0u);
        uint4 hi;
        const float ub0 = u01(rb.x), ub1 = u01(rb.y), ub2 = u01(rb.z), ub3 = u01(rb.w);
        if (type == 0u) {
          float s1, c1, s2, c2;
          const float r1 = m_sqrt<true>(-2.0f * __logf(ub0));
          sincospif(2.0f * ub1, &s1, &c1);
          const float r2 = m_sqrt<true>(-2.0f * __logf(ub2));
          sincospif(2.0f * ub3, &s2, &c2);
          lo.z = __float_as_uint(r1 * c1);
          lo.w = __float_as_uint(r1 * s1);
          const float wv = 1.0f + __fdividef(__logf(fmaf(1.0f - ub0, S.exp_m2ke, ub0)), S.kappa_end);
          hi = make_uint4(__float_as_uint(r2 * c2), __float_as_uint(wv), __float_as_uint(c1), __float_as_uint(s1));
        } else {
          const float et = __fdividef(ub1, 1.0f - ub1);
          const float iet = __fdividef(1.0f - ub1, ub1);
          float s3, c3;
          sincospif(2.0f * ub2, &s3, &c3);
          lo.z = __float_as_uint(ub0);
          lo.w = __float_as_uint(0.5f * (et - iet));
          hi = make_uint4(__float_as_uint(0.5f * (et + iet)), __float_as_uint(c3), __float_as_uint(s3), 0u);
        }
        __syncwarp();
        rng[2 * lane] = lo;
        rng[2 * lane + 1] = hi;
        __syncwarp();
        // proposals of this batch by kind (within-dimension moves split into
        // interior and end moves at the step)
        const unsigned live = (s0 + lane < P.n_steps) ? 1u : 0u;
        A.prop_w += __popc(__ballot_sync(kFull, live && type == 0u));
        A.prop_b += __popc(__ballot_sync(kFull, live && type == 2u));
        A.prop_d += __popc(__ballot_sync(kFull, live && type == 3u));
      }
      const int cnt = static_cast<int>(min(32ull, P.n_steps - s0));
      for (int i = 0; i < cnt; ++i) {
        const uint4 lo = rng[2 * i];
        const uint4 hi = rng[2 * i + 1];
        const uint32_t mtype = lo.x >> 24;
        const uint32_t v23 = lo.x & 0x7fffffu;
        const float logu = __uint_as_float(lo.y);
        const unsigned long long t = step0 + s0 + i;

        int move;
        bool proposed = true;
        int n_new = n, wlo = 0, nc = 0, olo = 0, onc = 0, jj = -1, kk = -1;
        int inew = -1, sh_from = INT_MAX, sh_by = 0;
        float3 fnew = f3(0.f, 0.f, 0.f);
        float extra = 0.f;
        float3 gx_mala = f3(0.f, 0.f, 0.f);
        if constexpr (kHmc) {
          if (mtype == 0u && 1 + static_cast<int>((static_cast<unsigned long long>(v23) * (n - 1)) >> 23) != n - 1) {
            // full-path HMC over the interior vertices (the end vertex, picked
            // with probability 1/(n-1), takes the usual vMF end move below)
            const float gain = hmc_propose<kGen>(M, S, zoff, w, tnx, tny, tnz, hmx, hmy, hmz, n, R.mala_eps,
                                                 R.hmc_steps, t, cid, key0, key1, lane);
            float lpo = 0.f;
            for (int q = lane; q < n; q += 32) lpo += w.vt(q) + ((q <= n - 2) ? w.seg(q) : 0.f);
            lpo = warp_sum(lpo);
            if (logu < gain - lpo) {
              A.acc_i++;
              close_state(A, t, R.burn_in, n, L, G);
              for (int q = lane; q < n; q += 32) w.set_pos(q, f3(tnx[q], tny[q], tnz[q]));
              __syncwarp();
              refresh_caches<kGen, kGen && kTree>(M, S, zoff, w, n, lane);
              const Sums s3 = path_sums(w, n, lane);
              L = s3.L;
              G = s3.G;
              if (A.nflush >= kFlushAccepts) flush64(A, lane);
            }
            __syncwarp();
            continue;
          }
        }
        if constexpr (kTree) {
          if (mtype == 0u) {
            // whole-path move in tree coordinates; a rejected proposal leaves
            // the path and its caches untouched
            const float3 nu = sensor_normal(S, w.pos(n - 1));
            float3 e1, e2;
            onb(nu, e1, e2);
            const float wv = __uint_as_float(hi.y);
            const float sw = m_sqrt<true>(fmaxf(0.f, 1.0f - wv * wv));
            const float3 nn = wv * nu + sw * (__uint_as_float(hi.z) * e1 + __uint_as_float(hi.w) * e2);
            const float3 end = cS + (f3(S.c_lo[0], S.c_lo[1], S.c_lo[2]) + S.R * nn);
            const float step = R.sigma * rsqrtf(static_cast<float>(n));
            const float gain = tree_propose<kGen>(M, S, zoff, w, tnx, tny, tnz, n, end, step, vref, t, cid, key0, key1,
                                                  lane);
            float lpo = 0.f;
            for (int q = lane; q < n; q += 32) lpo += w.vt(q) + ((q <= n - 2) ? w.seg(q) : 0.f);
            lpo = warp_sum(lpo);
            if (logu < gain - lpo) {
              A.acc_i++;
              close_state(A, t, R.burn_in, n, L, G);
              for (int q = lane; q < n; q += 32) w.set_pos(q, f3(tnx[q], tny[q], tnz[q]));
              __syncwarp();
              refresh_caches<kGen, kGen && kTree>(M, S, zoff, w, n, lane);
              const Sums s3 = path_sums(w, n, lane);
              L = s3.L;
              G = s3.G;
              if (A.nflush >= kFlushAccepts) flush64(A, lane);
            }
            __syncwarp();
            continue;
          }
        }
        if constexpr (kLam) {
          if (mtype == 0u && 1 + static_cast<int>((static_cast<unsigned long long>(v23) * n) >> 23) == n) {
            // wavelength move (the wavelength is the n-th movable coordinate):
            // a Gaussian step with the path held.  Only the coefficients
            // change: log p' - log p = log S(l') - log S(l) - (a' - a + b' - b) L
            // + (n - 2)(log b' - log b), L the path length summed afresh.
            const float lam_y = fmaf(R.sigma_lam, __uint_as_float(lo.z), lam);
            const float lsy = spectrum_log(R, lam_y);
            const Sums sl = path_sums(w, n, lane);
            bool acc_l = false;
            if (isfinite(lsy)) {
              const float r = logf(lam_y / P.M.lam0);
              const float ay = P.M.a * expf(-P.M.ka * r), by = P.M.b * expf(-P.M.ks * r);
              const float lby = P.M.log_b - P.M.ks * r;
              const float dlp = lsy - spectrum_log(R, lam) - ((ay - M.a) + (by - M.b)) * sl.L +
                                static_cast<float>(n - 2) * (lby - M.log_b);
              acc_l = logu < dlp;
            }
            if (acc_l) {
              A.acc_i++;
              close_state(A, t, R.burn_in, n, L, G);
              lam = lam_y;
              __syncwarp();
              if (lane == 0) medium_at(P.M, lam, *smed);
              __syncwarp();
              refresh_caches<kGen, kGen && kTree>(M, S, zoff, w, n, lane);
              if (A.nflush >= kFlushAccepts) flush64(A, lane);
            }
            __syncwarp();
            continue;
          }
        }
        if (!kTree && mtype == 0u) {
          const int j = 1 + static_cast<int>((static_cast<unsigned long long>(v23) * (n - 1 + (kLam ? 1 : 0))) >> 23);
          jj = j;
          inew = j;
          if (j == n - 1) {
            move = MV_END;
            A.prop_end++;
            const float3 nu = sensor_normal(S, w.pos(j));
            float3 e1, e2;
            onb(nu, e1, e2);
            const float wv = __uint_as_float(hi.y);
            const float sw = m_sqrt<true>(fmaxf(0.f, 1.0f - wv * wv));
            const float3 nn = wv * nu + sw * (__uint_as_float(hi.z) * e1 + __uint_as_float(hi.w) * e2);
            fnew = cS + (f3(S.c_lo[0], S.c_lo[1], S.c_lo[2]) + S.R * nn);
            wlo = n - 2; nc = 2; olo = n - 2; onc = 2;
          } else {
            move = MV_INTERIOR;
            const float3 fj = w.pos(j);
            const float3 z = f3(__uint_as_float(lo.z), __uint_as_float(lo.w), __uint_as_float(hi.x));
            if constexpr (kGen && kX == 0) {
              if (R.within == 1) {
                gx_mala = grad_vertex_warp(M, S, zoff, [&](int k) { return w.pos(k); }, n, j, lane);
                const float h = 0.5f * R.mala_eps * R.mala_eps;
                fnew = fj + h * gx_mala + R.mala_eps * z;
              } else {
                fnew = fj + R.sigma * z;
              }
            } else {
              fnew = fj + R.sigma * z;
            }
            wlo = j - 1; nc = 3; olo = j - 1; onc = 3;
          }
        } else if (mtype == 2u) {
          move = MV_BIRTH;
          if (n >= cap) {
            proposed = false;
          } else {
            float total;
            const float ui = __fmaf_rn(static_cast<float>(v23), 1.1920928955078125e-7f, 5.9604644775390625e-8f);
            const int k = select_segment(w, n - 1, ui, total, lane);
            kk = k;
            const float3 Af = w.pos(k), Bf = w.pos(k + 1);
            const float3 r = Bf - Af;
            const float rr = dot(r, r);
            const float irl = rsqrtf(rr);
            const float gamma = 0.5f * rr * irl;
            const float3 rh = irl * r;
            float3 xi, ze;
            onb(rh, xi, ze);
            const float beta = insertion_beta(M, R, zoff, Af, Bf, gamma);
            const float u0 = __uint_as_float(lo.z);
            float cs = -1.0f - __fdividef(__logf(fmaf(-u0, 1.0f - __expf(-2.0f * beta), 1.0f)), beta);
            cs = fminf(fmaxf(cs, -1.0f), 1.0f);
            const float sn = m_sqrt<true>(fmaxf(0.f, (1.0f - cs) * (1.0f + cs)));
            const float sc = __fdividef(gamma, __uint_as_float(hi.x) - cs);
            fnew = 0.5f * (Af + Bf) +
                   sc * (__uint_as_float(lo.w) * rh + sn * (__uint_as_float(hi.y) * xi + __uint_as_float(hi.z) * ze));
            const float tbk = w.tb(k);
            extra = R.log_pd - __logf(static_cast<float>(n - 1)) - R.log_pb - __logf(__fdividef(tbk, total)) -
                    log_insert_density<true>(M, R, zoff, Af, Bf, fnew);
            n_new = n + 1;
            inew = k + 1;
            sh_from = k + 2;
            sh_by = -1;
            wlo = k; nc = 3; olo = k; onc = 2;
          }
        } else {
          move = MV_DEATH;
          if (n <= 2) {
            proposed = false;
          } else {
            const int j = 1 + static_cast<int>((static_cast<unsigned long long>(v23) * (n - 2)) >> 23);
            jj = j;
            n_new = n - 1;
            sh_from = j;
            sh_by = 1;
            wlo = j - 1; nc = 2; olo = j - 1; onc = 3;
          }
        }

        bool accept = false;
        float nvt = 0.f, ngt = 0.f, nseg = 0.f, ntb = 0.f, nlen = 0.f;
        float ogt = 0.f, olen = 0.f;
        if (proposed) {
          // new-path vertex index -> position (old index shifted, or the new vertex)
          auto newpos = [&](int idx) -> float3 {
            int o = idx + ((idx >= sh_from) ? sh_by : 0);
            o = min(max(o, 0), n - 1);
            const float3 q = w.pos(o);
            return (idx == inew) ? fnew : q;
          };
          float ovt = 0.f, oseg = 0.f, otb = 0.f;
          if (lane < nc) {
            const int v = wlo + lane;
            const float3 Pc = newpos(v);
            const float3 Pp = newpos(v - 1);
            const float3 Pn = newpos(v + 1);
            float seg_, tb_, len_;
            vs_factors<kGen, kGen && kTree>(M, S, zoff, Pp, Pc, Pn, v, n_new, nvt, ngt, seg_, tb_, len_);
            if (lane < nc - 1) {
              nseg = seg_;
              ntb = tb_;
              nlen = len_;
            }
          }
          if (lane < onc) {
            const int o = olo + lane;
            ovt = w.vt(o);
            ogt = w.gt(o);
            if (lane < onc - 1) {
              oseg = w.seg(o);
              otb = w.tb(o);
              olen = w.len(o);
            }
          }
          float dlp = (nvt + nseg) - (ovt + oseg);
          dlp += __shfl_xor_sync(kFull, dlp, 1);
          dlp += __shfl_xor_sync(kFull, dlp, 2);
          dlp = __shfl_sync(kFull, dlp, 0);
          if (move == MV_DEATH) {
            float dtb = ntb - otb;
            dtb += __shfl_xor_sync(kFull, dtb, 1);
            dtb += __shfl_xor_sync(kFull, dtb, 2);
            dtb = __shfl_sync(kFull, dtb, 0);
            // T_b of the reduced path, summed afresh so that decisions depend
            // only on the current state (split runs replay exactly)
            float part = 0.f;
            for (int q = lane; q < n - 1; q += 32) part += w.tb(q);
            const float tb_new = __shfl_sync(kFull, ntb, 0);
            const float Tb_red = warp_sum(part) + dtb;
            extra = -R.log_pd + __logf(static_cast<float>(n - 2)) + R.log_pb + __logf(__fdividef(tb_new, Tb_red)) +
                    log_insert_density<true>(M, R, zoff, w.pos(jj - 1), w.pos(jj + 1), w.pos(jj));
          }
          if constexpr (kGen && kX == 0) {
            if (move == MV_INTERIOR && R.within == 1 && isfinite(dlp)) {
              const float3 gy = grad_vertex_warp(M, S, zoff, newpos, n, jj, lane);
              const float h = 0.5f * R.mala_eps * R.mala_eps;
              const float3 fj = w.pos(jj);
              const float3 dfw = fnew - fj - h * gx_mala;
              const float3 dbw = fj - fnew - h * gy;
              extra = (dot(dfw, dfw) - dot(dbw, dbw)) / (2.0f * R.mala_eps * R.mala_eps);
            }
          }
          accept = logu < dlp + extra;
        }
        if (accept) {
          A.acc_i += (move == MV_INTERIOR);
          A.acc_e += (move == MV_END);
          A.acc_b += (move == MV_BIRTH);
          A.acc_d += (move == MV_DEATH);
          close_state(A, t, R.burn_in, n, L, G);
          float dlen = nlen - olen;
          dlen += __shfl_xor_sync(kFull, dlen, 1);
          dlen += __shfl_xor_sync(kFull, dlen, 2);
          dlen = __shfl_sync(kFull, dlen, 0);
          float dg = 0.f;
          if constexpr (kGrad) {
            dg = ngt - ogt;
            dg += __shfl_xor_sync(kFull, dg, 1);
            dg += __shfl_xor_sync(kFull, dg, 2);
            dg = __shfl_sync(kFull, dg, 0);
          }
          if (move == MV_BIRTH) {
            shift_right(w, kk + 1, n, n - 1, lane);
          } else if (move == MV_DEATH) {
            shift_left(w, jj + 1, n, n - 1, lane);
          }
          if (lane < nc) {
            const int v = wlo + lane;
            w.set_vt(v, nvt);
            w.set_gt(v, ngt);
            if (lane < nc - 1) {
              w.set_seg(v, nseg);
              w.set_tb(v, ntb);
              w.set_len(v, nlen);
            }
          }
          if (lane == 0 && move != MV_DEATH) w.set_pos(inew, fnew);
          __syncwarp();
          n = n_new;
          L += dlen;
          G += dg;
          if (A.nflush >= kFlushAccepts) flush64(A, lane);
        }
      }
      done += cnt;
      if (((s0 + 32) & (kRefreshSteps - 1)) == 0) {
        const Sums s2 = path_sums(w, n, lane);
        L = s2.L;
        G = s2.G;
      }
    }
    close_state(A, step0 + done, R.burn_in, n, L, G);
    flush64(A, lane);
    // recorded states, proposal and acceptance counts
    const unsigned long long t_end = step0 + done;
    const unsigned long long first = step0 > R.burn_in ? step0 : R.burn_in;
    const double nrec = t_end > first ? static_cast<double>(t_end - first) : 0.0;
    double extra_w = 0.0;
    if (lane == ACC_NREC) extra_w = nrec;
    if (lane == ACC_PROP + 0) extra_w = static_cast<double>(A.prop_w - A.prop_end);
    if (lane == ACC_PROP + 1) extra_w = static_cast<double>(A.prop_end);
    if (lane == ACC_PROP + 2) extra_w = static_cast<double>(A.prop_b);
    if (lane == ACC_PROP + 3) extra_w = static_cast<double>(A.prop_d);
    if (lane == ACC_ACC + 0) extra_w = static_cast<double>(A.acc_i);
    if (lane == ACC_ACC + 1) extra_w = static_cast<double>(A.acc_e);
    if (lane == ACC_ACC + 2) extra_w = static_cast<double>(A.acc_b);
    if (lane == ACC_ACC + 3) extra_w = static_cast<double>(A.acc_d);
    A.my += extra_w;
    if (lane < ACC_WORDS) P.acc[static_cast<size_t>(c) * ACC_WORDS + lane] = A.my;
    for (int i = lane; i < min(n, cap_s); i += 32) {
      gx[i] = w.sm[WP::kX * cap_s + i];
      gy[i] = w.sm[WP::kY * cap_s + i];
      gz[i] = w.sm[WP::kZ * cap_s + i];
    }
    if (lane == 0) {
      P.n[c] = n;
      P.step[c] = t_end;
      if constexpr (kLam) P.lam[c] = lam;
      if (aborted) { P.status[c] |= ST_ABORTED; atomicOr(P.any_status, ST_ABORTED); }
    }
    __syncwarp();
  }
}

// Initial paths (one thread per chain), and initial wavelengths from the
// spectrum's quantile of u01 of Philox counter (0, 1, chain, init).
__global__ void init_kernel(const InitParams p) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.total) return;
  if (p.lam != nullptr) {
    const uint4 r = philox4x32_10(make_uint4(0u, 1u, static_cast<uint32_t>(c) + p.chain_id0, PUR_INIT),
                                  static_cast<uint32_t>(p.R.seed), static_cast<uint32_t>(p.R.seed >> 32));
    p.lam[c] = spectrum_quantile(p.R, u01(r.x));
  }
  const DPair S = p.pairs[p.chain_pair[c]];
  float* gx = p.xyz + p.chain_base[c];
  float* gy = gx + S.cap;
  float* gz = gy + S.cap;
  int n;
  if (p.init_kind == PMC_INIT_USER) {
    n = p.user_n[c];
    const size_t st = static_cast<size_t>(p.user_stride);
    const float* ux = p.user_xyz + static_cast<size_t>(c) * 3 * st;
    if (n < 2 || n > S.cap || n > p.user_stride) {
      p.status[c] = ST_BAD_N;
      n = 2;
    }
    for (int i = 0; i < n; ++i) {
      gx[i] = ux[i] - S.org[0];
      gy[i] = ux[st + i] - S.org[1];
      gz[i] = ux[2 * st + i] - S.org[2];
    }
  } else {
    const int k = (p.init_kind == PMC_INIT_DIRECT) ? 0 : p.init_k;
    n = k + 2;
    if (n > S.cap) {
      p.status[c] = ST_BAD_N;
      n = 2;
    }
    const uint32_t k0 = static_cast<uint32_t>(p.R.seed), k1 = static_cast<uint32_t>(p.R.seed >> 32);
    gx[0] = gy[0] = gz[0] = 0.f;
    const int kk = n - 2;
    for (int i = 1; i <= kk; ++i) {
      const float fr = static_cast<float>(i) / static_cast<float>(kk + 1);
      const uint4 r = philox4x32_10(make_uint4(static_cast<uint32_t>(i), 0u, static_cast<uint32_t>(c) + p.chain_id0, PUR_INIT),
                                    k0, k1);
      float s1, c1, s2, c2;
      const float r1 = sqrtf(-2.0f * logf(u01(r.x)));
      sincospif(2.0f * u01(r.y), &s1, &c1);
      const float r2 = sqrtf(-2.0f * logf(u01(r.z)));
      sincospif(2.0f * u01(r.w), &s2, &c2);
      gx[i] = fr * S.e_near[0] + p.jitter * r1 * c1;
      gy[i] = fr * S.e_near[1] + p.jitter * r1 * s1;
      gz[i] = fr * S.e_near[2] + p.jitter * r2 * c2;
    }
    gx[kk + 1] = S.e_near[0];
    gy[kk + 1] = S.e_near[1];
    gz[kk + 1] = S.e_near[2];
  }
  p.n[c] = n;
  p.step[c] = 0ull;
  for (int k = 0; k < ACC_WORDS; ++k) p.acc[static_cast<size_t>(c) * ACC_WORDS + k] = 0.0;
}

// The dynamic shared-memory limit is a property of the kernel, shared by every
// launch: set it once to the device's per-block maximum so that classes with
// different vertex caps can all launch.
template <bool kGen, bool kGrad, bool kSpill, int kX>
cudaError_t set_attributes() {
  static int done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(chain_kernel<kGen, kGrad, kSpill, kX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(chain_kernel<kGen, kGrad, kSpill, kX>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           100);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = 1;
  return e;
}

template <bool kGen, bool kGrad, bool kSpill, int kX>
cudaError_t occupancy_of(int warps_per_block, size_t sm, int* blocks_per_sm) {
  cudaError_t e = set_attributes<kGen, kGrad, kSpill, kX>();
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, chain_kernel<kGen, kGrad, kSpill, kX>,
                                                       warps_per_block * 32, sm);
}

template <bool kGen, bool kGrad, bool kSpill, int kX>
void launch_one(const ChainParams& p, int grid, int warps_per_block, size_t sm, cudaStream_t s) {
  chain_kernel<kGen, kGrad, kSpill, kX><<<grid, warps_per_block * 32, sm, s>>>(p);
}

// Instantiation key: lean / general (with or without gradient caches and
// spill), general with tree moves and general with HMC moves (never spilled).
int kernel_key(int kind, bool grad, bool spill) {
  if (kind == 2) return 8 + (grad ? 1 : 0);
  if (kind == 3) return 10 + (grad ? 1 : 0);
  if (kind == 6) return 12;
  if (kind == 7) return 14 + (grad ? 1 : 0);
  return (kind == 1 ? 4 : 0) + (grad ? 2 : 0) + (spill ? 1 : 0);
}

}  // namespace

int chain_arrays(bool general, bool grad) { return 6 + (general ? 1 : 0) + (grad ? 1 : 0); }

size_t chain_smem_bytes(int smem_cap, int warps_per_block, int kind, bool grad) {
  if (lane_kind(kind)) return lane_smem_bytes(smem_cap, warps_per_block, grad, kind == 8);
  const size_t arrays = static_cast<size_t>(chain_arrays(kind > 0 && kind != 7, grad) + (kind == 2 || kind == 7 ? 3 : 0) +
                                            (kind == 3 ? 6 : 0));
  return static_cast<size_t>(warps_per_block) *
         (arrays * static_cast<size_t>(smem_cap) + 32u * kRngWords + kPairWords + (kind == 6 ? kMedWords : 0)) *
         sizeof(float);
}

cudaError_t chain_occupancy(int kind, bool grad, bool spill, int warps_per_block, int smem_cap,
                            int* blocks_per_sm) {
  if (lane_kind(kind)) return lane_occupancy(kind, warps_per_block, smem_cap, grad, blocks_per_sm);
  if (kind >= 2 && spill) return cudaErrorInvalidValue;
  if (kind == 6 && grad) return cudaErrorInvalidValue;
  const size_t sm = chain_smem_bytes(smem_cap, warps_per_block, kind, grad);
  switch (kernel_key(kind, grad, spill)) {
    case 0: return occupancy_of<false, false, false, 0>(warps_per_block, sm, blocks_per_sm);
    case 1: return occupancy_of<false, false, true, 0>(warps_per_block, sm, blocks_per_sm);
    case 2: return occupancy_of<false, true, false, 0>(warps_per_block, sm, blocks_per_sm);
    case 3: return occupancy_of<false, true, true, 0>(warps_per_block, sm, blocks_per_sm);
    case 4: return occupancy_of<true, false, false, 0>(warps_per_block, sm, blocks_per_sm);
    case 5: return occupancy_of<true, false, true, 0>(warps_per_block, sm, blocks_per_sm);
    case 6: return occupancy_of<true, true, false, 0>(warps_per_block, sm, blocks_per_sm);
    case 7: return occupancy_of<true, true, true, 0>(warps_per_block, sm, blocks_per_sm);
    case 8: return occupancy_of<true, false, false, 1>(warps_per_block, sm, blocks_per_sm);
    case 9: return occupancy_of<true, true, false, 1>(warps_per_block, sm, blocks_per_sm);
    case 10: return occupancy_of<true, false, false, 2>(warps_per_block, sm, blocks_per_sm);
    case 12: return occupancy_of<true, false, false, 3>(warps_per_block, sm, blocks_per_sm);
    case 14: return occupancy_of<false, false, false, 1>(warps_per_block, sm, blocks_per_sm);
    case 15: return occupancy_of<false, true, false, 1>(warps_per_block, sm, blocks_per_sm);
    default: return occupancy_of<true, true, false, 2>(warps_per_block, sm, blocks_per_sm);
  }
}

cudaError_t launch_chain(const ChainParams& p, int kind, bool grad, bool spill, int grid, int warps_per_block,
                         cudaStream_t s) {
  if (lane_kind(kind)) return launch_lane_chain(p, kind, grid, warps_per_block, grad, s);
  if (kind >= 2 && spill) return cudaErrorInvalidValue;
  if (kind == 6 && grad) return cudaErrorInvalidValue;
  const size_t sm = chain_smem_bytes(p.smem_cap, warps_per_block, kind, grad);
  switch (kernel_key(kind, grad, spill)) {
    case 0: launch_one<false, false, false, 0>(p, grid, warps_per_block, sm, s); break;
    case 1: launch_one<false, false, true, 0>(p, grid, warps_per_block, sm, s); break;
    case 2: launch_one<false, true, false, 0>(p, grid, warps_per_block, sm, s); break;
    case 3: launch_one<false, true, true, 0>(p, grid, warps_per_block, sm, s); break;
    case 4: launch_one<true, false, false, 0>(p, grid, warps_per_block, sm, s); break;
    case 5: launch_one<true, false, true, 0>(p, grid, warps_per_block, sm, s); break;
    case 6: launch_one<true, true, false, 0>(p, grid, warps_per_block, sm, s); break;
    case 7: launch_one<true, true, true, 0>(p, grid, warps_per_block, sm, s); break;
    case 8: launch_one<true, false, false, 1>(p, grid, warps_per_block, sm, s); break;
    case 9: launch_one<true, true, false, 1>(p, grid, warps_per_block, sm, s); break;
    case 10: launch_one<true, false, false, 2>(p, grid, warps_per_block, sm, s); break;
    case 12: launch_one<true, false, false, 3>(p, grid, warps_per_block, sm, s); break;
    case 14: launch_one<false, false, false, 1>(p, grid, warps_per_block, sm, s); break;
    case 15: launch_one<false, true, false, 1>(p, grid, warps_per_block, sm, s); break;
    default: launch_one<true, true, false, 2>(p, grid, warps_per_block, sm, s); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_init(const InitParams& p, cudaStream_t s) {
  if (p.total == 0) return cudaSuccess;
  init_kernel<<<(p.total + 127) / 128, 128, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pmc
