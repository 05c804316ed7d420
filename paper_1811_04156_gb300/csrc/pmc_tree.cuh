// Tree coordinates of a path (Collin, arXiv:1811.04156: section "Path
// proposal distribution"; appendix "Path space coordinate system") and the
// per-node steps of the whole-path tree move, shared by the warp-per-chain
// kernel (nodes spread over the lanes) and the lane-per-chain kernel (nodes in
// sequence on one lane), so that there is one copy of the map.
//
// Interior vertex m = (k + l)/2 sits in the bispherical system of its foci
// f_k, f_l (root: f_0, f_{n-1}) with coordinates zeta = atanh(cos s),
// t = ln(d1/d2) and the azimuth phi about e = (f_l - f_k)/|f_l - f_k| in the
// frame (xi, eta): eta is the unit normal e_p x (f_p - mid_p) of the parent's
// triangle (the parent's axes turned by its phi), xi = eta x e; the root's xi
// is vref projected normal to e.  The volume element is
// (d1 d2 / (2 gamma))^3 sin^2 s per node.
//
// Transcendentals use the SFU forms (a few ulp): the map only has to be the
// same deterministic bijection in both directions up to rounding, far below
// the Monte-Carlo error, as for the density in the chain kernels.
#pragma once

#include "pmc_internal.h"

namespace pmc {

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Interval (k, l) of node j at depth d (binary descent on the bits of j, most
// significant first) and its parent's interval (kp = -1 at the root); false
// when the interval holds no vertex.
__device__ __forceinline__ bool tree_interval(int n, int d, int j, int& k, int& l, int& kp, int& lp) {
  k = 0;
  l = n - 1;
  kp = lp = -1;
  for (int b = d - 1; b >= 0; --b) {
    if (l - k < 2) return false;
    const int mid = (k + l) >> 1;
    kp = k;
    lp = l;
    if ((j >> b) & 1) k = mid;
    else l = mid;
  }
  return l - k >= 2;
}

// Foci (k, l) of interior vertex m and its parent's foci (kp = -1 at the root).
__device__ __forceinline__ void tree_node_of(int m, int n, int& k, int& l, int& kp, int& lp) {
  k = 0;
  l = n - 1;
  kp = lp = -1;
  for (;;) {
    const int mid = (k + l) >> 1;
    if (mid == m) return;
    kp = k;
    lp = l;
    if (m < mid) l = mid;
    else k = mid;
  }
}

struct TreeFrame {
  float3 e, xi, eta, mid;
  float gamma;
};

template <class PosF>
__device__ __forceinline__ TreeFrame tree_frame(PosF pos, int k, int l, int kp, int lp, float3 vref) {
  TreeFrame F;
  const float3 A = pos(k), B = pos(l);
  const float3 r = B - A;
  const float rr = dot(r, r);
  const float ir = rsqrtf(rr);
  F.e = ir * r;
  F.gamma = 0.5f * rr * ir;
  F.mid = 0.5f * (A + B);
  bool have = false;
  if (kp >= 0) {
    const int p = (kp + lp) >> 1;
    const float3 Ap = pos(kp), Bp = pos(lp);
    const float3 ep = Bp - Ap, rho = pos(p) - 0.5f * (Ap + Bp);
    float3 nrm = cross3(ep, rho);
    const float nn2 = dot(nrm, nrm);
    if (nn2 > 1e-12f * dot(ep, ep) * dot(rho, rho) && nn2 > 0.f) {
      nrm = nrm - dot(nrm, F.e) * F.e;
      F.eta = rsqrtf(dot(nrm, nrm)) * nrm;
      F.xi = cross3(F.eta, F.e);
      have = true;
    }
  }
  if (!have) {
    const float3 x = vref - dot(vref, F.e) * F.e;
    F.xi = rsqrtf(dot(x, x)) * x;
    F.eta = cross3(F.e, F.xi);
  }
  return F;
}

// Root frame reference of a pair: the first vector of the orthonormal
// completion of the unit direction from the source (frame origin) to the
// sensor centre.
__device__ __forceinline__ float3 tree_vref(const DPair& S) {
  const float3 cc = f3(S.c[0], S.c[1], S.c[2]) + f3(S.c_lo[0], S.c_lo[1], S.c_lo[2]);
  float3 vref, e2;
  onb(rsqrtf(dot(cc, cc)) * cc, vref, e2);
  return vref;
}

// First half of the move for interior node m of the current path (opos):
// its tree coordinates (zeta, t, phi), each stepped by `step` times a
// standard normal drawn from the node's Philox block (Box-Muller on one
// block: counter (step t, global chain index, PUR_TREE | m << 8)).  Returns
// the stepped coordinates; lj gains -log of the node's volume element at the
// current path.
template <class PosF>
__device__ __forceinline__ float3 tree_step_node(PosF opos, int m, int n, float3 vref, float step,
                                                 unsigned long long t, uint32_t cid, uint32_t key0, uint32_t key1,
                                                 float& lj) {
  int k, l, kp, lp;
  tree_node_of(m, n, k, l, kp, lp);
  const TreeFrame Fo = tree_frame(opos, k, l, kp, lp, vref);
  const float3 P = opos(m);
  const float3 a = opos(k) - P, b = opos(l) - P;
  const float d1 = sqrtf(dot(a, a)), d2 = sqrtf(dot(b, b));
  const float3 u = (1.0f / d1) * a, v = (1.0f / d2) * b;
  const float3 up = u + v, um = u - v;
  const float opc = 0.5f * dot(up, up), omc = 0.5f * dot(um, um);
  const float3 rho = P - Fo.mid;
  lj -= 3.0f * __logf(d1 * d2 / (2.0f * Fo.gamma)) + __logf(opc * omc);
  const uint4 rn = philox4x32_10(make_uint4(static_cast<uint32_t>(t), static_cast<uint32_t>(t >> 32), cid,
                                            PUR_TREE | (static_cast<uint32_t>(m) << 8)),
                                 key0, key1);
  float s1, c1, s2, c2;
  const float r1 = sqrtf(-2.0f * __logf(u01(rn.x)));
  sincospif(2.0f * u01(rn.y), &s1, &c1);
  const float r2 = sqrtf(-2.0f * __logf(u01(rn.z)));
  sincospif(2.0f * u01(rn.w), &s2, &c2);
  return f3(fmaf(step, r1 * c1, 0.5f * __logf(__fdividef(opc, omc))), fmaf(step, r1 * s1, __logf(__fdividef(d1, d2))),
            fmaf(step, r2 * c2, atan2f(dot(rho, Fo.eta), dot(rho, Fo.xi))));
}

// Second half for the node of interval (k, l) with parent interval (kp, lp):
// its new position from the coordinates zc = (zeta, t, phi) in the frame of
// the new path (npos; the foci and the parent's triangle are shallower nodes,
// already placed).  lj gains log of the node's volume element at the new path.
template <class PosF>
__device__ __forceinline__ float3 tree_place_node(PosF npos, int k, int l, int kp, int lp, float3 vref, float3 zc,
                                                  float& lj) {
  const TreeFrame Fn = tree_frame(npos, k, l, kp, lp, vref);
  const float ez = __expf(zc.x), emz = __expf(-zc.x);
  const float sn = 2.0f / (ez + emz);                 // 1 / cosh zeta = sin s
  const float omcs = 2.0f / (1.0f + ez * ez);          // 1 - tanh zeta
  const float eh = __expf(0.5f * zc.y), ieh = __expf(-0.5f * zc.y);
  const float sh = 0.5f * (eh - ieh);                 // sinh(t/2)
  const float den = fmaf(2.0f * sh, sh, omcs);        // cosh t - cos s
  float sp, cp;
  __sincosf(zc.z, &sp, &cp);
  const float sc = Fn.gamma / den;
  const float sht = 2.0f * sh * (0.5f * (eh + ieh));    // sinh t = 2 sinh(t/2) cosh(t/2)
  lj += 3.0f * __logf(sc) + 2.0f * __logf(sn);
  return Fn.mid + sc * (sht * Fn.e + sn * (cp * Fn.xi + sp * Fn.eta));
}

}  // namespace pmc
