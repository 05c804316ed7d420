// Normalised reference density q_ref and the geometric bridge estimator
// (Collin, arXiv:1811.04156: section "Comparison of relative light yield" for
// the estimator E_0[sqrt(p_1/p_0)] / E_1[sqrt(p_0/p_1)], here with p_0 := q_ref;
// appendix "Path space coordinate system" for the recursive tree of
// bispherical coordinates; appendix "Dimension matching transformation" for
// q(s), q(t), q(phi) and beta).
//
// q_ref(path) = P_ref(n) * q_end(f_{n-1}) * prod over interior vertices m of
//   q(s_m) q(t_m) q(phi_m) / J_m,
// where vertex m = floor((k + l)/2) sits in the bispherical system with foci
// f_k, f_l of its tree node (root: f_0, f_{n-1}); P_ref is a Poisson law in the
// straight-line scattering depth truncated to n - 2 in [0, cap - 2], and q_end
// is uniform over the part of the sensor visible from the source.
//
// Kernels: one warp per reference draw (sampled level by level down the tree
// in shared memory, then log p and log q_ref), one warp per chain state
// (log q_ref and log p of the current path), one warp per caller path.
#include <algorithm>

#include "pmc_internal.h"

namespace pmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Foci (k, l) of interior vertex m in the tree over [0, n-1], and its depth.
__device__ __forceinline__ int tree_node(int m, int n, int& k, int& l) {
  k = 0;
  l = n - 1;
  int depth = 0;
  for (;;) {
    const int mid = (k + l) >> 1;
    if (mid == m) return depth;
    if (m < mid) l = mid;
    else k = mid;
    ++depth;
  }
}

// log p and log q_ref of a path given by a position accessor (accurate math).
template <class PosF>
__device__ void path_logs(const DMedium& M, const DRun& R, const DPair& S, const QrefPair& Q, const double* qtab,
                          float zoff, PosF pos, int n, int lane, float& lp, float& lq) {
  float a = 0.f, b = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float3 P = pos(i);
    const float3 Pp = (i >= 1) ? pos(i - 1) : P;
    const float3 Pn = (i <= n - 2) ? pos(i + 1) : P;
    float g;
    a += vertex_term(M, S, zoff, Pp, P, Pn, i, n, g);
    if (i <= n - 2) a += segment_term(M, S, zoff, P, Pn, i <= n - 3).seg;
    if (i >= 1 && i <= n - 2) {
      int k, l;
      tree_node(i, n, k, l);
      b += log_insert_density<false>(M, R, zoff, pos(k), pos(l), P);
    }
  }
  lp = warp_sum_f(a);
  lq = warp_sum_f(b);
  // vertex count and end vertex
  const float3 e = pos(n - 1);
  const float3 nu = sensor_normal(S, e);
  const float3 u = f3(S.src[0] - S.c[0], S.src[1] - S.c[1], S.src[2] - S.c[2]);  // centre -> source
  const float D = sqrtf(dot(u, u));
  const bool visible = dot(nu, (1.0f / D) * u) > S.R / D;
  lq += static_cast<float>(qtab[Q.off + n] + Q.log_qend);
  if (!visible) lq = kNegInf;
}

}  // namespace

// Reference draws: each warp samples one path from q_ref and adds
// sqrt(p/q_ref) and p/q_ref to the pair's FP64 sums.
__global__ void __launch_bounds__(128) qref_draw_kernel(const DMedium M, const DRun R, const DPair* __restrict__ pairs,
                                                        const QrefPair* __restrict__ qp,
                                                        const double* __restrict__ qtab, int smem_cap, int stream_base,
                                                        unsigned long long seed, unsigned long long draw0,
                                                        unsigned long long n_draws, double* __restrict__ sums,
                                                        float* __restrict__ out_xyz, int* __restrict__ out_n,
                                                        int out_stride, float* __restrict__ out_logr) {
  extern __shared__ float smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* sx = smem + static_cast<size_t>(wib) * 3 * smem_cap;
  float* sy = sx + smem_cap;
  float* sz = sy + smem_cap;
  const int pair = blockIdx.y;
  const DPair S = pairs[pair];
  const QrefPair& Q = qp[pair];
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  const uint32_t purpose = PUR_QREF | (static_cast<uint32_t>(stream_base + pair) << 8);
  double acc_s = 0.0, acc_r = 0.0, acc_r2 = 0.0;
  const unsigned long long wstride = static_cast<unsigned long long>(gridDim.x) * (blockDim.x >> 5);
  for (unsigned long long q = blockIdx.x * (blockDim.x >> 5) + wib; q < n_draws; q += wstride) {
    const unsigned long long draw = draw0 + q;
    const uint4 r0 = philox4x32_10(make_uint4(static_cast<uint32_t>(draw), static_cast<uint32_t>(draw >> 32), 0u,
                                              purpose), k0, k1);
    // vertex count by inverse CDF (FP64 table)
    const double un = static_cast<double>(r0.x >> 9) * (1.0 / 8388608.0) + 0.5 / 8388608.0;
    int n = S.cap;
    for (int base = 2; base <= S.cap; base += 32) {
      const int nn = base + lane;
      const bool hit = nn <= S.cap && qtab[Q.off + S.cap + 1 + nn] > un;
      const unsigned bal = __ballot_sync(kFull, hit);
      if (bal) {
        n = base + __ffs(bal) - 1;
        break;
      }
    }
    // end vertex uniform on the visible cap
    if (lane == 0) {
      const float3 cc = f3(S.c[0], S.c[1], S.c[2]);
      const float D = sqrtf(dot(cc, cc));
      const float3 u = (-1.0f / D) * cc;
      float3 e1, e2;
      onb(u, e1, e2);
      const float wv = S.R / D + (1.0f - S.R / D) * u01(r0.y);
      float sp, cp;
      sincospif(2.0f * u01(r0.z), &sp, &cp);
      const float sw = sqrtf(fmaxf(0.f, 1.0f - wv * wv));
      const float3 nu = wv * u + sw * (cp * e1 + sp * e2);
      const float3 e = cc + (f3(S.c_lo[0], S.c_lo[1], S.c_lo[2]) + S.R * nu);
      sx[0] = sy[0] = sz[0] = 0.f;
      sx[n - 1] = e.x;
      sy[n - 1] = e.y;
      sz[n - 1] = e.z;
    }
    __syncwarp();
    // interior vertices level by level down the tree
    int maxdepth = 0;
    for (int m = 1 + lane; m <= n - 2; m += 32) {
      int kk, ll;
      maxdepth = max(maxdepth, tree_node(m, n, kk, ll));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxdepth = max(maxdepth, __shfl_xor_sync(kFull, maxdepth, o));
    for (int d = 0; d <= maxdepth && n > 2; ++d) {
      for (int m = 1 + lane; m <= n - 2; m += 32) {
        int kk, ll;
        if (tree_node(m, n, kk, ll) != d) continue;
        const uint4 rr = philox4x32_10(make_uint4(static_cast<uint32_t>(draw), static_cast<uint32_t>(draw >> 32),
                                                  static_cast<uint32_t>(m), purpose), k0, k1);
        const float3 A = f3(sx[kk], sy[kk], sz[kk]), B = f3(sx[ll], sy[ll], sz[ll]);
        const float3 ab = B - A;
        const float ell = sqrtf(dot(ab, ab));
        const float gamma = 0.5f * ell;
        const float3 eh = (1.0f / ell) * ab;
        float3 xi, ze;
        onb(eh, xi, ze);
        const float beta = insertion_beta(M, R, S.zoff, A, B, gamma);
        const float ub = u01(rr.x);
        float cs = -1.0f - log1pf(ub * expm1f(-2.0f * beta)) / beta;
        cs = fminf(fmaxf(cs, -1.0f), 1.0f);
        const float ut = u01(rr.y);
        const float t = logf(ut / (1.0f - ut));
        float sp, cp;
        sincospif(2.0f * u01(rr.z), &sp, &cp);
        const float sn = sqrtf(fmaxf(0.f, (1.0f - cs) * (1.0f + cs)));
        const float sc = gamma / (coshf(t) - cs);
        const float3 f = 0.5f * (A + B) + sc * (sinhf(t) * eh + sn * (cp * xi + sp * ze));
        sx[m] = f.x;
        sy[m] = f.y;
        sz[m] = f.z;
      }
      __syncwarp();
    }
    float lp, lq;
    path_logs(M, R, S, Q, qtab, S.zoff, [&](int i) { return f3(sx[i], sy[i], sz[i]); }, n, lane, lp, lq);
    if (lane == 0) {
      double ratio = 0.0;
      if (isfinite(lp) && isfinite(lq)) ratio = exp(static_cast<double>(lp) - static_cast<double>(lq));
      acc_s += sqrt(ratio);
      acc_r += ratio;
      acc_r2 += ratio * ratio;
      if (out_logr != nullptr) out_logr[q] = (isfinite(lp) && isfinite(lq)) ? lp - lq : kNegInf;
    }
    if (out_xyz != nullptr) {
      const size_t plane = static_cast<size_t>(n_draws) * out_stride;
      const size_t off = static_cast<size_t>(q) * out_stride;
      for (int i = lane; i < out_stride; i += 32) {
        const bool ok = i < n;
        out_xyz[off + i] = ok ? sx[i] + S.org[0] : 0.f;
        out_xyz[plane + off + i] = ok ? sy[i] + S.org[1] : 0.f;
        out_xyz[2 * plane + off + i] = ok ? sz[i] + S.org[2] : 0.f;
      }
      if (lane == 0) out_n[q] = n;
    }
    __syncwarp();
  }
  if (lane == 0 && sums != nullptr) {
    atomicAdd(sums + 4 * pair + 0, acc_s);
    atomicAdd(sums + 4 * pair + 1, acc_r);
    atomicAdd(sums + 4 * pair + 2, acc_r2);
  }
}

// Chain side of the bridge: sqrt(q_ref / p) at every chain's current state,
// summed per pair (sum, sum of squares, count).
__global__ void __launch_bounds__(128) qref_chain_kernel(const DMedium M, const DRun R, const DPair* __restrict__ pairs,
                                                         const QrefPair* __restrict__ qp, const double* __restrict__ qtab,
                                                         const int* __restrict__ chain_pair,
                                                         const long long* __restrict__ chain_base,
                                                         const float* __restrict__ xyz, const int* __restrict__ nn,
                                                         int total, double* __restrict__ sums) {
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= total) return;
  const int pair = chain_pair[c];
  const DPair S = pairs[pair];
  const int n = nn[c];
  const float* gx = xyz + chain_base[c];
  const float* gy = gx + S.cap;
  const float* gz = gy + S.cap;
  float lp, lq;
  path_logs(M, R, S, qp[pair], qtab, S.zoff, [&](int i) { return f3(gx[i], gy[i], gz[i]); }, n, lane, lp, lq);
  if (lane == 0) {
    const double v = (isfinite(lp) && isfinite(lq)) ? exp(0.5 * (static_cast<double>(lq) - static_cast<double>(lp))) : 0.0;
    atomicAdd(sums + 4 * pair + 0, v);
    atomicAdd(sums + 4 * pair + 1, v * v);
    atomicAdd(sums + 4 * pair + 2, 1.0);
  }
}

// Chain side of the optimal bridge for one pair: log(q_ref / p) at each of
// its chains' current paths, in chain order.
__global__ void __launch_bounds__(128) qref_chain_logr_kernel(const DMedium M, const DRun R, const DPair* __restrict__ S_,
                                                              const QrefPair* __restrict__ qp,
                                                              const double* __restrict__ qtab,
                                                              const long long* __restrict__ chain_base,
                                                              const float* __restrict__ xyz, const int* __restrict__ nn,
                                                              int chain0, int n_chains, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n_chains) return;
  const DPair S = *S_;
  const int c = chain0 + j;
  const int n = nn[c];
  const float* gx = xyz + chain_base[c];
  const float* gy = gx + S.cap;
  const float* gz = gy + S.cap;
  float lp, lq;
  path_logs(M, R, S, *qp, qtab, S.zoff, [&](int i) { return f3(gx[i], gy[i], gz[i]); }, n, lane, lp, lq);
  if (lane == 0) out[j] = (isfinite(lp) && isfinite(lq)) ? lq - lp : kNegInf;
}

// log q_ref of caller paths (absolute frame, SoA [3][batch][cap]).
__global__ void __launch_bounds__(128) qref_logdensity_kernel(const DMedium M, const DRun R, const DPair S,
                                                              const QrefPair* __restrict__ qp,
                                                              const double* __restrict__ qtab,
                                                              const float* __restrict__ xyz, const int* __restrict__ nn,
                                                              int batch, int cap, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= batch) return;
  const int n = nn[b];
  const size_t plane = static_cast<size_t>(batch) * cap, off = static_cast<size_t>(b) * cap;
  float lp, lq;
  if (n < 2 || n > cap || n > S.cap) {
    if (lane == 0) out[b] = __int_as_float(0x7fc00000);
    return;
  }
  path_logs(M, R, S, *qp, qtab, S.zoff,
            [&](int i) { return f3(xyz[off + i], xyz[plane + off + i], xyz[2 * plane + off + i]); }, n, lane, lp, lq);
  if (lane == 0) out[b] = lq;
}

cudaError_t launch_qref_draws(const DMedium& M, const DRun& R, const DPair* pairs, const QrefPair* qp,
                              const double* qtab, int n_pairs, int stream_base, int max_cap, unsigned long long seed, unsigned long long draw0,
                              unsigned long long n_draws, double* sums, float* out_xyz, int* out_n, int out_stride,
                              int n_sm, cudaStream_t s, float* out_logr) {
  if (n_pairs == 0 || n_draws == 0) return cudaSuccess;
  const int smem_cap = (max_cap + 31) / 32 * 32;
  const size_t smem = 4u * 3u * smem_cap * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(qref_draw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  unsigned long long blocks = (n_draws + 3) / 4;
  const unsigned long long maxb = std::max(1ull, static_cast<unsigned long long>(n_sm) * 16ull / n_pairs);
  if (blocks > maxb) blocks = maxb;
  dim3 grid(static_cast<unsigned>(blocks), static_cast<unsigned>(n_pairs));
  qref_draw_kernel<<<grid, 128, smem, s>>>(M, R, pairs, qp, qtab, smem_cap, stream_base, seed, draw0, n_draws, sums,
                                           out_xyz, out_n, out_stride, out_logr);
  return cudaGetLastError();
}

cudaError_t launch_qref_chain_logr(const DMedium& M, const DRun& R, const DPair* pair, const QrefPair* qp,
                                   const double* qtab, const long long* chain_base, const float* xyz, const int* n,
                                   int chain0, int n_chains, float* out, cudaStream_t s) {
  if (n_chains == 0) return cudaSuccess;
  qref_chain_logr_kernel<<<(n_chains + 3) / 4, 128, 0, s>>>(M, R, pair, qp, qtab, chain_base, xyz, n, chain0,
                                                            n_chains, out);
  return cudaGetLastError();
}

cudaError_t launch_qref_chains(const DMedium& M, const DRun& R, const DPair* pairs, const QrefPair* qp,
                               const double* qtab, const int* chain_pair, const long long* chain_base, const float* xyz, const int* n,
                               int total, double* sums, cudaStream_t s) {
  if (total == 0) return cudaSuccess;
  qref_chain_kernel<<<(total + 3) / 4, 128, 0, s>>>(M, R, pairs, qp, qtab, chain_pair, chain_base, xyz, n, total,
                                                    sums);
  return cudaGetLastError();
}

cudaError_t launch_qref_logdensity(const DMedium& M, const DRun& R, const DPair& S, const QrefPair* qp,
                                   const double* qtab, const float* xyz, const int* n, int batch, int cap, float* out, cudaStream_t s) {
  if (batch == 0) return cudaSuccess;
  qref_logdensity_kernel<<<(batch + 3) / 4, 128, 0, s>>>(M, R, S, qp, qtab, xyz, n, batch, cap, out);
  return cudaGetLastError();
}

}  // namespace pmc
