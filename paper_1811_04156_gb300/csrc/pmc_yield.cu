// Relative light yield of two sensors and path-length distributions
// (Collin, arXiv:1811.04156: section "Comparison of relative light yield" for
// the geometric estimator B = E_0[sqrt(p_1/p_0)] / E_1[sqrt(p_0/p_1)];
// appendix "Relative light yield transformation" for the map T of paths ending
// on sensor 0 to paths ending on sensor 1, p_1(x) = p(T x) |dT/dx|; section
// "Comparison of timing distributions" for the path-length distributions).
//
// T bends a path along a cylinder through the source: with intermediate
// coordinates xb = d.m / b0, yb = d.n / b0, w = d.k / b0 of d = f - f0,
//   T f = f0 - rC m + (rC + xb b1)(m cos(w Omega) + k sin(w Omega)) + n yb b1,
// a cylindrical map whose volume ratio is b1^2 Omega (rC + xb b1) / b0^3.  It
// is one-to-one where rC + xb b1 > 0 and |w Omega| < pi; outside that domain
// the other density is taken as 0.  The end vertex keeps its offset from the
// sensor centre, rotated by Omega in the (m, k) plane and scaled by R1/R0
// (area ratio (R1/R0)^2), so it lands exactly on sensor 1.
//
// FP32 forms: rC (cos a - 1) = -2 rC sin^2(a/2) and, for the inverse,
// rad - rC = ((p.m)(p.m + 2 rC) + (p.k)^2) / (rad + rC), which keep the
// vertices' precision where rC is much larger than the offsets.
#include <algorithm>

#include "pmc_internal.h"

namespace pmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ float3 ldv(const float* p) { return f3(p[0], p[1], p[2]); }

// Image of interior vertex f under T (side 0) or T^-1 (side 1); `lv`
// receives the log volume ratio log(vol (rC + xb b1)) at the side-0 point
// and `ok` is cleared outside the one-to-one domain.
__device__ __forceinline__ float3 map_interior(const DYMap& T, int side, float3 f, float& lv, bool& ok) {
  const float3 f0 = ldv(T.f0), k = ldv(T.k), m = ldv(T.m), n = ldv(T.n);
  const float3 d = f - f0;
  if (side == 0) {
    const float xb = dot(d, m) * T.inv_b0, yb = dot(d, n) * T.inv_b0, w = dot(d, k) * T.inv_b0;
    const float ang = w * T.Omega;
    const float rad = fmaf(xb, T.b1, T.rC);
    float sh, ch;
    sincosf(0.5f * ang, &sh, &ch);
    const float sa = 2.0f * sh * ch, ca = fmaf(-2.0f * sh, sh, 1.0f);
    const float cm = fmaf(-2.0f * T.rC * sh, sh, xb * T.b1 * ca);
    ok = ok && rad > 0.0f && fabsf(ang) < kPi;
    lv = logf(T.vol * rad);
    return f0 + (cm * m + (rad * sa) * k + (yb * T.b1) * n);
  }
  const float pm0 = dot(d, m), pk = dot(d, k), h = dot(d, n);
  const float pm = pm0 + T.rC;
  const float rad = sqrtf(fmaf(pm, pm, pk * pk));
  const float ang = atan2f(pk, pm);
  const float drad = fmaf(pm0, pm0 + 2.0f * T.rC, pk * pk) / (rad + T.rC);
  ok = ok && rad > 0.0f && fabsf(ang) < kPi;
  lv = logf(T.vol * rad);
  const float xb = drad / T.b1, yb = h / T.b1, w = ang / T.Omega;
  return f0 + T.b0 * (xb * m + yb * n + w * k);
}

// Image of the end vertex e on the sensor `Sin` on the sensor `Sout`.
__device__ __forceinline__ float3 map_end(const DYMap& T, int side, const DPair& Sin, const DPair& Sout, float3 e) {
  const float3 k = ldv(T.k), m = ldv(T.m), n = ldv(T.n);
  const float3 u = sensor_normal(Sin, e);
  const float um = dot(u, m), uk = dot(u, k), un = dot(u, n);
  const float s = side == 0 ? T.sinO : -T.sinO;
  const float vm = um * T.cosO - uk * s, vk = um * s + uk * T.cosO;
  const float Rout = side == 0 ? T.R1 : T.R0;
  const float3 v = vm * m + vk * k + un * n;
  return ldv(Sout.c) + (ldv(Sout.c_lo) + Rout * v);
}

// Log terms of one path for the ratio: own log density, the other density at
// the mapped path, log |dT/dx| (at the side-0 path), and the domain flag.
template <class PosF>
__device__ void ratio_terms(const DMedium& M, const DPair& Sself, const DPair& Soth, const DYMap& T, int side,
                            PosF pos, int n, int lane, float& l_self, float& l_oth, float& lj, bool& inside) {
  const float zoff = Sself.zoff;
  float a = 0.f, b = 0.f, c = 0.f;
  bool ok = true;
  auto mapped = [&](int i, float& lv) -> float3 {
    const float3 P = pos(i);
    if (i == 0) return P;  // the source is fixed
    if (i == n - 1) return map_end(T, side, Sself, Soth, P);
    return map_interior(T, side, P, lv, ok);
  };
  for (int i = lane; i < n; i += 32) {
    const float3 P = pos(i);
    const float3 Pp = (i >= 1) ? pos(i - 1) : P;
    const float3 Pn = (i <= n - 2) ? pos(i + 1) : P;
    float g;
    a += vertex_term(M, Sself, zoff, Pp, P, Pn, i, n, g);
    if (i <= n - 2) a += segment_term(M, Sself, zoff, P, Pn, i <= n - 3).seg;
    float lv = 0.f, dummy;
    const float3 Q = mapped(i, lv);
    const float3 Qp = (i >= 1) ? mapped(i - 1, dummy) : Q;
    const float3 Qn = (i <= n - 2) ? mapped(i + 1, dummy) : Q;
    b += vertex_term(M, Soth, zoff, Qp, Q, Qn, i, n, g);
    if (i <= n - 2) b += segment_term(M, Soth, zoff, Q, Qn, i <= n - 3).seg;
    if (i >= 1 && i <= n - 2) c += lv;
    if (i == n - 1) c += T.log_area;
  }
  l_self = wsum(a);
  l_oth = wsum(b);
  lj = wsum(c);
  inside = __all_sync(kFull, ok);
}

// log of the other density's ratio to the own one at this path: side 0
// (path on sensor 0) log p(T x; 1) + log|dT/dx| - log p(x; 0); side 1 (path
// y on sensor 1) log p(T^-1 y; 0) - log|dT/dx| - log p(y; 1).
__device__ __forceinline__ float log_ratio(int side, float l_self, float l_oth, float lj, bool inside) {
  if (!inside || !isfinite(l_oth) || !isfinite(l_self)) return kNegInf;
  return side == 0 ? (l_oth + lj) - l_self : (l_oth - lj) - l_self;
}

struct ChainPos {
  const float* x;
  int cap;
  __device__ float3 operator()(int i) const { return f3(x[i], x[cap + i], x[2 * cap + i]); }
};

struct BatchPos {
  const float* xyz;
  size_t plane, off;
  __device__ float3 operator()(int i) const {
    return f3(xyz[off + i], xyz[plane + off + i], xyz[2 * plane + off + i]);
  }
};

}  // namespace

// One warp per chain of pair0 (side 0) then pair1 (side 1): sums[j] += sqrt of
// the density ratio at the chain's current path (0 outside T's domain).
__global__ void __launch_bounds__(128) yield_chain_kernel(const DMedium M, const DPair* __restrict__ pairs, int pair0,
                                                          int pair1, const DYMap T,
                                                          const long long* __restrict__ chain_base,
                                                          const float* __restrict__ xyz, const int* __restrict__ nn,
                                                          int chain0_0, int n0, int chain0_1, int n1,
                                                          double* __restrict__ sums, float* __restrict__ logr) {
  const int lane = threadIdx.x & 31;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n0 + n1) return;
  const int side = j < n0 ? 0 : 1;
  const int c = side == 0 ? chain0_0 + j : chain0_1 + (j - n0);
  const DPair Sself = pairs[side == 0 ? pair0 : pair1];
  const DPair Soth = pairs[side == 0 ? pair1 : pair0];
  const int n = nn[c];
  float ls, lo, lj;
  bool inside;
  ratio_terms(M, Sself, Soth, T, side, ChainPos{xyz + chain_base[c], Sself.cap}, n, lane, ls, lo, lj, inside);
  if (lane == 0) {
    const float r = log_ratio(side, ls, lo, lj, inside);
    if (sums != nullptr) sums[j] += isfinite(r) ? exp(0.5 * static_cast<double>(r)) : 0.0;
    if (logr != nullptr) logr[j] = r;
  }
}

// Caller batch (absolute frame, SoA [3][batch][cap]): the log ratio per path
// and, optionally, the mapped path in the same layout.
__global__ void __launch_bounds__(128) yield_logratio_kernel(const DMedium M, const DPair S0, const DPair S1,
                                                             const DYMap T, int side, const float* __restrict__ xyz,
                                                             const int* __restrict__ nn, int batch, int cap,
                                                             float* __restrict__ out, float* __restrict__ out_xyz) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= batch) return;
  const int n = nn[b];
  const size_t plane = static_cast<size_t>(batch) * cap, off = static_cast<size_t>(b) * cap;
  if (n < 2 || n > cap) {
    if (lane == 0) out[b] = __int_as_float(0x7fc00000);
    return;
  }
  const DPair& Sself = side == 0 ? S0 : S1;
  const DPair& Soth = side == 0 ? S1 : S0;
  BatchPos pos{xyz, plane, off};
  float ls, lo, lj;
  bool inside;
  ratio_terms(M, Sself, Soth, T, side, pos, n, lane, ls, lo, lj, inside);
  if (lane == 0) out[b] = log_ratio(side, ls, lo, lj, inside);
  if (out_xyz != nullptr) {
    for (int i = lane; i < cap; i += 32) {
      float3 q = f3(0.f, 0.f, 0.f);
      if (i < n) {
        const float3 P = pos(i);
        float lv;
        bool ok = true;
        q = (i == 0) ? P : (i == n - 1) ? map_end(T, side, Sself, Soth, P) : map_interior(T, side, P, lv, ok);
      }
      out_xyz[off + i] = q.x;
      out_xyz[plane + off + i] = q.y;
      out_xyz[2 * plane + off + i] = q.z;
    }
  }
}

// B = E_0 / E_1 from per-chain sums of n_obs observations each; standard error
// by the delta method over the across-chain variances of the per-chain means.
__global__ void __launch_bounds__(256) yield_estimate_kernel(const double* __restrict__ sums, int n0, int n1,
                                                             double n_obs, double* __restrict__ out) {
  __shared__ double sh[4][8];
  double v[4] = {0, 0, 0, 0};
  for (int j = threadIdx.x; j < n0 + n1; j += blockDim.x) {
    const double x = sums[j] / n_obs;
    const int k = j < n0 ? 0 : 2;
    v[k] += x;
    v[k + 1] += x * x;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if (lane == 0) sh[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; ++k)
      for (int i = 0; i < 8; ++i) t[k] += sh[k][i];
    const double m0 = t[0] / n0, m1 = t[2] / n1;
    const double var0 = n0 > 1 ? fmax(t[1] - n0 * m0 * m0, 0.0) / (n0 - 1) : 0.0;
    const double var1 = n1 > 1 ? fmax(t[3] - n1 * m1 * m1, 0.0) / (n1 - 1) : 0.0;
    const double B = m0 / m1;
    out[0] = B;
    out[1] = B * sqrt(var0 / (n0 * m0 * m0) + var1 / (n1 * m1 * m1));
    out[2] = m0;
    out[3] = m1;
    out[4] = var0;
    out[5] = var1;
  }
}

// One warp per chain: the current path's length, binned per pair.
__global__ void __launch_bounds__(128) length_hist_kernel(const DPair* __restrict__ pairs,
                                                          const int* __restrict__ chain_pair,
                                                          const long long* __restrict__ chain_base,
                                                          const float* __restrict__ xyz, const int* __restrict__ nn,
                                                          int total, double lo, double bins_per_m, int n_bins,
                                                          double* __restrict__ hist) {
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= total) return;
  const int pair = chain_pair[c];
  const int cap = pairs[pair].cap;
  const ChainPos pos{xyz + chain_base[c], cap};
  const int n = nn[c];
  float L = 0.f;
  for (int i = lane; i < n - 1; i += 32) {
    const float3 r = pos(i + 1) - pos(i);
    L += sqrtf(dot(r, r));
  }
  L = wsum(L);
  if (lane == 0) {
    const double fb = (static_cast<double>(L) - lo) * bins_per_m;
    if (fb >= 0.0 && fb < static_cast<double>(n_bins))
      atomicAdd(hist + static_cast<size_t>(pair) * n_bins + static_cast<int>(fb), 1.0);
  }
}

cudaError_t launch_yield_chains(const DMedium& M, const DPair* pairs, int pair0, int pair1, const DYMap& T,
                                const long long* chain_base, const float* xyz, const int* n, int chain0_0, int n0,
                                int chain0_1, int n1, double* sums, float* logr, cudaStream_t s) {
  const int total = n0 + n1;
  if (total == 0) return cudaSuccess;
  yield_chain_kernel<<<(total + 3) / 4, 128, 0, s>>>(M, pairs, pair0, pair1, T, chain_base, xyz, n, chain0_0, n0,
                                                     chain0_1, n1, sums, logr);
  return cudaGetLastError();
}

// Optimal bridge (Meng & Wong 1996) from stored log ratios: rows of n0 side-0
// values log(q1/q0)(x), x ~ p0, then n1 side-1 values log(q0/q1)(x), x ~ p1.
// For the current ratio r_g of each chain group g (index `groups`: all
// chains), adds A_g = sum over side 0 of 1/(s1 + s0 r_g / l) and B_g = sum
// over side 1 of 1/(s1 l + s0 r_g), l = q1/q0, into acc[g][0..1]; with
// geometric != 0 it adds the geometric estimator's sums of sqrt(q1/q0) and
// sqrt(q0/q1) instead.  Group of a chain: its index within its side mod groups.
__global__ void __launch_bounds__(256) bridge_sums_kernel(const float* __restrict__ logr, unsigned long long rows,
                                                          int n0, int n1, int groups, const double* __restrict__ r,
                                                          double s0, double s1, int geometric,
                                                          unsigned long long rows_per, int n_chunks,
                                                          double* __restrict__ acc) {
  extern __shared__ double sh[];  // [groups + 1][2]
  for (int i = threadIdx.x; i < 2 * (groups + 1); i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  const int width = n0 + n1;
  // each thread owns one column (chain) and a range of rows, so its group is
  // fixed and its sums stay in registers until one shared-memory add
  const unsigned long long item = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x;
  if (item < static_cast<unsigned long long>(width) * n_chunks) {
    const int j = static_cast<int>(item % width);
    const unsigned long long chunk = item / width;
    const bool side0 = j < n0;
    const int g = (side0 ? j : j - n0) % groups;
    const double rg = r[g], rall = r[groups];
    double vg = 0.0, vall = 0.0;
    const unsigned long long r0 = chunk * rows_per, r1 = min(rows, r0 + rows_per);
    for (unsigned long long row = r0; row < r1; ++row) {
      const double lr = static_cast<double>(logr[row * width + j]);
      if (geometric) {
        const double v = isfinite(lr) ? exp(0.5 * lr) : 0.0;
        vg += v;
      } else if (side0) {
        const double l = exp(lr);  // q1/q0 at a p0 draw (0 outside T's domain)
        vg += 1.0 / (s1 + s0 * rg / l);
        vall += 1.0 / (s1 + s0 * rall / l);
      } else {
        const double l = exp(-lr);  // q1/q0 at a p1 draw
        vg += 1.0 / (s1 * l + s0 * rg);
        vall += 1.0 / (s1 * l + s0 * rall);
      }
    }
    if (geometric) vall = vg;
    const int k = side0 ? 0 : 1;
    atomicAdd(&sh[2 * g + k], vg);
    atomicAdd(&sh[2 * groups + k], vall);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * (groups + 1); i += blockDim.x)
    if (sh[i] != 0.0) atomicAdd(&acc[i], sh[i]);
}

cudaError_t launch_bridge_sums(const float* logr, unsigned long long rows, int n0, int n1, int groups,
                               const double* r, double s0, double s1, int geometric, double* acc, int n_sm,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 2 * (groups + 1), s);
  if (e != cudaSuccess) return e;
  const int width = n0 + n1;
  if (rows == 0 || width == 0) return cudaSuccess;
  // about 8 CTAs of 256 threads per SM: split the rows into chunks to get there
  const unsigned long long want = static_cast<unsigned long long>(n_sm) * 8ull * 256ull;
  unsigned long long n_chunks = std::max<unsigned long long>(1ull, want / width);
  n_chunks = std::min<unsigned long long>(n_chunks, rows);
  const unsigned long long rows_per = (rows + n_chunks - 1) / n_chunks;
  n_chunks = (rows + rows_per - 1) / rows_per;
  const unsigned long long threads = n_chunks * width;
  const unsigned blocks = static_cast<unsigned>((threads + 255) / 256);
  bridge_sums_kernel<<<blocks, 256, sizeof(double) * 2 * (groups + 1), s>>>(
      logr, rows, n0, n1, groups, r, s0, s1, geometric, rows_per, static_cast<int>(n_chunks), acc);
  return cudaGetLastError();
}

cudaError_t launch_yield_logratio(const DMedium& M, const DPair& S0, const DPair& S1, const DYMap& T, int side,
                                  const float* xyz, const int* n, int batch, int cap, float* out, float* out_xyz,
                                  cudaStream_t s) {
  if (batch == 0) return cudaSuccess;
  yield_logratio_kernel<<<(batch + 3) / 4, 128, 0, s>>>(M, S0, S1, T, side, xyz, n, batch, cap, out, out_xyz);
  return cudaGetLastError();
}

cudaError_t launch_yield_estimate(const double* sums, int n0, int n1, double n_obs, double* out, cudaStream_t s) {
  yield_estimate_kernel<<<1, 256, 0, s>>>(sums, n0, n1, n_obs, out);
  return cudaGetLastError();
}

cudaError_t launch_length_hist(const DPair* pairs, const int* chain_pair, const long long* chain_base,
                               const float* xyz, const int* n, int total, double lo, double hi, int n_bins,
                               double* hist, cudaStream_t s) {
  if (total == 0) return cudaSuccess;
  length_hist_kernel<<<(total + 3) / 4, 128, 0, s>>>(pairs, chain_pair, chain_base, xyz, n, total, lo,
                                                     static_cast<double>(n_bins) / (hi - lo), n_bins, hist);
  return cudaGetLastError();
}

}  // namespace pmc
