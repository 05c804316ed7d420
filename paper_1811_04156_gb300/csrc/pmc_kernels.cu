// Density, adjoint, score, normalisation, estimator and forward-tracer kernels
// (Collin, arXiv:1811.04156).
#include "pmc_internal.h"
#include "pmc_tracer.cuh"

namespace pmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Batch accessor: SoA [3][batch][cap] positions, evaluated in the caller's
// absolute frame (the pair struct passed to these kernels uses that frame).
struct BatchPos {
  const float* xyz;
  size_t plane, off;
  __device__ float3 operator()(int i) const {
    return f3(xyz[off + i], xyz[plane + off + i], xyz[2 * plane + off + i]);
  }
};

// log p of each path (one warp per path), and optionally d log p / d xyz.
__global__ void logp_kernel(const DMedium M, const DPair S, const float* __restrict__ xyz,
                            const int* __restrict__ nn, int batch, int cap, float* __restrict__ out_logp,
                            float* __restrict__ out_grad) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= batch) return;
  const int n = nn[b];
  const float zoff = S.zoff;
  BatchPos pos{xyz, static_cast<size_t>(batch) * cap, static_cast<size_t>(b) * cap};
  float lp = 0.f;
  if (n >= 2 && n <= cap) {
    for (int i = lane; i < n; i += 32) {
      const float3 P = pos(i);
      const float3 Pp = (i >= 1) ? pos(i - 1) : P;
      const float3 Pn = (i <= n - 2) ? pos(i + 1) : P;
      float g;
      lp += vertex_term(M, S, zoff, Pp, P, Pn, i, n, g);
      if (i <= n - 2) lp += segment_term(M, S, zoff, P, Pn, i <= n - 3).seg;
    }
    lp = warp_sum(lp);
  } else {
    lp = __int_as_float(0x7fc00000);  // NaN marks an invalid vertex count
  }
  if (lane == 0 && out_logp) out_logp[b] = lp;
  if (out_grad) {
    const size_t plane = static_cast<size_t>(batch) * cap;
    const size_t off = static_cast<size_t>(b) * cap;
    const bool ok = n >= 2 && n <= cap && isfinite(lp);
    for (int i = lane; i < cap; i += 32) {
      float3 g = f3(0.f, 0.f, 0.f);
      if (ok && i < n) g = grad_vertex(M, S, zoff, pos, n, i);
      out_grad[off + i] = g.x;
      out_grad[plane + off + i] = g.y;
      out_grad[2 * plane + off + i] = g.z;
    }
  }
}

// d log p / d theta per path.  Homogeneous theta = (lambda_s, lambda_a, g):
//   (L b^2 - (n-2) b, L a^2, sum_k d log sigma/d g);  layered theta =
// (lambda_s[l], lambda_a[l]): (len_l b_l^2 - n_l b_l, len_l a_l^2), with len_l
// the path length inside layer l and n_l its scattering vertices.
// `out` must be zeroed for layered media (per-layer terms are added atomically).
__global__ void score_kernel(const DMedium M, const DPair S, const float* __restrict__ xyz,
                             const int* __restrict__ nn, int batch, int cap, float* __restrict__ out,
                             int n_theta) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= batch) return;
  const int n = nn[b];
  if (n < 2 || n > cap) return;
  const float zoff = S.zoff;
  BatchPos pos{xyz, static_cast<size_t>(batch) * cap, static_cast<size_t>(b) * cap};
  float* o = out + static_cast<size_t>(b) * n_theta;
  if (M.kind == 0) {
    float L = 0.f, G = 0.f;
    for (int i = lane; i < n; i += 32) {
      const float3 P = pos(i);
      if (i <= n - 2) {
        const float3 r = pos(i + 1) - P;
        L += sqrtf(dot(r, r));
      }
      if (i >= 1 && i <= n - 2) {
        const float3 a0 = P - pos(i - 1), b0 = pos(i + 1) - P;
        float g;
        phase_term(M, rsqrtf(dot(a0, a0)) * a0, rsqrtf(dot(b0, b0)) * b0, g);
        G += g;
      }
    }
    L = warp_sum(L);
    G = warp_sum(G);
    if (lane == 0) {
      o[0] = L * M.b * M.b - static_cast<float>(n - 2) * M.b;
      o[1] = L * M.a * M.a;
      o[2] = G;
    }
    return;
  }
  const int NL = M.n_layers;
  for (int i = lane; i < n; i += 32) {
    const float3 P = pos(i);
    if (i >= 1 && i <= n - 2) {
      const int l = layer_of(M, P.z + zoff);
      atomicAdd(o + l, -__ldg(M.lb + l));
    }
    if (i <= n - 2) {
      const float3 Q = pos(i + 1);
      const float3 r = Q - P;
      const float ell = sqrtf(dot(r, r));
      const float zP = P.z + zoff, zQ = Q.z + zoff;
      const int lP = layer_of(M, zP), lQ = layer_of(M, zQ);
      const int l0 = min(lP, lQ), l1 = max(lP, lQ);
      const float zlo = fminf(zP, zQ), zhi = fmaxf(zP, zQ);
      for (int l = l0; l <= l1; ++l) {
        float frac = 1.0f;
        if (l0 != l1) {
          const float lo = (l == l0) ? zlo : M.z0 + l * M.dz;
          const float hi = (l == l1) ? zhi : M.z0 + (l + 1) * M.dz;
          frac = fmaxf(hi - lo, 0.f) / (zhi - zlo);
        }
        const float len = ell * frac;
        const float bl = __ldg(M.lb + l), al = __ldg(M.la + l);
        atomicAdd(o + l, len * bl * bl);
        atomicAdd(o + NL + l, len * al * al);
      }
    }
  }
}

// Block-wide sum of K doubles held by every thread (blockDim.x == 256).
template <int K>
__device__ void block_sum(double (&v)[K], double* sh) {
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if ((t & 31) == 0) sh[k * 8 + (t >> 5)] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = 0.0;
    for (int i = 0; i < 8; ++i) x += sh[k * 8 + i];
    v[k] = x;
  }
  __syncthreads();
}

// Direct-sector integral Z2 = int over the sensor seen from the source of
// eps(omega) exp(-tau) rho dOmega, with theta = theta_max (1 - v^2) to remove
// the square-root behaviour at the rim; FP32 integrand, FP64 sums.
__global__ void __launch_bounds__(256) z2_kernel(const DMedium M, const DPair* __restrict__ pairs, int n_v,
                                                 int n_phi, double* __restrict__ out) {
  __shared__ double sh[8 * 1];
  const DPair S = pairs[blockIdx.x];
  const float3 c = f3(S.c[0], S.c[1], S.c[2]);
  const float D = sqrtf(dot(c, c));
  const float3 ax = (1.0f / D) * c;
  float3 e1, e2;
  onb(ax, e1, e2);
  const float R = S.R;
  const float thmax = asinf(R / D);
  double acc = 0.0;
  const int total = n_v * n_phi;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int iv = idx / n_phi, ip = idx % n_phi;
    const float v = (iv + 0.5f) / n_v;
    const float th = thmax * (1.0f - v * v);
    const float jac = 2.0f * thmax * v / n_v;
    float st, ct, sp, cp;
    sincosf(th, &st, &ct);
    sincospif(2.0f * (ip + 0.5f) / n_phi, &sp, &cp);
    const float disc = fmaxf((R - D * st) * (R + D * st), 0.0f);
    const float r = D * ct - sqrtf(disc);
    const float3 om = ct * ax + st * (cp * e1 + sp * e2);
    const float3 h = r * om;
    float ta, tb;
    seg_tau(M, S.zoff, h.z + S.zoff, r, ta, tb);
    float lv = emission_term(S, om) - ta - tb;
    if (S.rho != 0) {
      const float3 nu = sensor_normal(S, h);
      const float x = dot(nu, f3(S.rho_hat[0], S.rho_hat[1], S.rho_hat[2]));
      lv += fmaf(3.0f, x, -1.0f) - logf(coshf(fmaf(2.0f, x, 0.7f)));
    }
    acc += static_cast<double>(expf(lv) * st * jac) * (2.0 * 3.14159265358979323846 / n_phi);
  }
  double vv[1] = {acc};
  block_sum<1>(vv, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = vv[0];
}

// Per-pair moments of the chain accumulators (one block per pair): sums
// over the pair's chains, each chain's terms from add_chain_moments.
__global__ void __launch_bounds__(256) moments_kernel(const double* __restrict__ acc, const DPair* __restrict__ pairs,
                                                      double ls, double la, double* __restrict__ out) {
  __shared__ double sh[8 * MOM_USED];
  const DPair S = pairs[blockIdx.x];
  double v[MOM_USED];
#pragma unroll
  for (int k = 0; k < MOM_USED; ++k) v[k] = 0.0;
  for (int c = S.chain0 + threadIdx.x; c < S.chain0 + S.n_chains; c += blockDim.x)
    add_chain_moments(acc + static_cast<size_t>(c) * ACC_WORDS, ls, la, v);
  block_sum<MOM_USED>(v, sh);
  if (threadIdx.x != 0) return;
  double* o = out + static_cast<size_t>(blockIdx.x) * PMC_MOMENT_WORDS;
#pragma unroll
  for (int k = 0; k < PMC_MOMENT_WORDS; ++k) o[k] = k < MOM_USED ? v[k] : 0.0;
}

// ---------------------------------------------------------------------------
// Forward tracer (appendix, "Ray tracer"; the photon itself in pmc_tracer.cuh):
// one thread per photon.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) trace_kernel(const DMedium M, const DPair S, unsigned long long seed,
                                                    unsigned long long photon0, unsigned long long n_photons,
                                                    float r_reject, int max_scatter, double* __restrict__ out5,
                                                    double* __restrict__ hist, double l_lo, double bins_per_m,
                                                    int n_bins) {
  __shared__ double sh[8 * 5];
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  double v[5] = {0, 0, 0, 0, 0};
  const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
  for (unsigned long long q = blockIdx.x * blockDim.x + threadIdx.x; q < n_photons; q += stride) {
    const PhotonResult pr = trace_photon<false>(M, S, k0, k1, photon0 + q, r_reject, max_scatter, nullptr, nullptr,
                                                nullptr);
    v[3] += 1.0;
    if (pr.hit) {
      const double W = static_cast<double>(expf(pr.lw));
      v[0] += W;
      v[1] += W * W;
      v[2] += 1.0;
      v[4] += W * static_cast<double>(pr.L);
      if (hist != nullptr) {
        const double fb = (static_cast<double>(pr.L) - l_lo) * bins_per_m;
        if (fb >= 0.0 && fb < static_cast<double>(n_bins)) atomicAdd(hist + static_cast<int>(fb), W);
      }
    }
  }
  block_sum<5>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) atomicAdd(out5 + k, v[k]);
  }
}

// Detected photons thinned by their weight w rho (<= 1): an accepted path is an
// exact draw from the normalised path density (cap-truncated by max_scatter).
// Accepted paths are written to out_xyz [3][max_paths][stride] (absolute) and
// out_n; *count counts every accepted path (also those beyond max_paths).
__global__ void __launch_bounds__(256) trace_paths_kernel(const DMedium M, const DPair S, unsigned long long seed,
                                                          unsigned long long photon0, unsigned long long n_photons,
                                                          float r_reject, int max_scatter, int max_paths, int stride,
                                                          float* __restrict__ out_xyz, int* __restrict__ out_n,
                                                          unsigned int* __restrict__ count) {
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  const unsigned long long gstride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
  const size_t plane = static_cast<size_t>(max_paths) * stride;
  for (unsigned long long q = blockIdx.x * blockDim.x + threadIdx.x; q < n_photons; q += gstride) {
    const PhotonResult pr = trace_photon<false>(M, S, k0, k1, photon0 + q, r_reject, max_scatter, nullptr, nullptr,
                                                nullptr);
    if (!pr.hit || !(pr.u_acc < expf(pr.lw))) continue;
    const unsigned int slot = atomicAdd(count, 1u);
    if (slot >= static_cast<unsigned int>(max_paths)) continue;
    float* ox = out_xyz + static_cast<size_t>(slot) * stride;
    trace_photon<true>(M, S, k0, k1, photon0 + q, r_reject, max_scatter, ox, ox + plane, ox + 2 * plane);
    out_n[slot] = pr.nsc + 2;
  }
}

// Per-layer scores of every chain's current path, summed per pair (layered
// media): theta = (lambda_s[l], lambda_a[l]) with d log p / d lambda_s[l] =
// len_l b_l^2 - n_l b_l and d log p / d lambda_a[l] = len_l a_l^2 (len_l: path
// length in layer l, n_l: scattering vertices in it).  One warp per chain; the
// chain's 2L scores are gathered in shared memory, then added (and squared)
// into the pair's FP64 sums.
__global__ void __launch_bounds__(128) chain_layer_score_kernel(const DMedium M, const DPair* __restrict__ pairs,
                                                                const int* __restrict__ chain_pair,
                                                                const long long* __restrict__ chain_base,
                                                                const float* __restrict__ xyz, const int* __restrict__ nn,
                                                                int total, double* __restrict__ sums) {
  extern __shared__ float sc[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int NL = M.n_layers;
  float* s = sc + static_cast<size_t>(wib) * 2 * NL;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= total) return;
  for (int j = lane; j < 2 * NL; j += 32) s[j] = 0.f;
  __syncwarp();
  const int pair = chain_pair[c];
  const DPair S = pairs[pair];
  const int n = nn[c];
  const float* gx = xyz + chain_base[c];
  const float* gy = gx + S.cap;
  const float* gz = gy + S.cap;
  const float zoff = S.zoff;
  for (int i = lane; i < n; i += 32) {
    const float3 P = f3(gx[i], gy[i], gz[i]);
    if (i >= 1 && i <= n - 2) {
      const int l = layer_of(M, P.z + zoff);
      atomicAdd(s + l, -__ldg(M.lb + l));
    }
    if (i <= n - 2) {
      const float3 Q = f3(gx[i + 1], gy[i + 1], gz[i + 1]);
      const float3 r = Q - P;
      const float ell = sqrtf(dot(r, r));
      const float zP = P.z + zoff, zQ = Q.z + zoff;
      const int lP = layer_of(M, zP), lQ = layer_of(M, zQ);
      const int l0 = min(lP, lQ), l1 = max(lP, lQ);
      const float zlo = fminf(zP, zQ), zhi = fmaxf(zP, zQ);
      for (int l = l0; l <= l1; ++l) {
        float frac = 1.0f;
        if (l0 != l1) {
          const float lo = (l == l0) ? zlo : M.z0 + l * M.dz;
          const float hi = (l == l1) ? zhi : M.z0 + (l + 1) * M.dz;
          frac = fmaxf(hi - lo, 0.f) / (zhi - zlo);
        }
        const float len = ell * frac;
        const float bl = __ldg(M.lb + l), al = __ldg(M.la + l);
        atomicAdd(s + l, len * bl * bl);
        atomicAdd(s + NL + l, len * al * al);
      }
    }
  }
  __syncwarp();
  double* out = sums + static_cast<size_t>(pair) * 4 * NL;
  for (int j = lane; j < 2 * NL; j += 32) {
    const double v = s[j];
    if (v != 0.0) {
      atomicAdd(out + j, v);
      atomicAdd(out + 2 * NL + j, v * v);
    }
  }
}

}  // namespace

cudaError_t launch_logp(const DMedium& M, const DPair& S, const float* xyz, const int* n, int batch, int cap,
                        float* out_logp, float* out_grad, cudaStream_t s) {
  if (batch == 0) return cudaSuccess;
  const int warps_per_block = 4;
  const int grid = (batch + warps_per_block - 1) / warps_per_block;
  logp_kernel<<<grid, warps_per_block * 32, 0, s>>>(M, S, xyz, n, batch, cap, out_logp, out_grad);
  return cudaGetLastError();
}

cudaError_t launch_score(const DMedium& M, const DPair& S, const float* xyz, const int* n, int batch, int cap,
                         float* out, int n_theta, const double*, const double*, cudaStream_t s) {
  if (batch == 0) return cudaSuccess;
  if (M.kind != 0) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * static_cast<size_t>(batch) * n_theta, s);
    if (e != cudaSuccess) return e;
  }
  const int grid = (batch + 3) / 4;
  score_kernel<<<grid, 128, 0, s>>>(M, S, xyz, n, batch, cap, out, n_theta);
  return cudaGetLastError();
}

cudaError_t launch_z2(const DMedium& M, const DPair* pairs, int n_pairs, int n_v, int n_phi, double* out,
                      cudaStream_t s) {
  if (n_pairs == 0) return cudaSuccess;
  z2_kernel<<<n_pairs, 256, 0, s>>>(M, pairs, n_v, n_phi, out);
  return cudaGetLastError();
}

cudaError_t launch_moments(const double* acc, const DPair* pairs, int n_pairs, double ls, double la, double* out,
                           cudaStream_t s) {
  if (n_pairs <= 0) return cudaSuccess;
  moments_kernel<<<n_pairs, 256, 0, s>>>(acc, pairs, ls, la, out);
  return cudaGetLastError();
}

cudaError_t launch_trace(const DMedium& M, const DPair& S, unsigned long long seed, unsigned long long photon0,
                         unsigned long long n_photons, float r_reject, int max_scatter, double* out5, int n_sm,
                         cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out5, 0, 5 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (n_photons == 0) return cudaSuccess;
  unsigned long long blocks = (n_photons + 255) / 256;
  const unsigned long long maxb = static_cast<unsigned long long>(n_sm) * 8ull;
  if (blocks > maxb) blocks = maxb;
  trace_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(M, S, seed, photon0, n_photons, r_reject,
                                                             max_scatter, out5, nullptr, 0.0, 0.0, 0);
  return cudaGetLastError();
}

cudaError_t launch_trace_lengths(const DMedium& M, const DPair& S, unsigned long long seed,
                                 unsigned long long photon0, unsigned long long n_photons, float r_reject,
                                 int max_scatter, double l_lo, double l_hi, int n_bins, double* out5, double* hist,
                                 int n_sm, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out5, 0, 5 * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, static_cast<size_t>(n_bins) * sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (n_photons == 0) return cudaSuccess;
  unsigned long long blocks = (n_photons + 255) / 256;
  const unsigned long long maxb = static_cast<unsigned long long>(n_sm) * 8ull;
  if (blocks > maxb) blocks = maxb;
  trace_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(M, S, seed, photon0, n_photons, r_reject,
                                                             max_scatter, out5, hist, l_lo,
                                                             static_cast<double>(n_bins) / (l_hi - l_lo), n_bins);
  return cudaGetLastError();
}

cudaError_t launch_layer_scores(const DMedium& M, const DPair* pairs, const int* chain_pair, const long long* chain_base,
                                const float* xyz, const int* n, int total, double* sums, cudaStream_t s) {
  if (total == 0) return cudaSuccess;
  const size_t smem = 4u * 2u * static_cast<size_t>(M.n_layers) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(chain_layer_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  chain_layer_score_kernel<<<(total + 3) / 4, 128, smem, s>>>(M, pairs, chain_pair, chain_base, xyz, n, total, sums);
  return cudaGetLastError();
}

// Chain seeding, first pass: the indices of the photons in [photon0,
// photon0 + n_photons) whose detection survives the thinning by w rho (the
// same test as trace_paths_kernel), in any order, into idx[0 .. cap_idx);
// *count receives how many there were (also beyond cap_idx).
__global__ void __launch_bounds__(256) seed_count_kernel(const DMedium M, const DPair S, unsigned long long seed,
                                                         unsigned long long photon0, unsigned long long n_photons,
                                                         float r_reject, int max_scatter,
                                                         unsigned long long* __restrict__ idx, unsigned int cap_idx,
                                                         unsigned int* __restrict__ count) {
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  const unsigned long long gstride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
  for (unsigned long long q = blockIdx.x * blockDim.x + threadIdx.x; q < n_photons; q += gstride) {
    const PhotonResult pr = trace_photon<false>(M, S, k0, k1, photon0 + q, r_reject, max_scatter, nullptr, nullptr,
                                                nullptr);
    if (!pr.hit || !(pr.u_acc < expf(pr.lw))) continue;
    const unsigned int slot = atomicAdd(count, 1u);
    if (slot < cap_idx) idx[slot] = photon0 + q;
  }
}

// Chain seeding, second pass: chain chain0 + i of pair S (i < n) takes the
// path of photon sel[i], traced again (the same photon gives the same path)
// and written straight into the chain's block in the source frame.
__global__ void __launch_bounds__(128) seed_record_kernel(const DMedium M, DPair S, unsigned long long seed,
                                                          float r_reject, const unsigned long long* __restrict__ sel,
                                                          int chain0, int n, const long long* __restrict__ chain_base,
                                                          float* __restrict__ xyz, int* __restrict__ nv,
                                                          int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = chain0 + i;
  S.org[0] = S.org[1] = S.org[2] = 0.f;  // record frame coordinates
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  float* gx = xyz + chain_base[c];
  const PhotonResult pr = trace_photon<true>(M, S, k0, k1, sel[i], r_reject, S.cap - 2, gx, gx + S.cap,
                                             gx + 2 * S.cap);
  nv[c] = pr.hit ? pr.nsc + 2 : 2;
  status[c] = pr.hit ? 0 : ST_BAD_N;
}

cudaError_t launch_seed_count(const DMedium& M, const DPair& S, unsigned long long seed, unsigned long long photon0,
                              unsigned long long n_photons, float r_reject, int max_scatter, unsigned long long* idx,
                              unsigned int cap_idx, unsigned int* count, int n_sm, cudaStream_t s) {
  if (n_photons == 0) return cudaSuccess;
  unsigned long long blocks = (n_photons + 255) / 256;
  const unsigned long long maxb = static_cast<unsigned long long>(n_sm) * 8ull;
  if (blocks > maxb) blocks = maxb;
  seed_count_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(M, S, seed, photon0, n_photons, r_reject,
                                                                  max_scatter, idx, cap_idx, count);
  return cudaGetLastError();
}

cudaError_t launch_seed_record(const DMedium& M, const DPair& S, unsigned long long seed, float r_reject,
                               const unsigned long long* sel, int chain0, int n, const long long* chain_base,
                               float* xyz, int* nv, int* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  seed_record_kernel<<<(n + 127) / 128, 128, 0, s>>>(M, S, seed, r_reject, sel, chain0, n, chain_base, xyz, nv,
                                                     status);
  return cudaGetLastError();
}

cudaError_t launch_trace_paths(const DMedium& M, const DPair& S, unsigned long long seed, unsigned long long photon0,
                               unsigned long long n_photons, float r_reject, int max_scatter, int max_paths, int stride,
                               float* out_xyz, int* out_n, unsigned int* count, int n_sm, cudaStream_t s) {
  if (n_photons == 0) return cudaSuccess;
  unsigned long long blocks = (n_photons + 255) / 256;
  const unsigned long long maxb = static_cast<unsigned long long>(n_sm) * 8ull;
  if (blocks > maxb) blocks = maxb;
  trace_paths_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(M, S, seed, photon0, n_photons, r_reject,
                                                                   max_scatter, max_paths, stride, out_xyz, out_n,
                                                                   count);
  return cudaGetLastError();
}

}  // namespace pmc
