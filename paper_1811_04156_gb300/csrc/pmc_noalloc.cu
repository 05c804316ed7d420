// Allocation-free variant of the forward-tracer launch (pmc_trace_noalloc).
//
// Some callers cannot call cudaMalloc: an application whose own pool
// allocator has reserved the device memory up front, one that enforces a
// fixed memory budget, or one that cannot accept the device-wide
// synchronisation a cudaMalloc / cudaFree pair can cause.  pmc_trace
// cudaMallocs its five FP64 accumulators on every call; this variant keeps
// its accumulators in a file-scope device array instead, which every GPU that
// loads the library holds until the process exits, so a call allocates nothing.
//
// The photon loop is the same computation as pmc_trace (appendix,
// Algorithm 1), repeated here for up to kNoAllocMaxPairs (128) source-sensor
// pairs per launch (grid.y = pair).
#include <mutex>

#include "pmc_internal.h"

namespace pmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Scratch shared by every call on a device: kNoAllocMaxPairs x 5 doubles (5 KB).
static __device__ __align__(256) double g_trace_scratch[kNoAllocMaxPairs * 5];

struct NoAllocPairs {
  DPair p[kNoAllocMaxPairs];
};

__device__ float na_free_path(const DMedium& M, float z_abs, float nz, float tau) {
  if (M.kind == 0) return tau / M.b;
  float dL = 0.f;
  float z = z_abs;
  int l = layer_of(M, z);
  for (int guard = 0; guard < 1 << 16; ++guard) {
    const float b = __ldg(M.lb + l);
    float dist = __int_as_float(0x7f800000);
    int next = l;
    if (nz > 0.f && l < M.n_layers - 1) {
      dist = (M.z0 + (l + 1) * M.dz - z) / nz;
      next = l + 1;
    } else if (nz < 0.f && l > 0) {
      dist = (M.z0 + l * M.dz - z) / nz;
      next = l - 1;
    }
    dist = fmaxf(dist, 0.f);
    if (tau <= b * dist) return dL + tau / b;
    tau -= b * dist;
    dL += dist;
    z += dist * nz;
    l = next;
  }
  return dL;
}

__device__ float na_ray_sphere(float3 x, float3 nh, float3 c, float R2) {
  const float3 w = x - c;
  const float b = dot(w, nh);
  const float cc = dot(w, w) - R2;
  const float disc = b * b - cc;
  if (disc < 0.f) return __int_as_float(0x7f800000);
  const float s1 = -b - sqrtf(disc);
  return s1 > 0.f ? s1 : __int_as_float(0x7f800000);
}

__device__ float na_sample_cos(const DMedium& M, float u, float umix) {
  if (M.f_sl > 0.f && umix < M.f_sl) {
    const float v = powf(u, 1.0f / (M.sl_alpha + 1.0f));
    return 2.0f * v - 1.0f;
  }
  const float g = M.g;
  if (fabsf(g) < 1e-6f) return 2.0f * u - 1.0f;
  const float q = (1.0f - g * g) / (1.0f - g + 2.0f * g * u);
  return fminf(fmaxf((1.0f + g * g - q * q) / (2.0f * g), -1.0f), 1.0f);
}

__global__ void __launch_bounds__(256) trace_pairs_kernel(const DMedium M, const NoAllocPairs pairs,
                                                          unsigned long long seed, unsigned long long photon0,
                                                          unsigned long long n_photons, float r_reject,
                                                          int max_scatter, double* __restrict__ scratch) {
  __shared__ double sh[8 * 5];
  const DPair& S = pairs.p[blockIdx.y];
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  const float3 c = f3(S.c[0], S.c[1], S.c[2]);
  double v[5] = {0, 0, 0, 0, 0};
  const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
  for (unsigned long long q = blockIdx.x * blockDim.x + threadIdx.x; q < n_photons; q += stride) {
    const unsigned long long ph = photon0 + q;
    const uint32_t plo = static_cast<uint32_t>(ph), phi = static_cast<uint32_t>(ph >> 32);
    uint4 r = philox4x32_10(make_uint4(plo, phi, 0u, PUR_TRACE), k0, k1);
    float3 x = f3(0.f, 0.f, 0.f);
    float3 nh;
    {
      float sp, cp;
      sincospif(2.0f * u01(r.y), &sp, &cp);
      if (S.emission != 0) {
        const float u0 = u01(r.x);
        const float ww = 1.0f + logf(fmaf(1.0f - u0, expf(-2.0f * S.kappa), u0)) / S.kappa;
        const float sw = sqrtf(fmaxf(0.f, 1.0f - ww * ww));
        const float3 d = f3(S.dir[0], S.dir[1], S.dir[2]);
        float3 e1, e2;
        onb(d, e1, e2);
        nh = ww * d + sw * (cp * e1 + sp * e2);
      } else {
        const float ww = 2.0f * u01(r.x) - 1.0f;
        const float sw = sqrtf(fmaxf(0.f, 1.0f - ww * ww));
        nh = f3(sw * cp, sw * sp, ww);
      }
    }
    float lnw = 0.f, L = 0.f;
    v[3] += 1.0;
    for (int i = 0; i <= max_scatter; ++i) {
      r = philox4x32_10(make_uint4(plo, phi, static_cast<uint32_t>(i + 1), PUR_TRACE), k0, k1);
      const float tau = -logf(u01(r.x));
      const float dL = na_free_path(M, x.z + S.zoff, nh.z, tau);
      const float dist = na_ray_sphere(x, nh, c, S.R2);
      const float go = fminf(dist, dL);
      const float3 end = x + go * nh;
      float ta, tb;
      seg_tau(M, x.z + S.zoff, end.z + S.zoff, go, ta, tb);
      lnw -= ta;
      if (dist < dL) {
        float lw = lnw;
        if (S.rho != 0) {
          const float3 nu = sensor_normal(S, end);
          const float xx = dot(nu, f3(S.rho_hat[0], S.rho_hat[1], S.rho_hat[2]));
          lw += fmaf(3.0f, xx, -1.0f) - logf(coshf(fmaf(2.0f, xx, 0.7f)));
        }
        const double W = static_cast<double>(expf(lw));
        v[0] += W;
        v[1] += W * W;
        v[2] += 1.0;
        v[4] += W * static_cast<double>(L + dist);
        break;
      }
      const float3 rel = x - c;
      if (dot(rel, rel) > r_reject * r_reject) break;
      if (i == max_scatter) break;
      x = end;
      L += dL;
      const float cs = na_sample_cos(M, u01(r.y), u01(r.w));
      const float sn = sqrtf(fmaxf(0.f, 1.0f - cs * cs));
      float sp, cp;
      sincospif(2.0f * u01(r.z), &sp, &cp);
      float3 e1, e2;
      onb(nh, e1, e2);
      nh = cs * nh + sn * (cp * e1 + sp * e2);
      nh = rsqrtf(dot(nh, nh)) * nh;
    }
  }
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double xk = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) xk += __shfl_xor_sync(kFull, xk, o);
    if ((t & 31) == 0) sh[k * 8 + (t >> 5)] = xk;
  }
  __syncthreads();
  if (t < 5) {
    double xk = 0.0;
    for (int i = 0; i < 8; ++i) xk += sh[t * 8 + i];
    atomicAdd(scratch + blockIdx.y * 5 + t, xk);
  }
}

// Device address of g_trace_scratch per device, looked up once per device
// (the array's name in host code is only a host-side stand-in for it).
std::mutex g_mu;
double* g_scratch_addr[64] = {};

cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_addr[device] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_trace_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_trace_noalloc(const DMedium& M, const DPair* pairs, int n_pairs, unsigned long long seed,
                                 unsigned long long photon0, unsigned long long n_photons, float r_reject,
                                 int max_scatter, double* host_out, int device, int n_sm, cudaStream_t s) {
  double* scratch = nullptr;
  cudaError_t e = scratch_address(device, &scratch);
  if (e != cudaSuccess) return e;
  NoAllocPairs pp{};
  for (int i = 0; i < n_pairs; ++i) pp.p[i] = pairs[i];
  // the array keeps the previous call's sums: clear the slots this call uses
  e = cudaMemsetAsync(scratch, 0, sizeof(double) * 5 * static_cast<size_t>(n_pairs), s);
  if (e != cudaSuccess) return e;
  if (n_photons > 0) {
    unsigned long long blocks = (n_photons + 255) / 256;
    const unsigned long long maxb = (static_cast<unsigned long long>(n_sm) * 8ull + n_pairs - 1) / n_pairs;
    if (blocks > maxb) blocks = maxb;
    if (blocks < 1) blocks = 1;
    dim3 grid(static_cast<unsigned>(blocks), static_cast<unsigned>(n_pairs));
    trace_pairs_kernel<<<grid, 256, 0, s>>>(M, pp, seed, photon0, n_photons, r_reject, max_scatter, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  e = cudaMemcpyAsync(host_out, scratch, sizeof(double) * 5 * static_cast<size_t>(n_pairs),
                      cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace pmc
