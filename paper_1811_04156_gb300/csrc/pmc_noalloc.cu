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
// Each photon is the tracer's own (trace_photon, pmc_tracer.cuh), for up to
// kNoAllocMaxPairs (128) source-sensor pairs per launch (grid.y = pair).
#include <mutex>

#include "pmc_internal.h"
#include "pmc_tracer.cuh"

namespace pmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Scratch shared by every call on a device: kNoAllocMaxPairs x 5 doubles (5 KB).
static __device__ __align__(256) double g_trace_scratch[kNoAllocMaxPairs * 5];

struct NoAllocPairs {
  DPair p[kNoAllocMaxPairs];
};

__global__ void __launch_bounds__(256) trace_pairs_kernel(const DMedium M, const NoAllocPairs pairs,
                                                          unsigned long long seed, unsigned long long photon0,
                                                          unsigned long long n_photons, float r_reject,
                                                          int max_scatter, double* __restrict__ scratch) {
  __shared__ double sh[8 * 5];
  const DPair& S = pairs.p[blockIdx.y];
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
// (the array's name in host code is only a host-side stand-in for it).  The
// address stays valid while the device's primary context lives; a
// cudaDeviceReset after the first call would leave it stale, which the
// library does not support.
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
