// Pipe-rate microbenchmark of the benchmark harness (a library of its own,
// libpmcprobe.so, outside the product library and its C ABI): the FP32 FMA
// and the MUFU (special-function unit) lane-operation rates of the device,
// measured rather than taken from unit counts, for the lane-op roofline of
// the chain kernels.
//
// Each thread runs 8 independent dependency chains so that the pipes, not
// their latency, bind; the grid fills every SM with 8 CTAs of 256 threads.
// FP32: a = fma(a, m, c) per chain and iteration.  MUFU: x = ex2(lg2(x)) per
// chain and iteration (two MUFU operations; the value stays ~x).
#include <algorithm>

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_rate_kernel(int iters, float m, float c, float* __restrict__ out) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-3f * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float mufu_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float mufu_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(kThreads) mufu_rate_kernel(int iters, float* __restrict__ out) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.5f + 1e-3f * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = mufu_ex2(mufu_lg2(a[k]));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t measure_pipes(int n_sm, double* fp32_per_s, double* mufu_per_s, cudaStream_t s) {
  const int blocks = n_sm * 8;
  float* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&d_out, sizeof(float) * static_cast<size_t>(blocks) * kThreads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int fma_iters = 1 << 14, mufu_iters = 1 << 12;
  float ms_f = 0.f, ms_m = 0.f;
  // untimed warm-up of both kernels, then one timed launch of each
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    const int fi = rep == 0 ? 64 : fma_iters, mi = rep == 0 ? 64 : mufu_iters;
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) fma_rate_kernel<<<blocks, kThreads, 0, s>>>(fi, 0.9999999f, 1e-7f, d_out);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess && rep == 1) e = cudaEventElapsedTime(&ms_f, e0, e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) mufu_rate_kernel<<<blocks, kThreads, 0, s>>>(mi, d_out);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess && rep == 1) e = cudaEventElapsedTime(&ms_m, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_out) cudaFree(d_out);
  if (e != cudaSuccess) return e;
  const double lanes = static_cast<double>(blocks) * kThreads * kChains;
  *fp32_per_s = lanes * 8.0 * fma_iters / (std::max(ms_f, 1e-6f) * 1e-3);
  *mufu_per_s = lanes * 8.0 * mufu_iters / (std::max(ms_m, 1e-6f) * 1e-3);
  return cudaSuccess;
}

}  // namespace

// out[0] = FP32 fused multiply-add lane-operations per second, out[1] = MUFU
// lane-operations per second of CUDA device `device` (8 independent
// dependency chains per thread, 8 CTAs of 256 threads per SM, one untimed and
// one timed launch of each kernel, CUDA events on `stream`).  Allocates and
// frees a 1.2 MB device buffer.  Returns 0, or the cudaError_t of the first
// failing call.  Synchronises `stream`.
extern "C" __attribute__((visibility("default"))) int pmcprobe_measure_pipes(int device, double* out, void* stream) {
  if (out == nullptr) return static_cast<int>(cudaErrorInvalidValue);
  cudaError_t e = cudaSetDevice(device);
  int n_sm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = measure_pipes(n_sm, &out[0], &out[1], static_cast<cudaStream_t>(stream));
  return static_cast<int>(e);
}
