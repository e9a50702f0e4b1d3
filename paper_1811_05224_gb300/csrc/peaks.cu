// Arithmetic-pipe peaks of the device, measured: the denominators of the
// rooflines of the ALU-bound kernels (assembly and single-right-hand-side
// products are bound by the FP64 pipe, the mixed-precision assembly by FP32
// FMA and the MUFU exponential).  Each kernel runs independent dependency
// chains per thread so that the pipe, not latency, limits it; the grid fills
// every SM with several resident blocks.  Timed with CUDA events on the
// caller's stream after a warm-up launch.
#include <cuda_runtime.h>

#include "assemble.h"
#include "device_info.h"

namespace stbem {

namespace {

constexpr int kPeakThreads = 256, kPeakBlocksPerSm = 8, kChains = 8;
constexpr int kSinkSlots = 1 << 14;   // >= blocks of any launch below (checked)

// Write-only target that keeps the chains live; no host code takes its address.
__device__ double g_peak_sink[kSinkSlots];

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)12345.678) g_peak_sink[blockIdx.x] = (double)s;     // never true; keeps the chains live
}

__device__ __forceinline__ float ex2_approx(float v) {
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ex2(int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = -1e-3f * (float)(threadIdx.x + c);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = -ex2_approx(x[c]);    // stays in [-1, -0.5]
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) g_peak_sink[blockIdx.x] = (double)s;
}

template <typename F>
cudaError_t time_kernel(F launch, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  launch();                              // warm-up
  e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    launch();
    e = cudaEventRecord(e1, s);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

cudaError_t pipe_peaks(double* out, cudaStream_t s) {
  const int blocks = sm_count() * kPeakBlocksPerSm;
  if (blocks > kSinkSlots) return cudaErrorInvalidConfiguration;
  const double threads = (double)blocks * kPeakThreads;
  float ms = 0.f;
  // FP64 FMA: 2 flops per FMA
  const int it64 = 256;
  cudaError_t e = time_kernel(
      [&] { k_peak_fma<double><<<blocks, kPeakThreads, 0, s>>>(it64, 0.999999, 1e-7); },
      s, &ms);
  if (e != cudaSuccess) return e;
  out[0] = 2.0 * threads * it64 * 16 * kChains / (ms * 1e-3) / 1e12;
  // FP32 FMA
  const int it32 = 8192;
  e = time_kernel(
      [&] { k_peak_fma<float><<<blocks, kPeakThreads, 0, s>>>(it32, 0.999999f, 1e-7f); },
      s, &ms);
  if (e != cudaSuccess) return e;
  out[1] = 2.0 * threads * it32 * 16 * kChains / (ms * 1e-3) / 1e12;
  // MUFU ex2 (results per second)
  const int itx = 1024;
  e = time_kernel([&] { k_peak_ex2<<<blocks, kPeakThreads, 0, s>>>(itx); }, s, &ms);
  if (e != cudaSuccess) return e;
  out[2] = threads * itx * 16 * kChains / (ms * 1e-3) / 1e12;
  count_launches(6);
  return cudaSuccess;
}

}  // namespace stbem
