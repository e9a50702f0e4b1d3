// Launch sizing from the device itself: grids are multiples of its SM count.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

namespace stbem {

// Streaming multiprocessors of the current device, queried once per device
// and cached.  Without a usable device (a size query on a host with no GPU)
// it returns 1; nothing is launched there, and workspace sizes derived from
// it are recomputed on the device that runs the work.
inline int sm_count() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return 1;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    (void)cudaGetLastError();
    return 1;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// Blocks for a grid-stride loop over n items with `threads` per block, at
// most `per_sm` blocks per SM.
inline int stride_grid(size_t n, int threads, int per_sm) {
  const size_t need = (n + threads - 1) / threads;
  const size_t cap = (size_t)sm_count() * per_sm;
  return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

}  // namespace stbem
