#pragma once
#include <cuda_runtime.h>
#include <cstddef>

#include "stbem.h"

namespace stbem {
size_t apply_workspace_bytes(int nt, int nx, int n_rhs);
// Fixed scratch of the allocation-free product (stbem_apply_noalloc).
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
constexpr int kNoAllocMaxDevices = 64;
// Device address of that scratch on `device` (which must be current); the
// first call per device resolves it with cudaGetSymbolAddress.
cudaError_t noalloc_scratch_ptr(int device, void** ptr);
cudaError_t apply_launch(int prec, bool trans, int nt, int nx, const void* A, int n_rhs,
                         const double* x, double* y, void* work, cudaStream_t s);
}  // namespace stbem
