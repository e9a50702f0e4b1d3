#pragma once
#include <cuda_runtime.h>
#include <cstddef>

#include "stbem.h"

namespace stbem {
size_t apply_workspace_bytes(int nt, int nx, int n_rhs);
cudaError_t apply_launch(int prec, bool trans, int nt, int nx, const void* A, int n_rhs,
                         const double* x, double* y, void* work, cudaStream_t s);
}  // namespace stbem
