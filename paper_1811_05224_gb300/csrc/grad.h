#pragma once
#include <cuda_runtime.h>
#include <cstddef>

#include "assemble.h"

namespace stbem {
// Device workspace of grad_launch for n_t steps and N segments.
size_t grad_workspace_bytes(int nt, int N);
// The gradient kernels' own copy of the rule tables.
cudaError_t upload_grad_rule_tables(const RuleTables& t, cudaStream_t s);
// dxy (N x 2) and dalpha (1) = lambda^T (df/dtheta - (dV/dtheta) w) for
// f = 1/2 M_h g + K_h g with g the datum of the source (ysx, ysy).
cudaError_t grad_launch(const DevMesh& M, const double* K, double ysx, double ysy, const double* g,
                        const double* w, const double* lam, double* dxy, double* dalpha, void* work,
                        cudaStream_t s);
}  // namespace stbem
