#pragma once
#include <cuda_runtime.h>

#include "rule.cuh"
#include "stbem.h"

namespace stbem {

// Device view of a boundary mesh (all arrays on the device).
struct DevMesh {
  int N, n_t;
  double ht, alpha;
  const double *sx0, *sy0, *sx1, *sy1, *slen, *snx, *sny;   // segments (N)
  const double *hx0, *hy0, *hx1, *hy1, *hlen, *hnx, *hny;   // half-segments (2N)
  const int* dpiece;                                         // dual pieces (4N)
  const double *dv0, *dv1, *dcurl;                           // psi at piece ends, d psi/ds
  const double *vx, *vy;                                     // vertices (N)
  double* sing;      // lag-0/1 moments of the 3 (2N) singular pairs (assembly scratch)
};

void build_rule_tables(RuleTables* t);
// process-wide count of kernel launches (incremented by every launcher)
void count_launches(unsigned n);
unsigned long long launch_count();
cudaError_t upload_rule_tables(const RuleTables& t, cudaStream_t s);
// Lags [lag_begin, lag_end) of op into out (the full n_t x N x N array).
cudaError_t assemble_launch(const DevMesh& M, int op, int prec, int lag_begin, int lag_end, void* out,
                            cudaStream_t s);

}  // namespace stbem
