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

// One problem of a ragged batch: its mesh and the element offsets of its
// data in the batch's concatenated arrays.
struct RaggedProblem {
  DevMesh M;
  long long op_off;    // lag blocks: n_t x N x N elements from here
  long long vec_off;   // n_t x N vectors
  long long mass_off;  // N-vectors (lumped mass)
};

// Work list of a persistent launch over a ragged batch: problems in the order
// `order` (P entries, largest first), item counts as prefix sums (P + 1).
struct RaggedItems {
  const int* order;
  const long long* prefix;
};

void build_rule_tables(RuleTables* t);
// tiles of one lag block (host copy of the assembly's tiling)
int assembly_tiles_per_lag(int op, int N);
// lag groups of op on n_t steps (lags 0, 1 singly, then runs of consecutive
// lags assembled together); the ragged tile items are groups x tiles
int assembly_lag_groups(int op, int prec, int nt);
// All lag blocks of op for every problem of a ragged batch: one persistent
// launch for the identical / vertex-sharing pairs at lags 0 and 1 (items:
// problem x lag x pair slot) and one for the tiles (problem x lag x tile).
// counters: two device words (reset here).
// tile_items must have been counted with assembly_lag_groups(op, prec, n_t).
cudaError_t ragged_assemble_launch(int op, int prec, const RaggedProblem* probs, int P, RaggedItems sing_items,
                                   RaggedItems tile_items, unsigned long long* counters, void* out,
                                   cudaStream_t s);
// process-wide count of kernel launches (incremented by every launcher)
void count_launches(unsigned n);
unsigned long long launch_count();
cudaError_t upload_rule_tables(const RuleTables& t, cudaStream_t s);
// Lags [lag_begin, lag_end) of op into out (the full n_t x N x N array).
cudaError_t assemble_launch(const DevMesh& M, int op, int prec, int lag_begin, int lag_end, void* out,
                            cudaStream_t s);
// Non-uniform time grid (tn: n_t + 1 device time nodes): every block (m, n),
// n <= m, of op into out, packed p = m (m + 1) / 2 + n, N x N each (FP64).
cudaError_t nu_assemble_launch(const DevMesh& M, const double* tn, int op, double* out, cudaStream_t s);
// y[m] = sum_{n <= m} A[p(m, n)] x[n] for packed blocks (one right-hand side).
cudaError_t nu_apply_launch(int nt, int nx, const double* A, const double* x, double* y, cudaStream_t s);

}  // namespace stbem
