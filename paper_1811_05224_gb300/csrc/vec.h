#pragma once
#include <cuda_runtime.h>

#include "assemble.h"

namespace stbem {
cudaError_t rhs_g_launch(const DevMesh& M, double ysx, double ysy, double* g, cudaStream_t s);
cudaError_t half_mass_add_launch(const DevMesh& M, const double* g, double* f, cudaStream_t s, int B = 1);
cudaError_t lumped_mass_launch(const DevMesh& M, double* L, cudaStream_t s);
// out[k] = <Q[k], v>, k = 0..k-1 (deterministic block reductions)
cudaError_t dots_launch(const double* Q, int k, const double* v, size_t n, double* out, cudaStream_t s);
// v -= sum_k h[k] Q[k]
cudaError_t sub_combination_launch(const double* Q, int k, const double* h, double* v, size_t n, cudaStream_t s);
// y = sum_k h[k] Q[k]
cudaError_t combination_launch(const double* Q, int k, const double* h, double* y, size_t n, cudaStream_t s);
cudaError_t scale_launch(const double* x, double a, double* y, size_t n, cudaStream_t s);
cudaError_t axpy_launch(double a, const double* x, double* y, size_t n, cudaStream_t s);       // y += a x
cudaError_t sub_launch(const double* a, const double* b, double* y, size_t n, cudaStream_t s);  // y = a - b
// y[m][i] = x[m][i] / L[i]
cudaError_t diag_div_launch(const double* x, const double* L, double* y, int nt, int nx, cudaStream_t s);
// batched (B right-hand sides of length n each, vectors [B][n], basis [k][B][n]):
// out[t][b] = <Q[t][b], U[b]>, t < k, one block per dot, fixed-order reduction
cudaError_t bdots_launch(const double* Q, int k, const double* U, int B, size_t n, double* out, cudaStream_t s);
// U[b] -= sum_t H[t][b] Q[t][b]
cudaError_t bsub_comb_launch(const double* Q, int k, const double* H, double* U, int B, size_t n, cudaStream_t s);
// Y[b] = sum_t C[t][b] Q[t][b]
cudaError_t bcomb_launch(const double* Q, int k, const double* C, double* Y, int B, size_t n, cudaStream_t s);
// Y[b] = a[b] X[b]
cudaError_t bscale_launch(const double* X, const double* a, double* Y, int B, size_t n, cudaStream_t s);
// ragged batches (P problems; vectors concatenated, vp = P + 1 prefix offsets):
// out[t][p] = <Q[t], U> on segment p (Q[t] = Q + t ldq), t < k
cudaError_t rdots_launch(const double* Q, size_t ldq, int k, const double* U, const long long* vp, int P,
                         double* out, cudaStream_t s);
// sub: U -= sum_t H[t][p] Q[t]; else U = sum_t H[t][p] Q[t]  (segment p)
cudaError_t rcomb_launch(const double* Q, size_t ldq, int k, const double* H, const long long* vp, int P, bool sub,
                         double* U, long long n, cudaStream_t s);
cudaError_t rscale_launch(const double* X, const double* a, const long long* vp, int P, double* Y, long long n,
                          cudaStream_t s);
// nrm = sqrt(sq), inv = active && nrm > 0 ? 1 / nrm : 0
cudaError_t rinv_launch(const double* sq, const int* active, int P, double* nrm, double* inv, cudaStream_t s);
cudaError_t rdiag_div_launch(const RaggedProblem* probs, const long long* vp, int P, const double* x, const double* L,
                             double* y, long long n, cudaStream_t s);
cudaError_t rrhs_g_launch(const RaggedProblem* probs, const long long* vp, int P, const double* ystar, double* g,
                          long long n, cudaStream_t s);
cudaError_t rhalf_mass_add_launch(const RaggedProblem* probs, const long long* vp, int P, const double* g, double* f,
                                  long long n, cudaStream_t s);
cudaError_t rlumped_launch(const RaggedProblem* probs, int P, int max_n, double* L, cudaStream_t s);
// Y[m] = B X[m] (or B^T X[m]) for each of `rows` steps; B N x N row-major (FP64)
cudaError_t blockmul_launch(int rows, int N, const double* B, bool trans, const double* X, double* Y,
                            cudaStream_t s);
// dst[i] = (float)src[i]
cudaError_t round_f32_launch(const double* src, float* dst, size_t n, cudaStream_t s);
// non-uniform time grids (tn: n_t + 1 device time nodes)
cudaError_t nu_rhs_launch(const DevMesh& M, const double* tn, double ysx, double ysy, double* g, cudaStream_t s);
cudaError_t nu_half_mass_add_launch(const DevMesh& M, const double* tn, const double* g, double* f, cudaStream_t s);
cudaError_t nu_lumped_launch(const DevMesh& M, const double* tn, double* L, cudaStream_t s);
}  // namespace stbem
