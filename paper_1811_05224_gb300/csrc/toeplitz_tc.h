#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <string>

#include "stbem.h"

namespace stbem {
bool apply_tc_supported(int nt, int nx, int n_rhs);
// y (FP64) = block-Toeplitz product of BF16 lag blocks A with BF16 x, on tcgen05.
// chunk <= 0: one FP32 accumulator over the whole chain; chunk > 0: FP32 partials
// of `chunk` 64-wide K steps each, Kahan-summed (compensated kernel).  The
// plain kernel's tile width (steps per tile) is tile_n (128 or 256), else the
// tuned value for this shape (stbem_tc_tune), else 256 for n_t > 128.
// With chunk > 0 and a partial-sum buffer `part` (exact_part_bytes()), products
// with few output tiles split each tile's lags into chunks and write (or add)
// the chunks' partial products to `part` instead of Y; tc_chunk_reduce_launch
// then sets Y to their sum (a no-op when the product does not split).
cudaError_t apply_tc_launch(int nt, int nx, const void* A_bf16, int n_rhs, const void* X_bf16, double* Y,
                            bool accumulate, cudaStream_t s, int chunk = 0, int tile_n = 0,
                            double* part = nullptr);
cudaError_t tc_chunk_reduce_launch(int nt, int nx, int n_rhs, const double* part, double* Y, cudaStream_t s);
// tune-cache key of the plain product's tile width, and the width in use
std::string tc_plain_tune_key(int nt, int nx, int n_rhs);
int tc_plain_tile_n(int nt, int nx, int n_rhs);
// hi/mid/lo BF16 slices of an FP64 array (mid and lo may be NULL)
cudaError_t bf16_split3_launch(const double* src, void* hi, void* mid, void* lo, size_t n, cudaStream_t s);
cudaError_t tc_error_reset(cudaStream_t s);
// Diagnostic: cycles > 0 makes every later plain tensor-core product wait on a
// barrier no thread arrives on (its pipeline waits limited to `cycles`), so it
// times out and reports through the error word; 0 restores normal operation.
void tc_set_stall(long long cycles);
cudaError_t tc_error_read(int* flag, cudaStream_t s);
// Exact-slice product (FP64-grade): S = n_slices integer slices of 6 bits per
// operand with power-of-two row scales (see exact_slices_launch), every slice
// pair with s + t < S multiplied exactly on the BF16 tensor cores.
constexpr int kExactMinSlices = 4, kExactMaxSlices = 8;
bool apply_tc_exact_supported(int nt, int nx, int n_rhs, int n_slices);
// slices [n_slices][rows][cols] BF16, row_exp [rows]
cudaError_t exact_slices_launch(const double* src, long long rows, int cols, int n_slices, void* slices,
                                int* row_exp, cudaStream_t s);
// part: scratch of exact_part_bytes() for products that split each output
// tile's lags into chunks (few output tiles: small n_rhs); NULL: no split
cudaError_t apply_tc_exact_launch(int nt, int nx, int n_slices, const void* A_slices, const int* A_exp, int n_rhs,
                                  const void* X_slices, const int* X_exp, double* Y, cudaStream_t s,
                                  double* part = nullptr);
constexpr int kExactLagChunk = 64;
int exact_lag_chunks(int nt, int nx, int n_rhs);
size_t exact_part_bytes(int nt, int nx, int n_rhs);
cudaError_t to_bf16_launch(int src_prec, const void* src, void* dst, size_t n, cudaStream_t s);
}  // namespace stbem
