#pragma once
#include <cuda_runtime.h>
#include <cstddef>

#include "assemble.h"
#include "stbem.h"

namespace stbem {
size_t apply_workspace_bytes(int nt, int nx, int n_rhs);
// Fixed scratch of the allocation-free product (stbem_apply_noalloc).
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
constexpr int kNoAllocMaxDevices = 64;
// Device address of that scratch on `device` (which must be current); the
// first call in each CUDA context of a device resolves it with
// cudaGetSymbolAddress (so a context made after cudaDeviceReset gets a fresh
// lookup), later calls reuse it.
cudaError_t noalloc_scratch_ptr(int device, void** ptr);
// The product's grid (n_rhs x time tiles in gridDim.z) is within the launch
// limit of 65535; larger right-hand-side counts must be split by the caller.
bool apply_grid_fits(int nt, int nx, int n_rhs);
// Measured pipe rates of the current device: out[0] FP64 FMA TFLOP/s,
// out[1] FP32 FMA TFLOP/s, out[2] MUFU ex2 results per second (1e12).
cudaError_t pipe_peaks(double* out, cudaStream_t s);
cudaError_t apply_launch(int prec, bool trans, int nt, int nx, const void* A, int n_rhs,
                         const double* x, double* y, void* work, cudaStream_t s);
// The product restricted to the lags [lag_lo, lag_hi): A holds those lag
// blocks only (block d at A[d - lag_lo]); y = (accumulate ? y : 0) + sum.
size_t apply_range_workspace_bytes(int nt, int nx, int nlag, int n_rhs);
cudaError_t apply_range_launch(int prec, bool trans, int nt, int nx, int lag_lo, int lag_hi, const void* A,
                               int n_rhs, const double* x, double* y, bool accumulate, void* work, cudaStream_t s);

// Product plan of one problem of a ragged batch with `lags_per_chunk` lags per
// partial (the tuned shape) and the offsets of its data.
struct RaggedApplyPlan {
  int nt, nx, MT, IT, CH, DC;
  long long units, part_elems;
  long long a_off, v_off, part_off;
};
// fp32_tiles: the plan of the register-tiled FP32 kernel (128 x 64 tiles,
// needs ragged_fp32_tiles_ok(nx) for every problem), else the generic one.
void ragged_apply_plan(int nt, int nx, int lags_per_chunk, bool fp32_tiles, RaggedApplyPlan* p);
bool ragged_fp32_tiles_ok(int nx);
// y = A x for every problem: one persistent launch over all units (items:
// problem order + unit prefix sums), then one reduction over all outputs
// (vprefix: n_t N_x prefix sums in problem order).  counter: one device word.
// prec F32 with fp32_tiles uses the register-tiled kernel and its plans.
cudaError_t ragged_apply_launch(int prec, bool fp32_tiles, const RaggedApplyPlan* plans, RaggedItems items,
                                const long long* vprefix, int P, unsigned long long* counter, const void* A,
                                const double* x, double* y, double* part, cudaStream_t s);
}  // namespace stbem
