// Multi-right-hand-side block-Toeplitz product on the 5th-generation tensor
// cores (tcgen05, sm_103a), BF16 operands with FP32 accumulation:
//
//   y[b][m][i] = sum_{d=0}^{m} sum_j A[d][i][j] x[b][m-d][j]
//
// (Section 3 block structure; with many right-hand sides each lag is a dense
// GEMM A^(d) X_shifted).  One CTA owns a 128 x 128 output tile -- rows i of
// one lag block, columns m (time steps) of one right-hand side b -- and loops
// over all lags d <= m and 64-wide chunks of j:
//   * one thread issues TMA loads of A^(d)[i0:i0+128][j0:j0+64] and of
//     x[b][m0-d : m0-d+128][j0:j0+64] (128B swizzle) into a 4-stage ring;
//     rows with m - d < 0 lie outside the tensor and arrive as zeros, which is
//     exactly the causal (block lower triangular) structure;
//   * one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = N =
//     128, K = 16) into a 128-column TMEM accumulator and frees each stage with
//     tcgen05.commit;
//   * all four warps read the accumulator with tcgen05.ld and write FP64.
// Every mbarrier wait is bounded (about a second of clock64); on time-out the
// thread records an error in g_tc_error, skips the rest of its work and the
// CTA still releases its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "assemble.h"
#include "device_info.h"
#include "toeplitz_tc.h"
#include "tune_cache.h"

namespace stbem {

__device__ int g_tc_error;

namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4, THREADS = 128;
constexpr uint32_t A_BYTES = BM * BK * 2;
constexpr uint32_t B_BYTES = BN * BK * 2;
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 128;
constexpr size_t SMEM_BYTES = 1024 + STAGES * (size_t)STAGE_BYTES + 256;
constexpr long long kWaitCycles = 1LL << 31;   // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kWaitCycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// After a failed pipeline wait some TMA loads may still be in flight into this
// CTA's shared memory: the producer waits (bounded) for the last load it
// issued on every stage before the CTA releases its resources and exits.
__device__ __forceinline__ void drain_loads(uint64_t* full, int issued, int stages = STAGES) {
  for (int s = 0; s < stages && s < issued; ++s) {
    const int last = s + ((issued - 1 - s) / stages) * stages;   // last iteration that used stage s
    mbar_wait(&full[s], static_cast<uint32_t>(last / stages) & 1);
  }
}

__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, uint64_t* bar, void* dst, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// K-major operand in the 128-byte swizzled layout written by TMA: rows of 128 B,
// 8-row atoms of 1024 B (stride byte offset), descriptor version 1, swizzle
// mode 2 (128B).  The tile base is 1024-aligned; a K step of 16 BF16 elements
// advances the start address by 32 B.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = (addr >> 4) & 0x3FFFull;
  d |= 1ull << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: 8 rows x 128 B
  d |= 1ull << 46;                   // descriptor version
  d |= 2ull << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N (N >> 3 at bit 17), M = 128 (M >> 4 at bit 24).
constexpr uint32_t idesc_for(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
constexpr uint32_t kIdesc = idesc_for(BN);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate,
                                          uint32_t idesc = kIdesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Plain kernel, output tile 128 x BN_ (BN_ = 128 or 256 time steps).
template <int BN_>
struct TcTile {
  static constexpr uint32_t b_bytes = BN_ * BK * 2;
  static constexpr uint32_t stage_bytes = A_BYTES + b_bytes;
  static constexpr uint32_t tmem_cols = BN_;
  static constexpr size_t smem_bytes = 1024 + STAGES * (size_t)stage_bytes + 256;
  static constexpr uint32_t idesc = idesc_for(BN_);
};

template <int BN_>
__global__ void __launch_bounds__(THREADS, 1)
    k_apply_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, int nt, int nx,
               int accumulate, double* __restrict__ Y, long long stall_cycles) {
  using TT = TcTile<BN_>;
  constexpr int BN = BN_;
  constexpr uint32_t B_BYTES = TT::b_bytes, STAGE_BYTES = TT::stage_bytes, TMEM_COLS = TT::tmem_cols;
  extern __shared__ unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023);
  unsigned char* smA = reinterpret_cast<unsigned char*>(base);
  unsigned char* smB = smA + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint64_t* stallbar = accum + 1;     // diagnostic: a barrier no thread arrives on
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(stallbar + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grid (row tiles, right-hand sides, step tiles), step tiles longest first
  const int i0 = blockIdx.x * BM, b = blockIdx.y, m0 = (gridDim.z - 1 - blockIdx.z) * BN;
  const int dmax = min(m0 + BN - 1, nt - 1);  // lags for which some m - d >= 0
  const int nj = (nx + BK - 1) / BK;
  const int iters = (dmax + 1) * nj;
  // pipeline waits give up after this many cycles (short in the diagnostic)
  const long long limit = stall_cycles > 0 ? stall_cycles : kWaitCycles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    mbar_init(stallbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued = 0;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int it = 0; it < iters; ++it) {
      const int s = it % STAGES;
      const uint32_t round = static_cast<uint32_t>(it / STAGES);
      if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1, limit)) {
        ok = false;
        break;
      }
      const int d = it / nj, j0 = (it % nj) * BK;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_3d(&tmA, &full[s], smA + s * A_BYTES, j0, i0, d);
      tma_load_3d(&tmX, &full[s], smB + s * B_BYTES, j0, m0 - d, b);
      issued = it + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer (in the diagnostic it first waits on a barrier nobody arrives on)
    if (stall_cycles > 0 && !mbar_wait(stallbar, 0, limit)) ok = false;
    for (int it = 0; it < iters && ok; ++it) {
      const int s = it % STAGES;
      const uint32_t round = static_cast<uint32_t>(it / STAGES);
      if (!mbar_wait(&full[s], round & 1, limit)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint64_t da = smem_desc(smA + s * A_BYTES);
      const uint64_t db = smem_desc(smB + s * B_BYTES);
      for (int k = 0; k < BK / 16; ++k)
        umma_bf16(tmem, da + (uint64_t)((k * 32) >> 4), db + (uint64_t)((k * 32) >> 4), (it > 0 || k > 0) ? 1u : 0u,
                  TT::idesc);
      umma_commit(&empty[s]);
    }
    umma_commit(accum);   // completes when every MMA issued above has completed
  }
  __syncwarp();
  // on any failure, let the loads already issued land before going on
  if (__syncthreads_or(!ok) && warp == 0 && lane == 0) drain_loads(full, issued);

  // epilogue: warp w holds accumulator rows (TMEM lanes) 32 w .. 32 w + 31
  // (this wait keeps the full limit: TMEM is released only after the MMAs)
  bool acc_ok = mbar_wait(accum, 0);
  acc_ok = __all_sync(0xffffffffu, acc_ok);
  tc_fence_after();
  if (acc_ok) {
    const int gi = i0 + warp * 32 + lane;
    const uint32_t trow = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(trow + c0, r);
      if (gi < nx) {
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int m = m0 + c0 + t;
          if (m < nt) {
            double* yp = Y + ((size_t)b * nt + m) * nx + gi;
            const double v = (double)__uint_as_float(r[t]);
            *yp = accumulate ? *yp + v : v;
          }
        }
      }
    }
  }
  if (!ok || !acc_ok) atomicExch(&g_tc_error, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// three 8-column TMEM loads, then one wait
__device__ __forceinline__ void tmem_ld8x3(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t (&r)[8],
                                           uint32_t (&h)[8], uint32_t (&l)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%24];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%25];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%26];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]), "=r"(h[7]),
        "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]), "=r"(l[7])
      : "r"(a0), "r"(a1), "r"(a2)
      : "memory");
}

// two 8-column TMEM stores, then a wait for their completion
__device__ __forceinline__ void tmem_st8x2(uint32_t a0, uint32_t a1, const uint32_t (&h)[8], const uint32_t (&l)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%10, %11, %12, %13, %14, %15, %16, %17};\n\t"
      "tcgen05.wait::st.sync.aligned;" ::"r"(a0),
      "r"(a1), "r"(h[0]), "r"(h[1]), "r"(h[2]), "r"(h[3]), "r"(h[4]), "r"(h[5]), "r"(h[6]), "r"(h[7]), "r"(l[0]),
      "r"(l[1]), "r"(l[2]), "r"(l[3]), "r"(l[4]), "r"(l[5]), "r"(l[6]), "r"(l[7])
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Same product with compensated accumulation.  A long FP32 accumulation chain
// (all lags x all 64-wide K steps of one output tile: up to 4 n_t n_x / 64 MMA
// roundings) loses accuracy in proportion to its length, which limits the
// refinement residual of the batched solve.  Here the MMA issuer restarts the
// accumulator every `chunk` K steps, alternating between two 128-column TMEM
// buffers, and sixteen epilogue warps drain each finished chunk into a Kahan
// (FP32 sum + FP32 compensation) pair per output while the next chunk is being
// multiplied.  The per-output error is then about (4 chunk + 2) u |partial
// sums| instead of 4 n_lags n_x / 64 u, u = 2^-24.
//   warp 0: TMA producer, warp 1: MMA issuer (and TMEM owner),
//   warps 2..17: epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31 and
//   columns 32 ((w - 2) / 4) .. + 31, so that its Kahan pairs (64 floats)
//   stay in registers.
constexpr int COMP_THREADS = 576;
constexpr int COMP_EPI_WARPS = 16;
constexpr uint32_t COMP_TMEM_COLS = 256;
constexpr size_t COMP_SMEM_BYTES = 1024 + STAGES * (size_t)STAGE_BYTES + 512;

__global__ void __launch_bounds__(COMP_THREADS, 1)
    k_apply_tc_comp(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, int nt, int nx,
                    int chunk, int accumulate, int n_lchunks, int lag_chunk, double* __restrict__ Y) {
  // grid (row tiles, right-hand sides, step tiles x lag chunks), step tiles
  // longest first; with n_lchunks > 1 the CTA takes the lags
  // [c lag_chunk, (c + 1) lag_chunk) of its tile and writes (or adds) its
  // partial product to Y + c n_rhs n_t n_x (summed by k_exact_reduce)
  const int zt = blockIdx.z / n_lchunks, lchunk = blockIdx.z % n_lchunks;
  const int m0 = ((int)(gridDim.z / n_lchunks) - 1 - zt) * BN;
  const int dmax = min(m0 + BN - 1, nt - 1);
  const int d_lo = n_lchunks > 1 ? lchunk * lag_chunk : 0;
  if (d_lo > dmax) return;                       // a chunk past the tile's last lag: nothing to do
  const int d_hi = n_lchunks > 1 ? min(d_lo + lag_chunk, dmax + 1) : dmax + 1;
  Y += (size_t)lchunk * gridDim.y * nt * nx;
  extern __shared__ unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023);
  unsigned char* smA = reinterpret_cast<unsigned char*>(base);
  unsigned char* smB = smA + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;   // [2]: chunk in buffer k complete
  uint64_t* acc_empty = acc_full + 2;    // [2]: buffer k drained by the epilogue
  uint64_t* done = acc_empty + 2;        // every MMA issued by warp 1 complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * BM, b = blockIdx.y;
  const int nj = (nx + BK - 1) / BK;
  const int iters = (d_hi - d_lo) * nj;
  const int nchunks = (iters + chunk - 1) / chunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&acc_full[k], 1);
      mbar_init(&acc_empty[k], COMP_EPI_WARPS);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, COMP_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      for (int it = 0; it < iters; ++it) {
        const int s = it % STAGES;
        const uint32_t round = static_cast<uint32_t>(it / STAGES);
        if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1)) {
          ok = false;
          break;
        }
        const int d = d_lo + it / nj, j0 = (it % nj) * BK;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_3d(&tmA, &full[s], smA + s * A_BYTES, j0, i0, d);
        tma_load_3d(&tmX, &full[s], smB + s * B_BYTES, j0, m0 - d, b);
        issued = it + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int buf = c & 1;
        if (c >= 2 && !mbar_wait(&acc_empty[buf], ((c >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + static_cast<uint32_t>(buf * BN);
        const int it_end = min(iters, (c + 1) * chunk);
        for (int first = 1; it < it_end; ++it, first = 0) {
          const int s = it % STAGES;
          const uint32_t round = static_cast<uint32_t>(it / STAGES);
          if (!mbar_wait(&full[s], round & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t da = smem_desc(smA + s * A_BYTES);
          const uint64_t db = smem_desc(smB + s * B_BYTES);
          for (int k = 0; k < BK / 16; ++k)
            umma_bf16(acc, da + (uint64_t)((k * 32) >> 4), db + (uint64_t)((k * 32) >> 4),
                      (first && k == 0) ? 0u : 1u);
          umma_commit(&empty[s]);
        }
        if (ok) umma_commit(&acc_full[buf]);
      }
      umma_commit(done);
      if (!mbar_wait(done, 0)) ok = false;
    }
    __syncwarp();
  } else {
    // epilogue: Kahan sums of the chunk partials, 32 outputs per thread
    const int q = warp & 3, cq = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    float sum[32], comp[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      sum[t] = 0.f;
      comp[t] = 0.f;
    }
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      // after a failed wait the remaining chunks are skipped without waiting
      const bool got = __all_sync(0xffffffffu, ok && mbar_wait(&acc_full[buf], (c >> 1) & 1));
      if (!got) ok = false;
      if (!ok) continue;
      tc_fence_after();
      const uint32_t taddr = tmem + lane_base + static_cast<uint32_t>(buf * BN + cq * 32);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t r[8];
        tmem_ld8(taddr + g * 8, r);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const float y = __uint_as_float(r[t]) - comp[g * 8 + t];
          const float s2 = sum[g * 8 + t] + y;
          comp[g * 8 + t] = (s2 - sum[g * 8 + t]) - y;
          sum[g * 8 + t] = s2;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    if (ok) {
      const int gi = i0 + q * 32 + lane;
      const int mb = m0 + cq * 32;
      if (gi < nx) {
        double* yp = Y + ((size_t)b * nt + mb) * nx + gi;
        const int tn = nt - mb;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          if (t < tn) {
            const double v = (double)sum[t] - (double)comp[t];
            yp[(size_t)t * nx] = accumulate ? yp[(size_t)t * nx] + v : v;
          }
        }
      }
    }
  }
  if (!ok) atomicExch(&g_tc_error, 1);
  // on any failure, let the loads already issued land before exiting
  if (__syncthreads_or(!ok) && warp == 0 && lane == 0) drain_loads(full, issued);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, COMP_TMEM_COLS);
  }
}

// ---- exact-slice product (FP64-grade accuracy on the BF16 tensor cores) --------
// A and x are split into S integer slices of kSliceBits bits each, with a
// power-of-two scale per row of A (lag d, row i: 2^{eA[d][i]}) and per row of
// x (right-hand side b, step n: 2^{eX[b][n]}):
//   A[d][i][j]  = sum_s a_s[d][i][j] 2^{eA[d][i] - 6 (s + 1)},  |a_0| <= 64, |a_s| <= 32,
//   x[b][n][j]  = sum_t x_t[b][n][j] 2^{eX[b][n] - 6 (t + 1)},
// so that a slice pair (s, t) contributes at 2^{eA + eX - 6 (s + t + 2)}.  The
// slice products are exact (12-bit integers), and a sum over at most 1024
// columns of the up to S <= 8 pairs with the same s + t stays below
// 1024 (4096 + 1024 (S - 2)) <= 10 2^20 < 2^24, so the FP32 tensor-core
// accumulator holds every partial sum exactly, whatever its internal rounding.
// The accumulator therefore restarts for every group (lag d, k = s + t, block
// of 1024 columns); each finished exact group is scaled by its power of two
// and added into a double-float (FP32 sum + FP32 error by Knuth's two-sum) per
// output y[b][m][i], relative to 2^{max_d eA[d][i] + max_{n <= m} eX[b][n]}
// (an upper bound of every contribution's scale; output steps with only small
// x keep their own small scale).  Pairs with s + t >= S are dropped.  The
// error is relative to the row scales, at most 2^{-6S} (1 + S / 4) n_x
// sum_d 2^{eA[d][i] + eX[b][m-d]} (S = 7: a few 1e-12 of that sum).
//   warp 0: TMA producer, warp 1: MMA issuer (TMEM owner), warps 2..17: the
//   epilogue; warp w owns TMEM lanes 32 (w % 4) .. + 31 and columns
//   32 ((w - 2) / 4) .. + 31 of the tile.  The double-float sums live in TMEM
//   too (columns 256.. and 384..), next to the two accumulator buffers
//   (0.., 128..), so that the epilogue holds no per-output arrays.
constexpr int kSliceBits = 6;
constexpr int kExactJSteps = 16;                 // 64-wide K steps per group: 1024 columns
constexpr int kZeroRowExp = -16384;              // scale of an all-zero row
constexpr int EX_THREADS = 576;
constexpr int EX_EPI_WARPS = 16;
constexpr uint32_t EX_TMEM_COLS = 512;
constexpr uint32_t EX_HI_COL = 256, EX_LO_COL = 384;
constexpr int EX_STAGES = 6;                     // 192 KB of operands in flight
constexpr int kExactMaxSteps = 4096;             // eX of one right-hand side staged in shared memory
constexpr size_t EX_SMEM_BYTES =
    1024 + EX_STAGES * (size_t)STAGE_BYTES + 512 + 2 * kExactMaxSteps * sizeof(short);

__device__ __forceinline__ void tma_load_4d(const CUtensorMap* map, uint64_t* bar, void* dst, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

// 2^e as a float for e <= 0 (0 below the subnormal range)
__device__ __forceinline__ float pow2f(int e) {
  if (e < -149) return 0.0f;
  if (e < -126) return __int_as_float(1 << (e + 149));
  return __int_as_float((e + 127) << 23);
}

template <int S>
__global__ void __launch_bounds__(EX_THREADS, 1)
    k_apply_tc_exact(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                     const int* __restrict__ eA, const int* __restrict__ eX, int nt, int nx, int n_chunks,
                     int lag_chunk, double* __restrict__ Y) {
  // grid (row tiles, right-hand sides, step tiles x lag chunks): the step
  // tiles run in decreasing order of m0, so the longest tiles (most lags)
  // start first and the short ones fill the tail; with n_chunks > 1 the CTA
  // takes the lags [c lag_chunk, (c + 1) lag_chunk) of its tile and writes
  // its partial products to Y + c n_rhs n_t n_x (summed by k_exact_reduce)
  const int zt = blockIdx.z / n_chunks, chunk = blockIdx.z % n_chunks;
  const int m0 = ((int)(gridDim.z / n_chunks) - 1 - zt) * BN;
  const int dmax = min(m0 + BN - 1, nt - 1);
  const int d_lo = n_chunks > 1 ? chunk * lag_chunk : 0;
  if (d_lo > dmax) return;                       // a chunk past the tile's last lag: nothing to do
  const int d_hi = n_chunks > 1 ? min(d_lo + lag_chunk, dmax + 1) : dmax + 1;
  Y += (size_t)chunk * gridDim.y * nt * nx;
  extern __shared__ unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023);
  unsigned char* smA = reinterpret_cast<unsigned char*>(base);
  unsigned char* smB = smA + EX_STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smB + EX_STAGES * B_BYTES);
  uint64_t* empty = full + EX_STAGES;
  uint64_t* acc_full = empty + EX_STAGES;   // [2]: group in buffer k complete
  uint64_t* acc_empty = acc_full + 2;    // [2]: buffer k drained by the epilogue
  uint64_t* done = acc_empty + 2;        // every MMA issued by warp 1 complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  // this b's step scales and their prefix maxima (16-bit: -16384 .. 1025)
  short* eXs = reinterpret_cast<short*>(reinterpret_cast<unsigned char*>(full) + 512);
  short* eXp = eXs + kExactMaxSteps;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * BM, b = blockIdx.y;
  const int nj = (nx + BK - 1) / BK;
  const int nb = (nj + kExactJSteps - 1) / kExactJSteps;
  const int ngroups = (d_hi - d_lo) * S * nb;    // (d, k, jb), jb fastest

  if (threadIdx.x == 0) {
    for (int s = 0; s < EX_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&acc_full[k], 1);
      mbar_init(&acc_empty[k], EX_EPI_WARPS);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {   // step scales and their running maximum (a warp scan per 32 steps)
    int carry = kZeroRowExp;
    for (int c0 = 0; c0 < nt; c0 += 32) {
      const int n = c0 + lane;
      const int v = n < nt ? eX[(size_t)b * nt + n] : kZeroRowExp;
      int pm = v;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, pm, off);
        if (lane >= off) pm = max(pm, u);
      }
      pm = max(pm, carry);
      if (n < nt) {
        eXs[n] = static_cast<short>(v);
        eXp[n] = static_cast<short>(pm);
      }
      carry = __shfl_sync(0xffffffffu, pm, 31);
    }
  }
  if (warp == 1) tmem_alloc(tmem_slot, EX_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  int issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int g = 0; g < ngroups && ok; ++g) {
        const int d = d_lo + g / (S * nb), k = (g / nb) % S, jb = g % nb;
        const int j_lo = jb * kExactJSteps, j_hi = min(nj, j_lo + kExactJSteps);
        for (int s = 0; s <= k && ok; ++s)
          for (int jc = j_lo; jc < j_hi; ++jc, ++it) {
            const int st = it % EX_STAGES;
            const uint32_t round = static_cast<uint32_t>(it / EX_STAGES);
            if (round > 0 && !mbar_wait(&empty[st], (round - 1) & 1)) {
              ok = false;
              break;
            }
            mbar_expect_tx(&full[st], STAGE_BYTES);
            tma_load_4d(&tmA, &full[st], smA + st * A_BYTES, jc * BK, i0, d, s);
            tma_load_4d(&tmX, &full[st], smB + st * B_BYTES, jc * BK, m0 - d, b, k - s);
            issued = it + 1;
          }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0;
      for (int g = 0; g < ngroups && ok; ++g) {
        const int buf = g & 1, k = (g / nb) % S, jb = g % nb;
        const int nsteps = (k + 1) * (min(nj, (jb + 1) * kExactJSteps) - jb * kExactJSteps);
        if (g >= 2 && !mbar_wait(&acc_empty[buf], ((g >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + static_cast<uint32_t>(buf * BN);
        const int it_end = it + nsteps;
        for (int first = 1; it < it_end; ++it, first = 0) {
          const int st = it % EX_STAGES;
          const uint32_t round = static_cast<uint32_t>(it / EX_STAGES);
          if (!mbar_wait(&full[st], round & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t da = smem_desc(smA + st * A_BYTES);
          const uint64_t db = smem_desc(smB + st * B_BYTES);
          for (int kk = 0; kk < BK / 16; ++kk)
            umma_bf16(acc, da + (uint64_t)((kk * 32) >> 4), db + (uint64_t)((kk * 32) >> 4),
                      (first && kk == 0) ? 0u : 1u);
          umma_commit(&empty[st]);
        }
        if (ok) umma_commit(&acc_full[buf]);
      }
      umma_commit(done);
      if (!mbar_wait(done, 0)) ok = false;
    }
    __syncwarp();
  } else {
    // epilogue: row i = i0 + 32 q + lane, columns m = m0 + 32 cq + t
    const int q = warp & 3, cq = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    const int i = i0 + q * 32 + lane;
    const int mb = m0 + cq * 32;
    // reference scale of y[b][m][i]: 2^{eAmax + eXp[m]}, eAmax the row's
    // largest over the CTA's lags (rows i >= n_x and steps outside
    // 0..n_t - 1 were zero-filled by the loads, so their partials are 0: the
    // clamped indexes give them finite scales)
    const int ic = min(i, nx - 1);
    int eAmax = kZeroRowExp;
    for (int d = d_lo; d < d_hi; ++d) eAmax = max(eAmax, eA[(size_t)d * nx + ic]);
    const uint32_t tcol = tmem + lane_base + static_cast<uint32_t>(cq * 32);
    int er = 0;
    for (int g = 0; g < ngroups; ++g) {
      const int buf = g & 1, d = d_lo + g / (S * nb), k = (g / nb) % S;
      if (g % (S * nb) == 0) er = eA[(size_t)d * nx + ic] - eAmax;
      // after a failed wait the remaining groups are skipped without waiting
      const bool got = __all_sync(0xffffffffu, ok && mbar_wait(&acc_full[buf], (g >> 1) & 1));
      if (!got) ok = false;
      if (!ok) continue;
      tc_fence_after();
      const int ek = -kSliceBits * (k + 2);
#pragma unroll 1
      for (int gg = 0; gg < 4; ++gg) {
        uint32_t r[8], h[8], l[8];
        const uint32_t c0 = static_cast<uint32_t>(gg * 8);
        if (g == 0) {
          tmem_ld8(tcol + buf * BN + c0, r);
#pragma unroll
          for (int t = 0; t < 8; ++t) h[t] = l[t] = 0u;
        } else {
          tmem_ld8x3(tcol + buf * BN + c0, tcol + EX_HI_COL + c0, tcol + EX_LO_COL + c0, r, h, l);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int mc = min(mb + gg * 8 + t, nt - 1), n = min(max(mb + gg * 8 + t - d, 0), nt - 1);
          const float v = __uint_as_float(r[t]) * pow2f(er + ek + eXs[n] - eXp[mc]);   // exact power-of-two scaling
          const float hv = __uint_as_float(h[t]);
          const float sm = hv + v;
          const float bp = sm - hv;
          h[t] = __float_as_uint(sm);
          l[t] = __float_as_uint(__uint_as_float(l[t]) + ((hv - (sm - bp)) + (v - bp)));
        }
        tmem_st8x2(tcol + EX_HI_COL + c0, tcol + EX_LO_COL + c0, h, l);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    if (ok) {   // warp-uniform: the TMEM loads are .sync.aligned
#pragma unroll 1
      for (int gg = 0; gg < 4; ++gg) {
        uint32_t h[8], l[8];
        tmem_ld8(tcol + EX_HI_COL + gg * 8, h);
        tmem_ld8(tcol + EX_LO_COL + gg * 8, l);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int m = mb + gg * 8 + t;
          if (i < nx && m < nt)
            Y[((size_t)b * nt + m) * nx + i] =
                ldexp((double)__uint_as_float(h[t]) + (double)__uint_as_float(l[t]), eAmax + eXp[m]);
        }
      }
    }
  }
  if (!ok) atomicExch(&g_tc_error, 1);
  // on any failure, let the loads already issued land before exiting
  if (__syncthreads_or(!ok) && warp == 0 && lane == 0) drain_loads(full, issued, EX_STAGES);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, EX_TMEM_COLS);
  }
}

// Integer slices of the rows of an FP64 matrix (rows x cols, row-major): per
// row e = the exponent with max |row| < 2^e (kZeroRowExp for a zero row), then
// R = row 2^{-e} and, S times, q = rint(R 2^6) (the slice), R = R 2^6 - q (exact
// steps: scaling by powers of two, an integer and a remainder below 1/2).
// One warp per row.
__global__ void k_exact_slices(const double* __restrict__ src, long long rows, int cols, int S,
                               __nv_bfloat16* __restrict__ out, int* __restrict__ rexp) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const double* row = src + w * (long long)cols;
  double mx = 0.0;
  for (int j = lane; j < cols; j += 32) mx = fmax(mx, fabs(row[j]));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  int e = kZeroRowExp;
  if (mx > 0.0) {
    int ex;
    frexp(mx, &ex);          // mx = f 2^ex, f in [1/2, 1): mx < 2^ex
    e = ex;
  }
  if (lane == 0) rexp[w] = e;
  const size_t plane = (size_t)rows * cols;
  for (int j = lane; j < cols; j += 32) {
    double R = ldexp(row[j], -e);
    for (int s = 0; s < S; ++s) {
      const double qv = rint(R * 64.0);
      out[(size_t)s * plane + w * (long long)cols + j] = __double2bfloat16(qv);
      R = R * 64.0 - qv;
    }
  }
}

__global__ void k_to_bf16_f64(const double* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = __double2bfloat16(src[e]);
}
__global__ void k_to_bf16_f32(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = __float2bfloat16(src[e]);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

bool apply_tc_supported(int nt, int nx, int n_rhs) {
  return nt >= 1 && nx >= 8 && nx % 8 == 0 && n_rhs >= 1 && n_rhs <= 65535 && (nt + BN - 1) / BN <= 65535;
}

namespace {
cudaError_t make_maps(int nt, int nx, const void* A_bf16, int n_rhs, const void* X_bf16, CUtensorMap* mA,
                      CUtensorMap* mX, int bn) {
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dimA[3] = {(cuuint64_t)nx, (cuuint64_t)nx, (cuuint64_t)nt};
  const cuuint64_t strA[2] = {(cuuint64_t)nx * 2, (cuuint64_t)nx * nx * 2};
  const cuuint64_t dimX[3] = {(cuuint64_t)nx, (cuuint64_t)nt, (cuuint64_t)n_rhs};
  const cuuint64_t strX[2] = {(cuuint64_t)nx * 2, (cuuint64_t)nt * nx * 2};
  const cuuint32_t boxA[3] = {BK, BM, 1}, boxX[3] = {BK, (cuuint32_t)bn, 1}, es[3] = {1, 1, 1};
  CUresult r = enc(mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(A_bf16), dimA, strA, boxA, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  r = enc(mX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(X_bf16), dimX, strX, boxX, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  return cudaSuccess;
}
}  // namespace

static std::atomic<long long> g_stall_cycles{0};

void tc_set_stall(long long cycles) { g_stall_cycles.store(cycles > 0 ? cycles : 0); }

std::string tc_plain_tune_key(int nt, int nx, int n_rhs) {
  int dev = 0;
  cudaGetDevice(&dev);
  return tune_device_key(dev) + "|tc_plain|nt=" + std::to_string(nt) + "|nx=" + std::to_string(nx) +
         "|rhs=" + std::to_string(n_rhs);
}

int tc_plain_tile_n(int nt, int nx, int n_rhs) {
  std::string v;
  if (tune_cache_get(tc_plain_tune_key(nt, nx, n_rhs), &v)) {
    if (v == "bn=128") return 128;
    if (v == "bn=256" && nt > 128) return 256;
  }
  // untuned: products on more than 128 steps take 128 x 256 tiles (N = 256
  // MMAs, a third less shared-memory operand traffic per flop)
  return nt > 128 ? 256 : BN;
}

cudaError_t apply_tc_launch(int nt, int nx, const void* A_bf16, int n_rhs, const void* X_bf16, double* Y,
                            bool accumulate, cudaStream_t s, int chunk, int tile_n, double* part) {
  const long long stall = g_stall_cycles.load();
  CUtensorMap mA, mX;
  int bn = BN;
  if (chunk <= 0) bn = (tile_n == 128 || tile_n == 256) ? tile_n : tc_plain_tile_n(nt, nx, n_rhs);
  cudaError_t e = make_maps(nt, nx, A_bf16, n_rhs, X_bf16, &mA, &mX, bn);
  if (e != cudaSuccess) return e;
  const dim3 grid((nx + BM - 1) / BM, n_rhs, (nt + bn - 1) / bn);
  if (chunk <= 0 && bn == 256) {
    e = cudaFuncSetAttribute(k_apply_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcTile<256>::smem_bytes);
    if (e != cudaSuccess) return e;
    k_apply_tc<256><<<grid, THREADS, TcTile<256>::smem_bytes, s>>>(mA, mX, nt, nx, accumulate ? 1 : 0, Y,
                                                                      stall);
  } else if (chunk <= 0) {
    e = cudaFuncSetAttribute(k_apply_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcTile<128>::smem_bytes);
    if (e != cudaSuccess) return e;
    k_apply_tc<128><<<grid, THREADS, TcTile<128>::smem_bytes, s>>>(mA, mX, nt, nx, accumulate ? 1 : 0, Y,
                                                                      stall);
  } else {
    e = cudaFuncSetAttribute(k_apply_tc_comp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)COMP_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    // few output tiles and a partial-sum buffer: lag chunks (tc_chunk_reduce_launch sums them)
    const int nch = part ? exact_lag_chunks(nt, nx, n_rhs) : 1;
    const dim3 gridc(grid.x, grid.y, grid.z * nch);
    k_apply_tc_comp<<<gridc, COMP_THREADS, COMP_SMEM_BYTES, s>>>(mA, mX, nt, nx, chunk, accumulate ? 1 : 0, nch,
                                                                 kExactLagChunk, nch > 1 ? part : Y);
  }
  count_launches(1);
  return cudaGetLastError();
}

bool apply_tc_exact_supported(int nt, int nx, int n_rhs, int n_slices) {
  return apply_tc_supported(nt, nx, n_rhs) && nt <= kExactMaxSteps && n_slices >= kExactMinSlices &&
         n_slices <= kExactMaxSlices;
}

cudaError_t exact_slices_launch(const double* src, long long rows, int cols, int n_slices, void* slices,
                                int* row_exp, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  const int threads = 256;
  const long long blocks = (rows * 32 + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_exact_slices<<<(unsigned)blocks, threads, 0, s>>>(src, rows, cols, n_slices,
                                                     static_cast<__nv_bfloat16*>(slices), row_exp);
  count_launches(1);
  return cudaGetLastError();
}

namespace {
template <int S>
cudaError_t launch_exact_s(const CUtensorMap& mA, const CUtensorMap& mX, dim3 grid, const int* eA, const int* eX,
                           int nt, int nx, int n_chunks, int lag_chunk, double* Y, cudaStream_t s) {
  cudaError_t e =
      cudaFuncSetAttribute(k_apply_tc_exact<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EX_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  k_apply_tc_exact<S><<<grid, EX_THREADS, EX_SMEM_BYTES, s>>>(mA, mX, eA, eX, nt, nx, n_chunks, lag_chunk, Y);
  return cudaSuccess;
}

// y = the sum, in chunk order, of the lag-chunk partials written for y's step
// tile (chunk c exists for the tile when c lag_chunk <= its last lag)
__global__ void k_exact_reduce(int nt, int nx, int n_rhs, int n_chunks, int lag_chunk,
                               const double* __restrict__ part, double* __restrict__ Y) {
  const size_t total = (size_t)n_rhs * nt * nx;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)((e / nx) % nt);
    const int dmax = min((m / BN) * BN + BN - 1, nt - 1);
    const int nc = min(n_chunks, dmax / lag_chunk + 1);
    double acc = 0.0;
    for (int c = 0; c < nc; ++c) acc += part[(size_t)c * total + e];
    Y[e] = acc;
  }
}
}  // namespace

int exact_lag_chunks(int nt, int nx, int n_rhs) {
  // products whose output tiles leave the GPU short of two CTAs per SM split
  // each tile's lags into chunks of kExactLagChunk
  const long long tiles = (long long)((nx + BM - 1) / BM) * n_rhs * ((nt + BN - 1) / BN);
  if (tiles >= 2LL * sm_count()) return 1;
  return (nt + kExactLagChunk - 1) / kExactLagChunk;
}

size_t exact_part_bytes(int nt, int nx, int n_rhs) {
  const int c = exact_lag_chunks(nt, nx, n_rhs);
  return c > 1 ? (size_t)c * n_rhs * nt * nx * sizeof(double) : 0;
}

cudaError_t apply_tc_exact_launch(int nt, int nx, int n_slices, const void* A_slices, const int* A_exp, int n_rhs,
                                  const void* X_slices, const int* X_exp, double* Y, cudaStream_t s, double* part) {
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // A slices [S][nt][nx][nx] and x slices [S][n_rhs][nt][nx], BF16, as 4-D maps
  CUtensorMap mA, mX;
  const cuuint64_t dimA[4] = {(cuuint64_t)nx, (cuuint64_t)nx, (cuuint64_t)nt, (cuuint64_t)n_slices};
  const cuuint64_t strA[3] = {(cuuint64_t)nx * 2, (cuuint64_t)nx * nx * 2, (cuuint64_t)nt * nx * nx * 2};
  const cuuint64_t dimX[4] = {(cuuint64_t)nx, (cuuint64_t)nt, (cuuint64_t)n_rhs, (cuuint64_t)n_slices};
  const cuuint64_t strX[3] = {(cuuint64_t)nx * 2, (cuuint64_t)nt * nx * 2, (cuuint64_t)n_rhs * nt * nx * 2};
  const cuuint32_t boxA[4] = {BK, BM, 1, 1}, boxX[4] = {BK, BN, 1, 1}, es[4] = {1, 1, 1, 1};
  CUresult r = enc(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(A_slices), dimA, strA, boxA, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  r = enc(&mX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(X_slices), dimX, strX, boxX, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int nch = part ? exact_lag_chunks(nt, nx, n_rhs) : 1;
  const int lc = nch > 1 ? kExactLagChunk : 0;
  double* out = nch > 1 ? part : Y;
  const dim3 grid((nx + BM - 1) / BM, n_rhs, ((nt + BN - 1) / BN) * nch);
  cudaError_t e = cudaErrorInvalidValue;
  switch (n_slices) {
    case 4: e = launch_exact_s<4>(mA, mX, grid, A_exp, X_exp, nt, nx, nch, lc, out, s); break;
    case 5: e = launch_exact_s<5>(mA, mX, grid, A_exp, X_exp, nt, nx, nch, lc, out, s); break;
    case 6: e = launch_exact_s<6>(mA, mX, grid, A_exp, X_exp, nt, nx, nch, lc, out, s); break;
    case 7: e = launch_exact_s<7>(mA, mX, grid, A_exp, X_exp, nt, nx, nch, lc, out, s); break;
    case 8: e = launch_exact_s<8>(mA, mX, grid, A_exp, X_exp, nt, nx, nch, lc, out, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess || nch == 1) return e;
  const size_t total = (size_t)n_rhs * nt * nx;
  k_exact_reduce<<<stride_grid(total, 256, 16), 256, 0, s>>>(nt, nx, n_rhs, nch, kExactLagChunk, part, Y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t tc_chunk_reduce_launch(int nt, int nx, int n_rhs, const double* part, double* Y, cudaStream_t s) {
  const int nch = exact_lag_chunks(nt, nx, n_rhs);
  if (nch == 1) return cudaSuccess;
  const size_t total = (size_t)n_rhs * nt * nx;
  k_exact_reduce<<<stride_grid(total, 256, 16), 256, 0, s>>>(nt, nx, n_rhs, nch, kExactLagChunk, part, Y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t tc_error_reset(cudaStream_t s) {
  const int zero = 0;
  return cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
}

cudaError_t tc_error_read(int* flag, cudaStream_t s) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(flag, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

// Three-term BF16 split of an FP64 array: hi = bf16(x), mid = bf16(x - hi),
// lo = bf16(x - hi - mid), so that x - (hi + mid + lo) is ~2^-24 |x|.
__global__ void k_bf16_split3(const double* __restrict__ src, __nv_bfloat16* __restrict__ hi,
                              __nv_bfloat16* __restrict__ mid, __nv_bfloat16* __restrict__ lo, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double x = src[e];
    const __nv_bfloat16 h = __double2bfloat16(x);
    const double r1 = x - (double)__bfloat162float(h);
    const __nv_bfloat16 m = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(m);
    hi[e] = h;
    if (mid) mid[e] = m;
    if (lo) lo[e] = __double2bfloat16(r2);
  }
}

cudaError_t bf16_split3_launch(const double* src, void* hi, void* mid, void* lo, size_t n, cudaStream_t s) {
  const int blocks = stride_grid(n, 256, 16);
  k_bf16_split3<<<blocks, 256, 0, s>>>(src, static_cast<__nv_bfloat16*>(hi), static_cast<__nv_bfloat16*>(mid),
                                        static_cast<__nv_bfloat16*>(lo), n);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t to_bf16_launch(int src_prec, const void* src, void* dst, size_t n, cudaStream_t s) {
  const int blocks = stride_grid(n, 256, 16);
  if (src_prec == STBEM_F64)
    k_to_bf16_f64<<<blocks, 256, 0, s>>>(static_cast<const double*>(src), static_cast<__nv_bfloat16*>(dst), n);
  else
    k_to_bf16_f32<<<blocks, 256, 0, s>>>(static_cast<const float*>(src), static_cast<__nv_bfloat16*>(dst), n);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace stbem
