// Block-lower-triangular block-Toeplitz products (Section 3 block structure,
// uniform time grid => block (m, n) = A^(m-n)).
//
//   y[b][m][i] = sum_{d=0}^{m} sum_j A[d][i][j] x[b][m-d][j]              (forward)
//   y[b][n][j] = sum_{d=0}^{nt-1-n} sum_i A[d][i][j] x[b][n+d][i]          (transpose)
//
// The transpose runs backward in time; with reversed time m' = nt-1-n it has
// the forward structure with A^(d) transposed, which is how it is computed.
//
// Work split: a CTA owns an output tile (TM time steps x TI rows) of one
// right-hand side and one chunk of lags; the (lag, column) reduction runs
// through shared-memory tiles of A^(d) and of the shifted x.  Lag chunks write
// partial tiles to the caller's workspace and a second kernel sums them in
// chunk order, so results do not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "assemble.h"
#include "device_info.h"
#include "toeplitz.h"

namespace stbem {

constexpr int TI = 64, TM = 32, TJ = 16, kApplyThreads = 256;
// FP32 register-tiled product: 128 rows x 128 steps per CTA (single
// problems), 128 x 64 (ragged batches of smaller problems), 16 columns per stage
constexpr int TI4 = 128, TM4 = 128, TM4R = 64, TJ4 = 16;

struct ApplyPlan {
  int MT, IT, CH, DC;
};

// Plan of a product over the nlag lags of a range (nlag = nt: all of them).
static ApplyPlan make_plan(int nt, int nx, int tm = TM, int ti = TI, int nlag = -1) {
  if (nlag < 0) nlag = nt;
  if (nlag < 1) nlag = 1;
  ApplyPlan p;
  p.MT = (nt + tm - 1) / tm;
  p.IT = (nx + ti - 1) / ti;
  // aim at ~4 waves of (tile, chunk) units over the device's SMs
  const long long target = 4LL * sm_count();
  long long per_chunk = (long long)p.IT * ((p.MT + 1) / 2);
  if (per_chunk < 1) per_chunk = 1;
  int ch = (int)((target + per_chunk - 1) / per_chunk);
  if (ch < 1) ch = 1;
  if (ch > nlag) ch = nlag;
  p.DC = (nlag + ch - 1) / ch;
  p.CH = (nlag + p.DC - 1) / p.DC;
  return p;
}

// FP32 forward products use the register-tiled kernel (128 x 128 tiles) when
// rows are 16-byte aligned and its causal tiles alone fill one wave of one
// CTA per SM (lag chunks multiply them further); smaller products keep the
// 64 x 32 tiles, which need fewer lag chunks (and partial sums) for the same
// parallelism.
static bool use_apply32(int nx) { return nx % 4 == 0; }
static bool use_apply32(int nt, int nx, int n_rhs) {
  const long long it = (nx + TI4 - 1) / TI4, mt = (nt + TM4 - 1) / TM4;
  return use_apply32(nx) && (long long)n_rhs * it * mt * (mt + 1) / 2 >= (long long)sm_count();
}

size_t apply_range_workspace_bytes(int nt, int nx, int nlag, int n_rhs) {
  const ApplyPlan p = make_plan(nt, nx, TM, TI, nlag);
  size_t b = (size_t)n_rhs * p.MT * p.CH * TM * (size_t)nx * sizeof(double);
  if (use_apply32(nt, nx, n_rhs)) {
    const ApplyPlan q = make_plan(nt, nx, TM4, TI4, nlag);
    b = std::max(b, (size_t)n_rhs * q.MT * q.CH * TM4 * (size_t)nx * sizeof(double));
  }
  return b;
}

size_t apply_workspace_bytes(int nt, int nx, int n_rhs) { return apply_range_workspace_bytes(nt, nx, nt, n_rhs); }

// One (row tile it, lag chunk ch, right-hand side b, time tile mt) unit over
// the lags [lag_lo, lag_hi); A points at the block of lag lag_lo.
template <typename TA, typename TC, bool TRANS>
__device__ __forceinline__ void apply_body(int nt, int nx, int MT, int CH, int DC, int lag_lo, int lag_hi,
                                           const TA* __restrict__ A, const double* __restrict__ x,
                                           double* __restrict__ part, int it, int ch, int b, int mt,
                                           TC (*As)[TI + 1], TC (*Xs)[TM + 1]) {
  const int m0 = mt * TM, i0 = it * TI;
  const int mmax = min(m0 + TM, nt) - 1;        // largest m in the tile
  const int d0 = lag_lo + ch * DC;
  if (d0 > mmax || d0 >= lag_hi) return;
  const int d1 = min(min(d0 + DC, mmax + 1), lag_hi);
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;        // rows tx*4.., time ty*2..
  const double* xb = x + (size_t)b * nt * nx;
  // FP32 products are summed in FP32 over one lag block's columns only and
  // flushed into FP64 after every lag, so no FP32 chain is longer than N_x
  TC acc[2][4];
  double acc64[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[a][c] = (TC)0;
      acc64[a][c] = 0.0;
    }

  for (int d = d0; d < d1; ++d) {
    const TA* Ad = A + (size_t)(d - lag_lo) * nx * nx;
    for (int j0 = 0; j0 < nx; j0 += TJ) {
      // A tile: element (row i0+ii, column j0+jj)
#pragma unroll
      for (int q = 0; q < (TI * TJ) / kApplyThreads; ++q) {
        const int e = tid + q * kApplyThreads;
        int ii, jj;
        if (!TRANS) { jj = e % TJ; ii = e / TJ; } else { ii = e % TI; jj = e / TI; }
        const int gi = i0 + ii, gj = j0 + jj;
        TC v = (TC)0;
        if (gi < nx && gj < nx) v = (TC)(!TRANS ? Ad[(size_t)gi * nx + gj] : Ad[(size_t)gj * nx + gi]);
        As[jj][ii] = v;
      }
      // x tile: element (column j0+jj, time m0+mm) = x[m - d][j]
#pragma unroll
      for (int q = 0; q < (TM * TJ) / kApplyThreads; ++q) {
        const int e = tid + q * kApplyThreads;
        const int jj = e % TJ, mm = e / TJ;
        const int m = m0 + mm, gj = j0 + jj;
        TC v = (TC)0;
        if (m <= mmax && m - d >= 0 && gj < nx) {
          const int src = TRANS ? (nt - 1 - (m - d)) : (m - d);
          v = (TC)xb[(size_t)src * nx + gj];
        }
        Xs[jj][mm] = v;
      }
      __syncthreads();
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj) {
        TC av[4], xv[2];
#pragma unroll
        for (int c = 0; c < 4; ++c) av[c] = As[jj][tx * 4 + c];
#pragma unroll
        for (int a = 0; a < 2; ++a) xv[a] = Xs[jj][ty * 2 + a];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[c], xv[a], acc[a][c]);
      }
      __syncthreads();
    }
    if constexpr (sizeof(TC) == 4) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc64[a][c] += (double)acc[a][c];
          acc[a][c] = (TC)0;
        }
    }
  }
  if constexpr (sizeof(TC) == 8) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc64[a][c] = (double)acc[a][c];
  }
  // partial tile -> part[b][mt][ch][mm][i]
  double* pt = part + ((((size_t)b * MT + mt) * CH + ch) * TM) * nx;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int mm = ty * 2 + a;
    if (m0 + mm > mmax) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gi = i0 + tx * 4 + c;
      if (gi < nx) pt[(size_t)mm * nx + gi] = acc64[a][c];
    }
  }
}

template <typename TA, typename TC, bool TRANS>
__global__ void __launch_bounds__(kApplyThreads)
k_apply(int nt, int nx, int MT, int CH, int DC, int lag_lo, int lag_hi, const TA* __restrict__ A,
        const double* __restrict__ x, double* __restrict__ part) {
  __shared__ TC As[TJ][TI + 1];
  __shared__ TC Xs[TJ][TM + 1];
  apply_body<TA, TC, TRANS>(nt, nx, MT, CH, DC, lag_lo, lag_hi, A, x, part, blockIdx.x, blockIdx.y,
                            blockIdx.z / MT, blockIdx.z % MT, As, Xs);
}

// ---- FP32 forward product, register-tiled ----------------------------------------------
// A CTA of 16 x 16 threads owns 128 rows x 128 time steps (one right-hand
// side, one lag chunk); thread (ty, tx) computes the rows ty*4.. and
// 64 + ty*4.. and the steps tx*4.. and 64 + tx*4.. (split halves keep the
// float4 shared-memory reads conflict-free): 64 FFMA per 4 float4 loads.  Each
// lag's FP32 partial (a chain of N_x terms) is added into a compensated
// (hi, lo) FP32 pair per output (Knuth's two-sum, 6 FP32 operations), so lags
// accumulate without FP32 loss and without FP64 arithmetic, which runs at 1/72
// of the FP32 rate here.  The (hi, lo) pairs live in shared memory
// ([k][thread], conflict-free) and are touched once per lag; the 16-column
// stages of all lags of the chunk form one software pipeline: the next
// stage's A and x are loaded into registers while the current one is
// multiplied from the other half of a double-buffered shared tile (one
// barrier per stage).  Requires N_x % 4 == 0 (16-byte rows).
// dynamic shared memory of a TMV-step tile: two stages of A (16 x 128) and x
// (16 x (TMV + 4): transposing stores 2-way at most), then the (hi, lo) pairs
// (2 x 8 TMV / 16 x 256 floats)
template <int TMV>
constexpr size_t apply32_smem() {
  return (2 * TJ4 * TI4 + 2 * TJ4 * (TMV + 4) + 2 * (8 * TMV / 16) * 256) * sizeof(float);
}
constexpr size_t kApply32Smem = apply32_smem<TM4>();
constexpr size_t kApply32SmemR = apply32_smem<TM4R>();

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (v - bp);
  hi = s;
  lo += err;
}

template <int TMV>
__device__ __forceinline__ void apply32_body(int nt, int nx, int MT, int CH, int DC, int lag_lo, int lag_hi,
                                             const float* __restrict__ A, const double* __restrict__ x,
                                             double* __restrict__ part, int it, int ch, int b, int mt,
                                             float* smem) {
  constexpr int NC = TMV / 16;            // steps per thread: tx*4.. (and 64 + tx*4.. for 128)
  constexpr int kXsLd = TMV + 4;
  const int m0 = mt * TMV, i0 = it * TI4;
  const int mmax = min(m0 + TMV, nt) - 1;
  const int d0 = lag_lo + ch * DC;
  if (d0 > mmax || d0 >= lag_hi) return;
  const int d1 = min(min(d0 + DC, mmax + 1), lag_hi);
  float (*As)[TJ4][TI4] = reinterpret_cast<float (*)[TJ4][TI4]>(smem);                   // [2]
  float (*Xs)[TJ4][kXsLd] = reinterpret_cast<float (*)[TJ4][kXsLd]>(smem + 2 * TJ4 * TI4);  // [2]
  float* H = smem + 2 * TJ4 * TI4 + 2 * TJ4 * kXsLd;                                        // [8 NC][256]
  float* Lo = H + 8 * NC * 256;                                                             // [8 NC][256]
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const double* xb = x + (size_t)b * nt * nx;
#pragma unroll
  for (int k = 0; k < 8 * NC; ++k) {
    H[k * 256 + tid] = 0.f;
    Lo[k * 256 + tid] = 0.f;
  }
  const int nj = (nx + TJ4 - 1) / TJ4;
  const int stages = (d1 - d0) * nj;
  // this thread's loads of one stage: 2 float4 of A, NC values of x (kept in
  // FP64 until the store, so that no conversion waits on a load in flight)
  float4 ra[2];
  double rx[NC];
  auto load = [&](int st) {
    const int d = d0 + st / nj, j0 = (st % nj) * TJ4;
    const float* Ad = A + (size_t)(d - lag_lo) * nx * nx;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + q * 256;
      const int ii = e % TI4, jq = e / TI4;
      const int gi = i0 + ii, gj = j0 + jq * 4;
      ra[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gi < nx && gj < nx) ra[q] = *reinterpret_cast<const float4*>(Ad + (size_t)gi * nx + gj);
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const int e = tid + q * 256;
      const int jj = e % TJ4, mm = e / TJ4;
      const int m = m0 + mm, gj = j0 + jj;
      rx[q] = (m <= mmax && m - d >= 0 && gj < nx) ? xb[(size_t)(m - d) * nx + gj] : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + q * 256;
      const int ii = e % TI4, jq = e / TI4;
      As[buf][jq * 4 + 0][ii] = ra[q].x;
      As[buf][jq * 4 + 1][ii] = ra[q].y;
      As[buf][jq * 4 + 2][ii] = ra[q].z;
      As[buf][jq * 4 + 3][ii] = ra[q].w;
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const int e = tid + q * 256;
      Xs[buf][e % TJ4][e / TJ4] = (float)rx[q];
    }
  };
  float acc[8][NC];   // [row r: ty*4 + r (r < 4), 64 + ty*4 + r - 4][step c likewise]
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[r][c] = 0.f;
  load(0);
  for (int st = 0; st < stages; ++st) {
    const int buf = st & 1;
    store(buf);
    __syncthreads();
    if (st + 1 < stages) load(st + 1);     // in flight while this stage is multiplied
#pragma unroll
    for (int jj = 0; jj < TJ4; ++jj) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][jj][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][jj][64 + ty * 4]);
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[buf][jj][tx * 4]);
      float bv[NC];
      bv[0] = x0.x;
      bv[1] = x0.y;
      bv[2] = x0.z;
      bv[3] = x0.w;
      if constexpr (NC == 8) {
        const float4 x1 = *reinterpret_cast<const float4*>(&Xs[buf][jj][64 + tx * 4]);
        bv[4] = x1.x;
        bv[5] = x1.y;
        bv[6] = x1.z;
        bv[7] = x1.w;
      }
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    if (st % nj == nj - 1) {   // the lag's partial is complete: fold it, restart
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int k = r * NC + c;
          float h = H[k * 256 + tid], l = Lo[k * 256 + tid];
          two_sum_add(h, l, acc[r][c]);
          H[k * 256 + tid] = h;
          Lo[k * 256 + tid] = l;
          acc[r][c] = 0.f;
        }
    }
  }
  double* pt = part + ((((size_t)b * MT + mt) * CH + ch) * TMV) * nx;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int mm = (c < 4 ? 0 : 64) + tx * 4 + (c & 3);
    if (m0 + mm > mmax) continue;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int gi = i0 + (r < 4 ? 0 : 64) + ty * 4 + (r & 3);
      const int k = r * NC + c;
      if (gi < nx) pt[(size_t)mm * nx + gi] = (double)H[k * 256 + tid] + (double)Lo[k * 256 + tid];
    }
  }
}

__global__ void __launch_bounds__(256, 1)
k_apply32(int nt, int nx, int MT, int CH, int DC, int lag_lo, int lag_hi, const float* __restrict__ A,
          const double* __restrict__ x, double* __restrict__ part) {
  extern __shared__ __align__(16) float smem32[];
  apply32_body<TM4>(nt, nx, MT, CH, DC, lag_lo, lag_hi, A, x, part, blockIdx.x, blockIdx.y, blockIdx.z / MT,
                    blockIdx.z % MT, smem32);
}

// ---- ragged batches ------------------------------------------------------------------
__device__ __forceinline__ int ragged_find(const long long* __restrict__ prefix, int P, long long item) {
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Persistent product over the units of every problem (order: largest first);
// unit u of a problem is (ch, mt, it) with it fastest, so that concurrent
// units share lag blocks in L2.
template <typename TA, typename TC>
__global__ void __launch_bounds__(kApplyThreads)
k_ragged_apply(const RaggedApplyPlan* __restrict__ plans, const int* __restrict__ order,
               const long long* __restrict__ prefix, int P, unsigned long long* __restrict__ counter,
               const TA* __restrict__ A, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ TC As[TJ][TI + 1];
  __shared__ TC Xs[TJ][TM + 1];
  __shared__ long long item_s;
  const long long total = prefix[P];
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ULL);
    __syncthreads();
    const long long item = item_s;
    __syncthreads();
    if (item >= total) break;
    const int s = ragged_find(prefix, P, item);
    const RaggedApplyPlan pl = plans[order[s]];
    const long long u = item - prefix[s];
    const int it = (int)(u % pl.IT);
    const long long r = u / pl.IT;
    const int mt = (int)(r % pl.MT), ch = (int)(r / pl.MT);
    apply_body<TA, TC, false>(pl.nt, pl.nx, pl.MT, pl.CH, pl.DC, 0, pl.nt, A + pl.a_off, x + pl.v_off,
                              part + pl.part_off, it, ch, 0, mt, As, Xs);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256, 2)
k_ragged_apply32(const RaggedApplyPlan* __restrict__ plans, const int* __restrict__ order,
                 const long long* __restrict__ prefix, int P, unsigned long long* __restrict__ counter,
                 const float* __restrict__ A, const double* __restrict__ x, double* __restrict__ part) {
  extern __shared__ __align__(16) float smem32[];
  __shared__ long long item_s;
  const long long total = prefix[P];
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ULL);
    __syncthreads();
    const long long item = item_s;
    __syncthreads();
    if (item >= total) break;
    const int s = ragged_find(prefix, P, item);
    const RaggedApplyPlan pl = plans[order[s]];
    const long long u = item - prefix[s];
    const int it = (int)(u % pl.IT);
    const long long r = u / pl.IT;
    const int mt = (int)(r % pl.MT), ch = (int)(r / pl.MT);
    apply32_body<TM4R>(pl.nt, pl.nx, pl.MT, pl.CH, pl.DC, 0, pl.nt, A + pl.a_off, x + pl.v_off, part + pl.part_off,
                       it, ch, 0, mt, smem32);
    __syncthreads();
  }
}

// y = sum of the lag-chunk partials, every problem (vprefix: natural order)
template <int TM_>
__global__ void k_ragged_reduce(const RaggedApplyPlan* __restrict__ plans, const long long* __restrict__ vprefix,
                                int P, const double* __restrict__ part, double* __restrict__ y) {
  const long long total = vprefix[P];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int p = ragged_find(vprefix, P, e);
    const RaggedApplyPlan pl = plans[p];
    const long long local = e - vprefix[p];
    const int i = (int)(local % pl.nx), m = (int)(local / pl.nx);
    const int mt = m / TM_, mm = m % TM_;
    const int mmax = min(mt * TM_ + TM_, pl.nt) - 1;
    const int nch = min(pl.CH, mmax / pl.DC + 1);
    const double* pt = part + pl.part_off + (((size_t)mt * pl.CH) * TM_ + mm) * pl.nx + i;
    double acc = 0.0;
    for (int c = 0; c < nch; ++c) acc += pt[(size_t)c * TM_ * pl.nx];
    y[pl.v_off + local] = acc;
  }
}

// y (= or +=) the sum of the lag-chunk partials of a product over the lags
// [lag_lo, lag_lo + CH DC): chunk c holds lags lag_lo + c DC .., written only
// where it has a lag <= the tile's last step (mmax)
template <bool TRANS, int TM_ = TM>
__global__ void k_apply_reduce(int nt, int nx, int n_rhs, int MT, int CH, int DC, int lag_lo, int accumulate,
                               const double* __restrict__ part, double* __restrict__ y) {
  const size_t total = (size_t)n_rhs * nt * nx;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % nx);
    const int m = (int)((e / nx) % nt);       // time index in the computed order
    const int b = (int)(e / ((size_t)nx * nt));
    const int mt = m / TM_, mm = m % TM_;
    const int mmax = min(mt * TM_ + TM_, nt) - 1;
    const int nch = mmax < lag_lo ? 0 : min(CH, (mmax - lag_lo) / DC + 1);
    const double* pt = part + ((((size_t)b * MT + mt) * CH) * TM_ + mm) * nx + i;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += pt[(size_t)c * TM_ * nx];
    const int mo = TRANS ? (nt - 1 - m) : m;
    double* yp = y + ((size_t)b * nt + mo) * nx + i;
    *yp = accumulate ? *yp + s : s;
  }
}

static cudaError_t launch32(int nt, int nx, int lag_lo, int lag_hi, const float* A, int n_rhs, const double* x,
                            double* y, bool accumulate, double* part, cudaStream_t s) {
  const ApplyPlan p = make_plan(nt, nx, TM4, TI4, lag_hi - lag_lo);
  cudaError_t e = cudaFuncSetAttribute(k_apply32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApply32Smem);
  if (e != cudaSuccess) return e;
  k_apply32<<<dim3(p.IT, p.CH, n_rhs * p.MT), 256, kApply32Smem, s>>>(nt, nx, p.MT, p.CH, p.DC, lag_lo, lag_hi,
                                                                       A, x, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launches(2);
  const size_t total = (size_t)n_rhs * nt * nx;
  const int blocks = stride_grid(total, 256, 16);
  k_apply_reduce<false, TM4><<<blocks, 256, 0, s>>>(nt, nx, n_rhs, p.MT, p.CH, p.DC, lag_lo, accumulate ? 1 : 0,
                                                    part, y);
  return cudaGetLastError();
}

template <typename TA, typename TC>
static cudaError_t launch(bool trans, int nt, int nx, int lag_lo, int lag_hi, const TA* A, int n_rhs,
                          const double* x, double* y, bool accumulate, double* part, cudaStream_t s) {
  if constexpr (sizeof(TA) == 4) {
    if (!trans && use_apply32(nt, nx, n_rhs)) return launch32(nt, nx, lag_lo, lag_hi, A, n_rhs, x, y, accumulate,
                                                               part, s);
  }
  const ApplyPlan p = make_plan(nt, nx, TM, TI, lag_hi - lag_lo);
  dim3 grid(p.IT, p.CH, n_rhs * p.MT);
  if (trans)
    k_apply<TA, TC, true><<<grid, kApplyThreads, 0, s>>>(nt, nx, p.MT, p.CH, p.DC, lag_lo, lag_hi, A, x, part);
  else
    k_apply<TA, TC, false><<<grid, kApplyThreads, 0, s>>>(nt, nx, p.MT, p.CH, p.DC, lag_lo, lag_hi, A, x, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launches(2);
  const size_t total = (size_t)n_rhs * nt * nx;
  const int threads = 256;
  const int blocks = stride_grid(total, threads, 16);
  const int acc = accumulate ? 1 : 0;
  if (trans)
    k_apply_reduce<true><<<blocks, threads, 0, s>>>(nt, nx, n_rhs, p.MT, p.CH, p.DC, lag_lo, acc, part, y);
  else
    k_apply_reduce<false><<<blocks, threads, 0, s>>>(nt, nx, n_rhs, p.MT, p.CH, p.DC, lag_lo, acc, part, y);
  return cudaGetLastError();
}

// ---- allocation-free variant --------------------------------------------------
// Scratch for callers that cannot allocate device memory: a fixed array in the
// library's own device image.  Every GPU that loads this library keeps these
// kNoAllocScratchBytes until the process exits.  Host code must not use the
// symbol as a pointer; its device address is looked up once per device.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
static unsigned long long g_noalloc_ctx_id[kNoAllocMaxDevices] = {};

// Unique id of the current CUDA context (driver entry points cuCtxGetCurrent
// and cuCtxGetId, fetched through the runtime).  Ids are never reused, so a
// context created after cudaDeviceReset has a new one.
static cudaError_t current_context_id(unsigned long long* id) {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  if (!get_current || !get_id) {
    void* p = nullptr;
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r1, r2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &r1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &q, 12000, cudaEnableDefault, &r2);
    if (e != cudaSuccess) return e;
    if (r1 != cudaDriverEntryPointSuccess || r2 != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
    get_current = reinterpret_cast<GetCurrent>(p);
    get_id = reinterpret_cast<GetId>(q);
  }
  void* c = nullptr;
  if (get_current(&c) != 0 || !c) return cudaErrorDeviceUninitialized;
  return get_id(c, id) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}

cudaError_t noalloc_scratch_ptr(int device, void** ptr) {
  if (device < 0 || device >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  // the caller has made `device` current (and so created its context)
  unsigned long long id = 0;
  cudaError_t e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  if (!g_noalloc_ptr[device] || g_noalloc_ctx_id[device] != id) {
    // first call in this context of the device: resolve the symbol once
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = p;
    g_noalloc_ctx_id[device] = id;
  }
  *ptr = g_noalloc_ptr[device];
  return cudaSuccess;
}

bool apply_grid_fits(int nt, int nx, int n_rhs) {
  const ApplyPlan p = make_plan(nt, nx);
  if ((long long)n_rhs * p.MT > 65535) return false;
  if (use_apply32(nt, nx, n_rhs)) {
    const ApplyPlan q = make_plan(nt, nx, TM4, TI4);
    if ((long long)n_rhs * q.MT > 65535) return false;
  }
  return true;
}

void ragged_apply_plan(int nt, int nx, int lags_per_chunk, bool fp32_tiles, RaggedApplyPlan* p) {
  const int tm = fp32_tiles ? TM4R : TM, ti = fp32_tiles ? TI4 : TI;
  p->nt = nt;
  p->nx = nx;
  p->MT = (nt + tm - 1) / tm;
  p->IT = (nx + ti - 1) / ti;
  p->DC = lags_per_chunk < 1 ? 1 : (lags_per_chunk > nt ? nt : lags_per_chunk);
  p->CH = (nt + p->DC - 1) / p->DC;
  p->units = (long long)p->IT * p->MT * p->CH;
  p->part_elems = (long long)p->MT * p->CH * tm * nx;
}

bool ragged_fp32_tiles_ok(int nx) { return use_apply32(nx); }

cudaError_t ragged_apply_launch(int prec, bool fp32_tiles, const RaggedApplyPlan* plans, RaggedItems items,
                                const long long* vprefix, int P, unsigned long long* counter, const void* A,
                                const double* x, double* y, double* part, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (prec == STBEM_F64) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ragged_apply<double, double>, kApplyThreads, 0);
    if (e != cudaSuccess) return e;
    k_ragged_apply<double, double><<<sms * (occ > 0 ? occ : 1), kApplyThreads, 0, s>>>(
        plans, items.order, items.prefix, P, counter, static_cast<const double*>(A), x, part);
  } else if (fp32_tiles) {
    e = cudaFuncSetAttribute(k_ragged_apply32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApply32SmemR);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ragged_apply32, 256, kApply32SmemR);
    if (e != cudaSuccess) return e;
    k_ragged_apply32<<<sms * (occ > 0 ? occ : 1), 256, kApply32SmemR, s>>>(plans, items.order, items.prefix, P,
                                                                          counter, static_cast<const float*>(A), x,
                                                                          part);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ragged_apply<float, float>, kApplyThreads, 0);
    if (e != cudaSuccess) return e;
    k_ragged_apply<float, float><<<sms * (occ > 0 ? occ : 1), kApplyThreads, 0, s>>>(
        plans, items.order, items.prefix, P, counter, static_cast<const float*>(A), x, part);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (prec != STBEM_F64 && fp32_tiles)
    k_ragged_reduce<TM4R><<<sms * 8, 256, 0, s>>>(plans, vprefix, P, part, y);
  else
    k_ragged_reduce<TM><<<sms * 8, 256, 0, s>>>(plans, vprefix, P, part, y);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t apply_range_launch(int prec, bool trans, int nt, int nx, int lag_lo, int lag_hi, const void* A,
                               int n_rhs, const double* x, double* y, bool accumulate, void* work, cudaStream_t s) {
  double* part = static_cast<double*>(work);
  if (prec == STBEM_F64)
    return launch<double, double>(trans, nt, nx, lag_lo, lag_hi, static_cast<const double*>(A), n_rhs, x, y,
                                  accumulate, part, s);
  return launch<float, float>(trans, nt, nx, lag_lo, lag_hi, static_cast<const float*>(A), n_rhs, x, y, accumulate,
                              part, s);
}

cudaError_t apply_launch(int prec, bool trans, int nt, int nx, const void* A, int n_rhs,
                         const double* x, double* y, void* work, cudaStream_t s) {
  return apply_range_launch(prec, trans, nt, nx, 0, nt, A, n_rhs, x, y, false, work, s);
}

}  // namespace stbem
