// The block-Toeplitz product through time-domain FFTs (see toeplitz_fft.h).
//
// Transforms: radix-2 decimation in time on length-L sequences held in shared
// memory, two real columns packed as one complex sequence (z = a + i b; the
// transforms of a and b are separated with the Hermitian symmetry).  The
// twiddles w^m = e^{-2 pi i m / L}, m < L/2, are computed once per CTA with
// sincospi at the exact arguments 2m/L.  The frequency products read each
// block row of Ahat_k once with 16-byte loads and reduce with warp shuffles
// (forward) or across warps in shared memory (transposed): the product is
// bound by the HBM bytes of Ahat.
#include <cuda_runtime.h>

#include "assemble.h"
#include "stbem.h"
#include "toeplitz_fft.h"

namespace stbem {

namespace {

constexpr int kFftThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// w^m, m < L/2, into tw (sign -1: forward transform, +1: inverse)
__device__ __forceinline__ void twiddles(double2* tw, int L, double sign) {
  for (int m = threadIdx.x; m < L / 2; m += blockDim.x) {
    double sn, cs;
    sincospi(sign * 2.0 * (double)m / (double)L, &sn, &cs);
    tw[m] = make_double2(cs, sn);
  }
}

// In-place radix-2 butterflies of Q bit-reversed sequences z[q][0..L), from
// stage s0 on (stage s combines pairs 2^s apart).  The twiddles of stage 1
// are 1 and w^{L/4} = -i (sign -1) or +i (sign +1): no multiplication.
__device__ __forceinline__ void fft_stages(double2* z, const double2* tw, int Q, int L, int logL, int s0,
                                           double sign) {
  const int H = L / 2;
  for (int s = s0; s < logL; ++s) {
    const int half = 1 << s;
    for (int idx = threadIdx.x; idx < Q * H; idx += blockDim.x) {
      const int q = idx / H, b = idx - q * H;
      const int pos = b & (half - 1);
      const int i0 = ((b >> s) << (s + 1)) + pos;
      double2* zq = z + (size_t)q * L;
      const double2 u = zq[i0], v = zq[i0 + half];
      double2 t;
      if (s == 0 || (s == 1 && pos == 0)) t = v;
      else if (s == 1) t = sign < 0 ? make_double2(v.y, -v.x) : make_double2(-v.y, v.x);
      else t = cmul(tw[pos << (logL - 1 - s)], v);
      zq[i0] = make_double2(u.x + t.x, u.y + t.y);
      zq[i0 + half] = make_double2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int v, int logL) { return (int)(__brev((unsigned)v) >> (32 - logL)); }

// Forward real FFT of the columns [c0, c0 + 2Q) of in[d][c] (row stride ld,
// rows d < nt, zero to L): out[k][c], k = 0..L/2, row stride ncols.
// blockIdx.y selects a batch (strides in_batch, out_batch).
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_rfft_cols(const T* __restrict__ in, long long ld, int ncols, int nt,
                                                           int L, int logL, int Q, long long in_batch,
                                                           long long out_batch, double2* __restrict__ out) {
  extern __shared__ double2 fsm[];
  double2* tw = fsm;
  double2* z = fsm + L / 2;
  in += (long long)blockIdx.y * in_batch;
  out += (long long)blockIdx.y * out_batch;
  const long long c0 = (long long)blockIdx.x * 2 * Q;
  twiddles(tw, L, -1.0);
  const int G = 2 * Q;
  // The second half of every sequence is zero padding (n_t <= L/2), so the
  // first stage maps the pair (x_d, x_{d + L/2} = 0), d < L/2, at bit-reversed
  // positions p, p + 1 to (x_d, x_d): it is done here, on load.  Eight loads
  // in flight per thread before their shared-memory stores.
  constexpr int U = 8;
  const int HG = (L / 2) * G;
  for (int base = 0; base < HG; base += U * kFftThreads) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * kFftThreads + threadIdx.x;
      const int d = idx / G, cc = idx - d * G;
      const long long c = c0 + cc;
      v[u] = (idx < HG && d < nt && c < ncols) ? (double)in[(long long)d * ld + c] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * kFftThreads + threadIdx.x;
      if (idx >= HG) break;
      const int d = idx / G, cc = idx - d * G;
      double* p = reinterpret_cast<double*>(z + (size_t)(cc >> 1) * L + bitrev(d, logL));
      p[cc & 1] = v[u];
      p[2 + (cc & 1)] = v[u];
    }
  }
  __syncthreads();
  fft_stages(z, tw, Q, L, logL, 1, -1.0);
  const int K = L / 2 + 1;
  for (int idx = threadIdx.x; idx < K * G; idx += blockDim.x) {
    const int k = idx / G, cc = idx - k * G;
    const long long c = c0 + cc;
    if (c >= ncols) continue;
    const double2* zq = z + (size_t)(cc >> 1) * L;
    const double2 zk = zq[k], zm = zq[(L - k) & (L - 1)];
    // a: (Z_k + conj Z_{L-k}) / 2;  b: (Z_k - conj Z_{L-k}) / (2 i)
    const double2 r = (cc & 1) ? make_double2(0.5 * (zk.y + zm.y), 0.5 * (zm.x - zk.x))
                               : make_double2(0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y));
    out[(long long)k * ncols + c] = r;
  }
}

// Inverse: in[k][c], k = 0..L/2 (row stride ncols), the transforms of real
// sequences; out[n][c] = (1/L) sum_k Y_k w^{-n k} for n < nt (row stride ncols).
// Y_0 and Y_{L/2} are real for a real sequence: their imaginary parts are dropped.
__global__ void __launch_bounds__(kFftThreads) k_irfft_cols(const double2* __restrict__ in, int ncols, int nt, int L,
                                                            int logL, int Q, long long in_batch, long long out_batch,
                                                            double* __restrict__ out) {
  extern __shared__ double2 fsm[];
  double2* tw = fsm;
  double2* z = fsm + L / 2;
  in += (long long)blockIdx.y * in_batch;
  out += (long long)blockIdx.y * out_batch;
  const long long c0 = (long long)blockIdx.x * 2 * Q;
  twiddles(tw, L, 1.0);
  const int H = L / 2, K = H + 1;
  for (int idx = threadIdx.x; idx < K * Q; idx += blockDim.x) {
    const int k = idx / Q, q = idx - k * Q;
    const long long c = c0 + 2 * q;
    double2 ya = make_double2(0.0, 0.0), yb = ya;
    if (c < ncols) ya = in[(long long)k * ncols + c];
    if (c + 1 < ncols) yb = in[(long long)k * ncols + c + 1];
    if (k == 0 || k == H) ya.y = yb.y = 0.0;
    double2* zq = z + (size_t)q * L;
    // Z_k = Ya_k + i Yb_k;  Z_{L-k} = conj(Ya_k) + i conj(Yb_k)
    zq[bitrev(k, logL)] = make_double2(ya.x - yb.y, ya.y + yb.x);
    if (k > 0 && k < H) zq[bitrev(L - k, logL)] = make_double2(ya.x + yb.y, yb.x - ya.y);
  }
  __syncthreads();
  fft_stages(z, tw, Q, L, logL, 0, 1.0);
  const int G = 2 * Q;
  const double inv = 1.0 / (double)L;
  for (int idx = threadIdx.x; idx < nt * G; idx += blockDim.x) {
    const int n = idx / G, cc = idx - n * G;
    const long long c = c0 + cc;
    if (c >= ncols) continue;
    const double2 v = z[(size_t)(cc >> 1) * L + n];
    out[(long long)n * ncols + c] = ((cc & 1) ? v.y : v.x) * inv;
  }
}

// Forward frequency products: a group of 8 lanes per row, each lane a
// stride-8 eighth of the row (16-byte loads, 128 contiguous bytes per row and
// step), two rows per group, four steps of both rows in flight; the group's
// sums are combined in 3 shuffle steps, so the reduction's FP64 adds stay a
// few percent of the multiply-adds (a warp per row spends 5 steps, a quarter
// of the work at N_x = 256).
constexpr int kMvGroup = 8;
constexpr int kMvGroups = kFftThreads / kMvGroup;
constexpr int kMvRowsPerGroup = 2;
constexpr int kMvRows = kMvGroups * kMvRowsPerGroup;

__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 x) {
  acc.x = fma(a.x, x.x, fma(-a.y, x.y, acc.x));
  acc.y = fma(a.x, x.y, fma(a.y, x.x, acc.y));
}

// Yh[r][k][i] = sum_j Ahat[k][i][j] Xh[r][k][j]; grid (row blocks, K, n_rhs)
__global__ void __launch_bounds__(kFftThreads) k_fft_matvec(const double2* __restrict__ Ahat, int nx, int K,
                                                            const double2* __restrict__ Xh, double2* __restrict__ Yh) {
  extern __shared__ double2 xs[];
  const int k = blockIdx.y, r = blockIdx.z;
  const double2* xk = Xh + ((long long)r * K + k) * nx;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) xs[j] = xk[j];
  __syncthreads();
  const int g = threadIdx.x / kMvGroup, l = threadIdx.x % kMvGroup;
  const int i0 = blockIdx.x * kMvRows + g;
  const double2* Ak = Ahat + (long long)k * nx * nx;
  double2 acc[kMvRowsPerGroup];
  const double2* row[kMvRowsPerGroup];
#pragma unroll
  for (int t = 0; t < kMvRowsPerGroup; ++t) {
    acc[t] = make_double2(0.0, 0.0);
    const int i = i0 + t * kMvGroups;
    row[t] = i < nx ? Ak + (long long)i * nx : nullptr;
  }
  constexpr int S = 4;     // steps of 8 columns in flight
  int j = l;
  for (; j + (S - 1) * kMvGroup < nx; j += S * kMvGroup) {
    double2 a[kMvRowsPerGroup][S];
#pragma unroll
    for (int t = 0; t < kMvRowsPerGroup; ++t)
#pragma unroll
      for (int u = 0; u < S; ++u) a[t][u] = row[t] ? __ldg(row[t] + j + u * kMvGroup) : make_double2(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < S; ++u) {
      const double2 x = xs[j + u * kMvGroup];
#pragma unroll
      for (int t = 0; t < kMvRowsPerGroup; ++t) cmac(acc[t], a[t][u], x);
    }
  }
  for (; j < nx; j += kMvGroup) {
    const double2 x = xs[j];
#pragma unroll
    for (int t = 0; t < kMvRowsPerGroup; ++t)
      cmac(acc[t], row[t] ? __ldg(row[t] + j) : make_double2(0.0, 0.0), x);
  }
#pragma unroll
  for (int t = 0; t < kMvRowsPerGroup; ++t) {
#pragma unroll
    for (int o = kMvGroup / 2; o > 0; o >>= 1) {
      acc[t].x += __shfl_xor_sync(0xffffffffu, acc[t].x, o);
      acc[t].y += __shfl_xor_sync(0xffffffffu, acc[t].y, o);
    }
  }
  if (l == 0) {
    double2* yk = Yh + ((long long)r * K + k) * nx;
#pragma unroll
    for (int t = 0; t < kMvRowsPerGroup; ++t)
      if (row[t]) yk[i0 + t * kMvGroups] = acc[t];
  }
}

// Yh[r][k][j] = sum_i conj(Ahat[k][i][j]) Xh[r][k][i]: lanes over 32 columns,
// warps over rows, the 8 warps' sums combined in shared memory; grid
// (column blocks of 32, K, n_rhs)
__global__ void __launch_bounds__(kFftThreads) k_fft_matvec_t(const double2* __restrict__ Ahat, int nx, int K,
                                                              const double2* __restrict__ Xh,
                                                              double2* __restrict__ Yh) {
  extern __shared__ double2 xs[];
  __shared__ double2 red[kFftThreads / 32][32];
  const int k = blockIdx.y, r = blockIdx.z;
  const double2* xk = Xh + ((long long)r * K + k) * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) xs[i] = xk[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 32 + lane;
  const bool on = j < nx;
  const double2* Ak = Ahat + (long long)k * nx * nx + (on ? j : 0);
  constexpr int W = kFftThreads / 32;
  double2 acc = make_double2(0.0, 0.0);
  int i = warp;
  for (; i + 3 * W < nx; i += 4 * W) {
    double2 a[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t] = on ? __ldg(Ak + (long long)(i + t * W) * nx) : make_double2(0.0, 0.0);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const double2 x = xs[i + t * W];
      acc.x = fma(a[t].x, x.x, fma(a[t].y, x.y, acc.x));
      acc.y = fma(a[t].x, x.y, fma(-a[t].y, x.x, acc.y));
    }
  }
  for (; i < nx; i += W) {
    const double2 a = on ? __ldg(Ak + (long long)i * nx) : make_double2(0.0, 0.0);
    const double2 x = xs[i];
    acc.x = fma(a.x, x.x, fma(a.y, x.y, acc.x));
    acc.y = fma(a.x, x.y, fma(-a.y, x.x, acc.y));
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && on) {
    double2 s = red[0][lane];
#pragma unroll
    for (int w = 1; w < W; ++w) {
      s.x += red[w][lane].x;
      s.y += red[w][lane].y;
    }
    Yh[((long long)r * K + k) * nx + j] = s;
  }
}

int log2i(int L) {
  int l = 0;
  while ((1 << l) < L) ++l;
  return l;
}

size_t fft_smem(int L, int Q) { return ((size_t)Q * L + L / 2) * sizeof(double2); }

template <typename T>
cudaError_t rfft_cols(const T* in, long long ld, int ncols, int nt, int Q, int batches, long long in_batch,
                      long long out_batch, double2* out, cudaStream_t s) {
  const int L = fft_len(nt), logL = log2i(L);
  const size_t smem = fft_smem(L, Q);
  cudaError_t e = cudaFuncSetAttribute(k_rfft_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long gx = (ncols + 2LL * Q - 1) / (2LL * Q);
  k_rfft_cols<T><<<dim3((unsigned)gx, batches), kFftThreads, smem, s>>>(in, ld, ncols, nt, L, logL, Q, in_batch,
                                                                       out_batch, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

int fft_len(int nt) {
  int L = 2;
  while (L < 2 * nt) L <<= 1;
  return L;
}

size_t fft_operator_bytes(int nt, int nx) { return (size_t)fft_freqs(nt) * nx * nx * sizeof(double2); }

size_t fft_apply_bytes(int nt, int nx, int n_rhs) {
  return 2 * (size_t)n_rhs * fft_freqs(nt) * nx * sizeof(double2);
}

cudaError_t fft_operator_launch(int prec, int nt, int nx, const void* A, double2* Ahat, cudaStream_t s) {
  const int L = fft_len(nt);
  int Q = 4096 / L;
  Q = Q < 1 ? 1 : (Q > 16 ? 16 : Q);
  const long long cols = (long long)nx * nx;
  if (cols > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (prec == STBEM_F32)
    return rfft_cols(static_cast<const float*>(A), cols, (int)cols, nt, Q, 1, 0, 0, Ahat, s);
  return rfft_cols(static_cast<const double*>(A), cols, (int)cols, nt, Q, 1, 0, 0, Ahat, s);
}

cudaError_t fft_apply_launch(bool trans, int nt, int nx, int n_rhs, const double2* Ahat, const double* x, double* y,
                             void* work, cudaStream_t s) {
  const int L = fft_len(nt), logL = log2i(L), K = L / 2 + 1;
  double2* Xh = static_cast<double2*>(work);
  double2* Yh = Xh + (size_t)n_rhs * K * nx;
  // one complex sequence (two columns) per CTA: the vectors are short
  cudaError_t e = rfft_cols(x, nx, nx, nt, 1, n_rhs, (long long)nt * nx, (long long)K * nx, Xh, s);
  if (e != cudaSuccess) return e;
  const size_t xs_bytes = (size_t)nx * sizeof(double2);
  if (trans) {
    e = cudaFuncSetAttribute(k_fft_matvec_t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs_bytes);
    if (e != cudaSuccess) return e;
    k_fft_matvec_t<<<dim3((nx + 31) / 32, K, n_rhs), kFftThreads, xs_bytes, s>>>(Ahat, nx, K, Xh, Yh);
  } else {
    e = cudaFuncSetAttribute(k_fft_matvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs_bytes);
    if (e != cudaSuccess) return e;
    k_fft_matvec<<<dim3((nx + kMvRows - 1) / kMvRows, K, n_rhs), kFftThreads, xs_bytes, s>>>(Ahat, nx, K, Xh, Yh);
  }
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = fft_smem(L, 1);
  e = cudaFuncSetAttribute(k_irfft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_irfft_cols<<<dim3((nx + 1) / 2, n_rhs), kFftThreads, smem, s>>>(Yh, nx, nt, L, logL, 1, (long long)K * nx,
                                                                    (long long)nt * nx, y);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace stbem
