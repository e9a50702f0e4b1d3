// Vector kernels: right-hand side data, mass matrices and the FP64 building
// blocks of GMRES (dot products, linear combinations, diagonal scaling).
#include <cuda_runtime.h>

#include "device_info.h"
#include "special.cuh"
#include "vec.h"

#include <atomic>

namespace stbem {

static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned n) { g_launches += n; }
unsigned long long launch_count() { return g_launches.load(); }

// g[n][p] = (1/ht) int_{tau_n} U*(x_p - y*, t) dt
//         = alpha/(4 pi) [E1(a_p/t_{n+1}) - E1(a_p/t_n)] / ht,  a_p = alpha |x_p - y*|^2 / 4
__global__ void k_rhs_g(DevMesh M, double ysx, double ysy, double* __restrict__ g) {
  const int total = M.n_t * M.N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int p = e % M.N, n = e / M.N;
    const double dx = M.vx[p] - ysx, dy = M.vy[p] - ysy;
    const double a = M.alpha * (dx * dx + dy * dy) / 4.0;
    const double t1 = (double)(n + 1) * M.ht, t0 = (double)n * M.ht;
    const double E1 = e1_only(a / t1);
    const double E0 = n > 0 ? e1_only(a / t0) : 0.0;
    g[e] = (E1 - E0) * M.alpha / (4.0 * kPi) / M.ht;
  }
}

// f[b][m][i] += (1/2) M_h g[b]: M_h[(i,m),(p,m)] = ht h_i / 2 for p in {i, i+1}
__global__ void k_half_mass_add(DevMesh M, int B, const double* __restrict__ g, double* __restrict__ f) {
  const size_t total = (size_t)B * M.n_t * M.N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % M.N);
    const size_t row = e - i;                 // start of this (b, m) row
    const int ip = (i + 1) % M.N;
    const double hm = 0.5 * M.ht * 0.5 * M.slen[i] * (g[e] + g[row + ip]);
    f[e] = hm + f[e];
  }
}

// L_l = ht (h_{l-1} + 2 h_l + h_{l+1}) / 4  (row sums of <phi0_k, psi_l>)
__global__ void k_lumped(DevMesh M, double* __restrict__ L) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= M.N) return;
  const int N = M.N;
  L[l] = M.ht * (M.slen[(l - 1 + N) % N] + 2.0 * M.slen[l] + M.slen[(l + 1) % N]) / 4.0;
}

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 64;

// Stage 1: per (vector k, block) partial sums; stage 2: sum partials in order.
__global__ void k_dots_partial(const double* __restrict__ Q, const double* __restrict__ v,
                               size_t n, double* __restrict__ part) {
  __shared__ double red[kRedThreads];
  const int k = blockIdx.y;
  const double* q = Q + (size_t)k * n;
  double s = 0.0;
  for (size_t e = (size_t)blockIdx.x * kRedThreads + threadIdx.x; e < n; e += (size_t)kRedBlocks * kRedThreads)
    s = fma(q[e], v[e], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)k * kRedBlocks + blockIdx.x] = red[0];
}

__global__ void k_dots_final(const double* __restrict__ part, int k, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k) return;
  double s = 0.0;
  for (int b = 0; b < kRedBlocks; ++b) s += part[(size_t)t * kRedBlocks + b];
  out[t] = s;
}

// out holds k results followed by k * kRedBlocks scratch partials.
cudaError_t dots_launch(const double* Q, int k, const double* v, size_t n, double* out, cudaStream_t s) {
  double* part = out + k;
  k_dots_partial<<<dim3(kRedBlocks, k), kRedThreads, 0, s>>>(Q, v, n, part);
  k_dots_final<<<(k + 127) / 128, 128, 0, s>>>(part, k, out);
  count_launches(2);
  return cudaGetLastError();
}

__global__ void k_sub_comb(const double* __restrict__ Q, int k, const double* __restrict__ h,
                           double* __restrict__ v, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double s = v[e];
    for (int t = 0; t < k; ++t) s -= h[t] * Q[(size_t)t * n + e];
    v[e] = s;
  }
}
__global__ void k_comb(const double* __restrict__ Q, int k, const double* __restrict__ h,
                       double* __restrict__ y, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < k; ++t) s += h[t] * Q[(size_t)t * n + e];
    y[e] = s;
  }
}
__global__ void k_scale(const double* __restrict__ x, double a, double* __restrict__ y, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = a * x[e];
}
__global__ void k_axpy(double a, const double* __restrict__ x, double* __restrict__ y, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}
__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = a[e] - b[e];
}
__global__ void k_diag_div(const double* __restrict__ x, const double* __restrict__ L,
                           double* __restrict__ y, int nt, int nx) {
  const size_t n = (size_t)nt * nx;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = x[e] / L[e % nx];
}

__global__ void k_round_f32(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}

__global__ void k_bdots(const double* __restrict__ Q, const double* __restrict__ U, int B, size_t n,
                        double* __restrict__ out) {
  __shared__ double red[kRedThreads];
  const int b = blockIdx.x, t = blockIdx.y;
  const double* q = Q + ((size_t)t * B + b) * n;
  const double* u = U + (size_t)b * n;
  double s = 0.0;
  for (size_t e = threadIdx.x; e < n; e += kRedThreads) s = fma(q[e], u[e], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(size_t)t * B + b] = red[0];
}

__global__ void k_bsub_comb(const double* __restrict__ Q, int k, const double* __restrict__ H,
                            double* __restrict__ U, int B, size_t n) {
  const size_t total = (size_t)B * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / n);
    double v = U[e];
    for (int t = 0; t < k; ++t) v -= H[(size_t)t * B + b] * Q[(size_t)t * total + e];
    U[e] = v;
  }
}

__global__ void k_bcomb(const double* __restrict__ Q, int k, const double* __restrict__ C, double* __restrict__ Y,
                        int B, size_t n) {
  const size_t total = (size_t)B * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / n);
    double v = 0.0;
    for (int t = 0; t < k; ++t) v += C[(size_t)t * B + b] * Q[(size_t)t * total + e];
    Y[e] = v;
  }
}

__global__ void k_bscale(const double* __restrict__ X, const double* __restrict__ a, double* __restrict__ Y, int B,
                         size_t n) {
  const size_t total = (size_t)B * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    Y[e] = a[e / n] * X[e];
}

// ---- ragged batches: P problems, vectors concatenated (vprefix[p] = start) -----
__device__ __forceinline__ int seg_of(const long long* __restrict__ prefix, int P, long long e) {
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

// out[t][p] = <Q[t] | seg p, U | seg p>; one block per (p, t), fixed-order reduction
__global__ void __launch_bounds__(256) k_rdots(const double* __restrict__ Q, size_t ldq,
                                               const double* __restrict__ U, const long long* __restrict__ vp,
                                               int P, double* __restrict__ out) {
  __shared__ double red[256];
  const int p = blockIdx.x, t = blockIdx.y;
  const double* q = Q + (size_t)t * ldq;
  double acc = 0.0;
  for (long long e = vp[p] + threadIdx.x; e < vp[p + 1]; e += 256) acc = fma(q[e], U[e], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(size_t)t * P + p] = red[0];
}

// U -= sum_t H[t][p] Q[t] (sign = -1) or Y = sum_t H[t][p] Q[t] (sign = 0)
__global__ void k_rcomb(const double* __restrict__ Q, size_t ldq, int k, const double* __restrict__ H,
                        const long long* __restrict__ vp, int P, int sub, double* __restrict__ U) {
  const long long n = vp[P];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int p = seg_of(vp, P, e);
    double acc = 0.0;
    for (int t = 0; t < k; ++t) acc = fma(H[(size_t)t * P + p], Q[(size_t)t * ldq + e], acc);
    U[e] = sub ? U[e] - acc : acc;
  }
}

// Y = a[p] X per segment
__global__ void k_rscale(const double* __restrict__ X, const double* __restrict__ a, const long long* __restrict__ vp,
                         int P, double* __restrict__ Y) {
  const long long n = vp[P];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    Y[e] = a[seg_of(vp, P, e)] * X[e];
}

// nrm[p] = sqrt(sq[p]); inv[p] = 1 / nrm[p] for active problems with a
// positive finite norm, else 0
__global__ void k_rinv(const double* __restrict__ sq, const int* __restrict__ active, int P, double* __restrict__ nrm,
                       double* __restrict__ inv) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double v = sqrt(sq[p]);
  nrm[p] = v;
  inv[p] = (active[p] && v > 0.0 && isfinite(v)) ? 1.0 / v : 0.0;
}

// y[e] = x[e] / L[mass_off + i] per problem
__global__ void k_rdiag_div(const RaggedProblem* __restrict__ probs, const long long* __restrict__ vp, int P,
                            const double* __restrict__ x, const double* __restrict__ L, double* __restrict__ y) {
  const long long n = vp[P];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int p = seg_of(vp, P, e);
    const int N = probs[p].M.N;
    const int i = (int)((e - vp[p]) % N);
    y[e] = x[e] / L[probs[p].mass_off + i];
  }
}

// right-hand side data of every problem (source ystar[p]) and masses
__global__ void k_rrhs_g(const RaggedProblem* __restrict__ probs, const long long* __restrict__ vp, int P,
                         const double* __restrict__ ystar, double* __restrict__ g) {
  const long long n = vp[P];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int p = seg_of(vp, P, e);
    const DevMesh& M = probs[p].M;
    const long long local = e - vp[p];
    const int q = (int)(local % M.N), t = (int)(local / M.N);
    const double dx = M.vx[q] - ystar[2 * p], dy = M.vy[q] - ystar[2 * p + 1];
    const double a = M.alpha * (dx * dx + dy * dy) / 4.0;
    const double E1 = e1_only(a / ((double)(t + 1) * M.ht));
    const double E0 = t > 0 ? e1_only(a / ((double)t * M.ht)) : 0.0;
    g[e] = (E1 - E0) * M.alpha / (4.0 * kPi) / M.ht;
  }
}

__global__ void k_rhalf_mass_add(const RaggedProblem* __restrict__ probs, const long long* __restrict__ vp, int P,
                                 const double* __restrict__ g, double* __restrict__ f) {
  const long long n = vp[P];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int p = seg_of(vp, P, e);
    const DevMesh& M = probs[p].M;
    const int i = (int)((e - vp[p]) % M.N);
    const long long row = e - i;
    const int ip = (i + 1) % M.N;
    f[e] += 0.5 * M.ht * 0.5 * M.slen[i] * (g[e] + g[row + ip]);
  }
}

__global__ void k_rlumped(const RaggedProblem* __restrict__ probs, int P, double* __restrict__ L) {
  const int p = blockIdx.y;
  const DevMesh& M = probs[p].M;
  const int N = M.N;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < N; l += gridDim.x * blockDim.x)
    L[probs[p].mass_off + l] = M.ht * (M.slen[(l - 1 + N) % N] + 2.0 * M.slen[l] + M.slen[(l + 1) % N]) / 4.0;
}

static int grid_for(size_t n) { return stride_grid(n, 256, 8); }

// ---- non-uniform time grids (tn: the n_t + 1 time nodes) ----------------------------
// g[n][p] = (1/h_n) int_{tau_n} U*(x_p - y*, t) dt, h_n = t_{n+1} - t_n
__global__ void k_nu_rhs_g(DevMesh M, const double* __restrict__ tn, double ysx, double ysy, double* __restrict__ g) {
  const int total = M.n_t * M.N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int p = e % M.N, n = e / M.N;
    const double dx = M.vx[p] - ysx, dy = M.vy[p] - ysy;
    const double a = M.alpha * (dx * dx + dy * dy) / 4.0;
    const double E1 = e1_only(a / tn[n + 1]);
    const double E0 = n > 0 ? e1_only(a / tn[n]) : 0.0;
    g[e] = (E1 - E0) * M.alpha / (4.0 * kPi) / (tn[n + 1] - tn[n]);
  }
}

// f[m][i] += (1/2) M_h g: M_h[(i,m),(p,m)] = h_m h_i / 2 for p in {i, i+1}
__global__ void k_nu_half_mass_add(DevMesh M, const double* __restrict__ tn, const double* __restrict__ g,
                                   double* __restrict__ f) {
  const int total = M.n_t * M.N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e % M.N, m = e / M.N;
    const int row = e - i, ip = (i + 1) % M.N;
    const double hm = 0.5 * (tn[m + 1] - tn[m]) * 0.5 * M.slen[i] * (g[e] + g[row + ip]);
    f[e] = hm + f[e];
  }
}

// L[m][l] = h_m (h_{l-1} + 2 h_l + h_{l+1}) / 4: the lumped dual mass of step m
__global__ void k_nu_lumped(DevMesh M, const double* __restrict__ tn, double* __restrict__ L) {
  const int total = M.n_t * M.N;
  const int N = M.N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int l = e % N, m = e / N;
    L[e] = (tn[m + 1] - tn[m]) * (M.slen[(l - 1 + N) % N] + 2.0 * M.slen[l] + M.slen[(l + 1) % N]) / 4.0;
  }
}

cudaError_t nu_rhs_launch(const DevMesh& M, const double* tn, double ysx, double ysy, double* g, cudaStream_t s) {
  k_nu_rhs_g<<<grid_for((size_t)M.n_t * M.N), 256, 0, s>>>(M, tn, ysx, ysy, g);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t nu_half_mass_add_launch(const DevMesh& M, const double* tn, const double* g, double* f, cudaStream_t s) {
  k_nu_half_mass_add<<<grid_for((size_t)M.n_t * M.N), 256, 0, s>>>(M, tn, g, f);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t nu_lumped_launch(const DevMesh& M, const double* tn, double* L, cudaStream_t s) {
  k_nu_lumped<<<grid_for((size_t)M.n_t * M.N), 256, 0, s>>>(M, tn, L);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t rhs_g_launch(const DevMesh& M, double ysx, double ysy, double* g, cudaStream_t s) {
  k_rhs_g<<<grid_for((size_t)M.n_t * M.N), 256, 0, s>>>(M, ysx, ysy, g);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t half_mass_add_launch(const DevMesh& M, const double* g, double* f, cudaStream_t s, int B) {
  k_half_mass_add<<<grid_for((size_t)B * M.n_t * M.N), 256, 0, s>>>(M, B, g, f);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t lumped_mass_launch(const DevMesh& M, double* L, cudaStream_t s) {
  k_lumped<<<(M.N + 127) / 128, 128, 0, s>>>(M, L);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t sub_combination_launch(const double* Q, int k, const double* h, double* v, size_t n, cudaStream_t s) {
  k_sub_comb<<<grid_for(n), 256, 0, s>>>(Q, k, h, v, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t combination_launch(const double* Q, int k, const double* h, double* y, size_t n, cudaStream_t s) {
  k_comb<<<grid_for(n), 256, 0, s>>>(Q, k, h, y, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t scale_launch(const double* x, double a, double* y, size_t n, cudaStream_t s) {
  k_scale<<<grid_for(n), 256, 0, s>>>(x, a, y, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t axpy_launch(double a, const double* x, double* y, size_t n, cudaStream_t s) {
  k_axpy<<<grid_for(n), 256, 0, s>>>(a, x, y, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t sub_launch(const double* a, const double* b, double* y, size_t n, cudaStream_t s) {
  k_sub<<<grid_for(n), 256, 0, s>>>(a, b, y, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t bdots_launch(const double* Q, int k, const double* U, int B, size_t n, double* out, cudaStream_t s) {
  k_bdots<<<dim3(B, k), kRedThreads, 0, s>>>(Q, U, B, n, out);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t bsub_comb_launch(const double* Q, int k, const double* H, double* U, int B, size_t n, cudaStream_t s) {
  k_bsub_comb<<<grid_for((size_t)B * n), 256, 0, s>>>(Q, k, H, U, B, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t bcomb_launch(const double* Q, int k, const double* C, double* Y, int B, size_t n, cudaStream_t s) {
  k_bcomb<<<grid_for((size_t)B * n), 256, 0, s>>>(Q, k, C, Y, B, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t bscale_launch(const double* X, const double* a, double* Y, int B, size_t n, cudaStream_t s) {
  k_bscale<<<grid_for((size_t)B * n), 256, 0, s>>>(X, a, Y, B, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t round_f32_launch(const double* src, float* dst, size_t n, cudaStream_t s) {
  k_round_f32<<<grid_for(n), 256, 0, s>>>(src, dst, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t diag_div_launch(const double* x, const double* L, double* y, int nt, int nx, cudaStream_t s) {
  k_diag_div<<<grid_for((size_t)nt * nx), 256, 0, s>>>(x, L, y, nt, nx);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace stbem

namespace stbem {
static int rgrid(long long n) { return stride_grid(n < 0 ? 0 : (size_t)n, 256, 8); }
cudaError_t rdots_launch(const double* Q, size_t ldq, int k, const double* U, const long long* vp, int P,
                         double* out, cudaStream_t s) {
  k_rdots<<<dim3(P, k), 256, 0, s>>>(Q, ldq, U, vp, P, out);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t rcomb_launch(const double* Q, size_t ldq, int k, const double* H, const long long* vp, int P, bool sub,
                         double* U, long long n, cudaStream_t s) {
  k_rcomb<<<rgrid(n), 256, 0, s>>>(Q, ldq, k, H, vp, P, sub ? 1 : 0, U);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t rscale_launch(const double* X, const double* a, const long long* vp, int P, double* Y, long long n,
                          cudaStream_t s) {
  k_rscale<<<rgrid(n), 256, 0, s>>>(X, a, vp, P, Y);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t rinv_launch(const double* sq, const int* active, int P, double* nrm, double* inv, cudaStream_t s) {
  k_rinv<<<(P + 127) / 128, 128, 0, s>>>(sq, active, P, nrm, inv);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t rdiag_div_launch(const RaggedProblem* probs, const long long* vp, int P, const double* x, const double* L,
                             double* y, long long n, cudaStream_t s) {
  k_rdiag_div<<<rgrid(n), 256, 0, s>>>(probs, vp, P, x, L, y);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t rrhs_g_launch(const RaggedProblem* probs, const long long* vp, int P, const double* ystar, double* g,
                          long long n, cudaStream_t s) {
  k_rrhs_g<<<rgrid(n), 256, 0, s>>>(probs, vp, P, ystar, g);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t rhalf_mass_add_launch(const RaggedProblem* probs, const long long* vp, int P, const double* g, double* f,
                                  long long n, cudaStream_t s) {
  k_rhalf_mass_add<<<rgrid(n), 256, 0, s>>>(probs, vp, P, g, f);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t rlumped_launch(const RaggedProblem* probs, int P, int max_n, double* L, cudaStream_t s) {
  k_rlumped<<<dim3((max_n + 127) / 128, P), 128, 0, s>>>(probs, P, L);
  count_launches(1);
  return cudaGetLastError();
}
}  // namespace stbem

namespace stbem {
// Y[m] = B X[m] (trans = 0) or B^T X[m] (trans = 1) for every time step m:
// Y (rows x N) = X (rows x N) op(B)^T, B an N x N row-major FP64 matrix.
// 64 x 64 output tiles (steps x entries), 16-wide chunks of the sum.
__global__ void __launch_bounds__(256) k_blockmul(int rows, int N, const double* __restrict__ B, int trans,
                                                  const double* __restrict__ X, double* __restrict__ Y) {
  __shared__ double Xs[16][65], Bs[16][65];
  const int m0 = blockIdx.y * 64, i0 = blockIdx.x * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int j0 = 0; j0 < N; j0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int jj = e % 16, r = e / 16;
      const int m = m0 + r, i = i0 + r, j = j0 + jj;
      Xs[jj][r] = (m < rows && j < N) ? X[(size_t)m * N + j] : 0.0;
      Bs[jj][r] = (i < N && j < N) ? (trans ? B[(size_t)j * N + i] : B[(size_t)i * N + j]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      double xv[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xv[q] = Xs[jj][ty * 4 + q];
        bv[q] = Bs[jj][tx * 4 + q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] = fma(xv[q], bv[r], acc[q][r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int m = m0 + ty * 4 + q, i = i0 + tx * 4 + r;
      if (m < rows && i < N) Y[(size_t)m * N + i] = acc[q][r];
    }
}

cudaError_t blockmul_launch(int rows, int N, const double* B, bool trans, const double* X, double* Y,
                            cudaStream_t s) {
  k_blockmul<<<dim3((N + 63) / 64, (rows + 63) / 64), 256, 0, s>>>(rows, N, B, trans ? 1 : 0, X, Y);
  count_launches(1);
  return cudaGetLastError();
}
}  // namespace stbem
