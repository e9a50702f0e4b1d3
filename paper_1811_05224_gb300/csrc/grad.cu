// Shape (vertex) and alpha gradient of a loss on the solution w of
// V_h w = f, f = (1/2 M_h + K_h) g (Section 1, eq. (4)), by the adjoint method:
// given lambda with V_h^T lambda = dL/dw,
//
//   dL/dtheta = lambda^T (df/dtheta - (dV_h/dtheta) w)
//             = sum_d sum_ij [C^K_ij(d) dK^(d)_ij - C^V_ij(d) dV^(d)_ij]
//               + lambda^T (1/2 dM_h) g + gbar^T dg,
//   C^V(d) = sum_m lambda_m w_{m-d}^T,  C^K(d) = sum_m lambda_m g_{m-d}^T,
//   gbar = (1/2 M_h + K_h)^T lambda.
//
// The lag blocks are never differentiated into storage: each kernel recomputes
// the quadrature of its pair at every lag and contracts the derivative of the
// integrand with the weight C(d) on the fly.  Per rule point x - y is linear in
// the pair's four endpoints P_r (A0, A1 = test segment, B0, B1 = trial
// segment), x - y = sum_r c_r P_r, so
//   dc/dP_r = (alpha/2) c_r (x - y)          (c = alpha |x - y|^2 / 4)
//   dq/dP_r = c_r n_B + (B0: +, B1: -) ((x - y) . t_B / h_B) n_B,
//   d(h_A h_B)/dA1 = -d/dA0 = h_B t_A  (and likewise for B),
// with the time kernels' c-derivatives from dtimeint.cuh (K is proportional to
// alpha at fixed c).  The identical / shared-vertex rules give c_r from their
// own offsets, so that shared endpoints combine without cancellation.
//
// Kernels (all FP64, deterministic: fixed loops and fixed reduction trees):
//   k_corr          C(d) for all lags (tiled FP64 products over time),
//   k_grad_tensor   one thread per pair (V: i <= j, symmetric blocks; K: i != j),
//                   a block walks a chunk of lags, Peano tables per lag in
//                   shared memory; pairs of the singular classes skip lags 0, 1,
//   k_grad_singular one CTA per identical / shared-vertex pair, lags 0 and 1,
//                   graded / Duffy rules,
//   k_grad_datum    gbar^T dg per vertex, k_grad_mass lambda^T (1/2 dM) g per
//                   segment,
//   k_grad_gather   per vertex: the endpoint roles of every pair that touches it,
//   k_grad_alpha    the alpha total.
#include <cuda_runtime.h>

#include "assemble.h"
#include "dtimeint.cuh"
#include "grad.h"
#include "pairs.cuh"
#include "toeplitz.h"

namespace stbem {

namespace {

constexpr int kGradThreads = 128;
constexpr int kLagChunk = 32;
constexpr int kVals = 9;       // 4 endpoint roles x 2 coordinates + alpha

// value and c-derivative at lags >= 2 from the per-lag tables
template <int K>
__device__ __forceinline__ void dlag2(double c, int d, double alpha, const LagNodes<double>& L, double* k,
                                      double* dk) {
  if (c * L.inv_dht > 0.5 * (double)d) {
    double f[3], df[3];
    for (int q = 0; q < 3; ++q) dF_closed<K>(c, L.s[q], L.inv_s[q], alpha, &f[q], &df[q]);
    *k = (f[0] - 2.0 * f[1]) + f[2];
    *dk = (df[0] - 2.0 * df[1]) + df[2];
    return;
  }
  double a = 0.0, b = 0.0;
  for (int g = 0; g < L.n; ++g) {
    const double e = exp_neg_fast(c * L.sig[g]);
    const double wg = K == kV ? L.wv[g] : L.wk[g];
    a = fma(wg, e, a);
    b = fma(-wg * L.sig[g], e, b);
  }
  *k = a;
  *dk = b;
}

// Point p of the identical / shared-vertex rule (same points as the assembly)
// with the coefficients c_r of x - y in the endpoints A0, A1, B0, B1.
__device__ __forceinline__ void singular_point_coef(int cls, int p, const Piece& A, const Piece& B, double* xi,
                                                    double* eta, double* w, double* dx, double* dy, double cr[4]) {
  const double eax = A.x1 - A.x0, eay = A.y1 - A.y0;
  const double ebx = B.x1 - B.x0, eby = B.y1 - B.y0;
  if (cls == kIdentical) {
    const int per = kGradedN * kSingularInner;
    const int tri = p / per, rem = p % per;
    const int iu = rem / kSingularInner, it = rem % kSingularInner;
    const int o4 = gauss_offset(kSingularInner);
    const double U = c_tab.grx[iu], WU = c_tab.grw[iu];
    const double TA = c_tab.gx[o4 + it], WT = c_tab.gw[o4 + it];
    const double lo = (1.0 - U) * TA;
    *w = WU * WT * (1.0 - U);
    const double u = tri == 0 ? U : -U;          // xi - eta
    *xi = tri == 0 ? lo + U : lo;
    *eta = tri == 0 ? lo : lo + U;
    *dx = u * eax;
    *dy = u * eay;
    cr[0] = -u; cr[1] = u; cr[2] = 0.0; cr[3] = 0.0;
    return;
  }
  const int per = kGradedN * kDuffyAngular;
  const int tri = p / per, rem = p % per;
  const int ir = rem / kDuffyAngular, it = rem % kDuffyAngular;
  const int o16 = gauss_offset(kDuffyAngular);
  const double Rr = c_tab.grx[ir], WR = c_tab.grw[ir];
  const double T = c_tab.gx[o16 + it], WT = c_tab.gw[o16 + it];
  *w = WR * WT * Rr;
  const double xp = tri == 0 ? Rr : Rr * T;
  const double ep = tri == 0 ? Rr * T : Rr;
  if (cls == kAdjNext) {   // end of A == start of B: x - y = -xp e_A - ep e_B
    *xi = 1.0 - xp;
    *eta = ep;
    *dx = -xp * eax - ep * ebx;
    *dy = -xp * eay - ep * eby;
    cr[0] = xp; cr[1] = -xp; cr[2] = ep; cr[3] = -ep;
  } else {                 // start of A == end of B: x - y = xp e_A + ep e_B
    *xi = xp;
    *eta = 1.0 - ep;
    *dx = xp * eax + ep * ebx;
    *dy = xp * eay + ep * eby;
    cr[0] = -xp; cr[1] = xp; cr[2] = -ep; cr[3] = ep;
  }
}

// Role gradients of one pair from its accumulated sums (see the kernels):
// out[2 r + c] for roles r = A0, A1, B0, B1, out[8] alpha.
template <int OP>
__device__ __forceinline__ void finish_roles(const Piece& A, const Piece& B, double alpha, double val,
                                             const double T[4][2], const double Q[4], double al, double* out) {
  const double LL = A.len * B.len, ha = 0.5 * alpha;
  const double tax = (A.x1 - A.x0) / A.len, tay = (A.y1 - A.y0) / A.len;
  const double tbx = (B.x1 - B.x0) / B.len, tby = (B.y1 - B.y0) / B.len;
  const double sgn[4] = {-1.0, 1.0, -1.0, 1.0};
  for (int r = 0; r < 4; ++r) {
    double gx = LL * ha * T[r][0], gy = LL * ha * T[r][1];
    if (OP == STBEM_OP_K) {
      gx += LL * Q[r] * B.nx;
      gy += LL * Q[r] * B.ny;
    }
    const double lw = r < 2 ? val * B.len : val * A.len;
    gx += sgn[r] * lw * (r < 2 ? tax : tbx);
    gy += sgn[r] * lw * (r < 2 ? tay : tby);
    out[2 * r] = gx;
    out[2 * r + 1] = gy;
  }
  out[8] = LL * (0.25 * al + (OP == STBEM_OP_K ? val / alpha : 0.0));
}

// ---- C(d) = sum_{m >= d} lam[m] x[m-d]^T ---------------------------------------
constexpr int kCT = 64, kCM = 16;

__global__ void __launch_bounds__(256) k_corr(int nt, int N, const double* __restrict__ lam,
                                              const double* __restrict__ x, double* __restrict__ C) {
  __shared__ double Ls[kCM][kCT], Xs[kCM][kCT];
  const int d = blockIdx.z;
  const int i0 = blockIdx.y * kCT, j0 = blockIdx.x * kCT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int m0 = d; m0 < nt; m0 += kCM) {
    for (int e = threadIdx.x; e < kCM * kCT; e += 256) {
      const int mm = e / kCT, c = e % kCT;
      const int m = m0 + mm;
      const bool in_t = m < nt;
      Ls[mm][c] = (in_t && i0 + c < N) ? lam[(size_t)m * N + i0 + c] : 0.0;
      Xs[mm][c] = (in_t && j0 + c < N) ? x[(size_t)(m - d) * N + j0 + c] : 0.0;
    }
    __syncthreads();
    for (int mm = 0; mm < kCM; ++mm) {
      double a[4], b[4];
      for (int q = 0; q < 4; ++q) {
        a[q] = Ls[mm][ty * 4 + q];
        b[q] = Xs[mm][tx * 4 + q];
      }
      for (int q = 0; q < 4; ++q)
        for (int r = 0; r < 4; ++r) acc[q][r] = fma(a[q], b[r], acc[q][r]);
    }
    __syncthreads();
  }
  for (int q = 0; q < 4; ++q)
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + ty * 4 + q, j = j0 + tx * 4 + r;
      if (i < N && j < N) C[((size_t)d * N + i) * N + j] = acc[q][r];
    }
}

// ---- tensor-rule pairs -------------------------------------------------------------
__device__ __forceinline__ long long tri_start(long long r, int N) { return r * N - r * (r - 1) / 2; }

template <int OP>
__global__ void __launch_bounds__(kGradThreads) k_grad_tensor(DevMesh M, const double* __restrict__ C,
                                                              double* __restrict__ out) {
  __shared__ LagNodes<double> LN;
  const int N = M.N, nt = M.n_t;
  const double ht = M.ht, alpha = M.alpha;
  const long long npair = OP == STBEM_OP_V ? (long long)N * (N + 1) / 2 : (long long)N * N;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool live = p < npair;
  int i = 0, j = 0;
  if (live) {
    if (OP == STBEM_OP_V) {
      const double B2 = 2.0 * N + 1.0;
      i = (int)floor((B2 - sqrt(B2 * B2 - 8.0 * (double)p)) * 0.5);
      while (i > 0 && tri_start(i, N) > p) --i;
      while (tri_start(i + 1, N) <= p) ++i;
      j = i + (int)(p - tri_start(i, N));
    } else {
      i = (int)(p / N);
      j = (int)(p % N);
    }
  }
  const bool skip = OP == STBEM_OP_K && i == j;   // K: q = 0 on the identical pair
  Piece A = seg_piece(M, i), B = seg_piece(M, j);
  const int cls = live ? pair_class(N, i, j, A, B) : kRegular;
  const bool singular01 = cls == kIdentical || cls == kAdjNext || cls == kAdjPrev;
  const int jn = (j + 1) % N;

  const double eax = A.x1 - A.x0, eay = A.y1 - A.y0;
  const double ebx = B.x1 - B.x0, eby = B.y1 - B.y0;
  const double abx = A.x0 - B.x0, aby = A.y0 - B.y0;
  const double qab = abx * B.nx + aby * B.ny, qea = eax * B.nx + eay * B.ny;
  const double tbx = ebx / B.len, tby = eby / B.len, inv_lb = 1.0 / B.len;
  double val = 0.0, al = 0.0, TA[2] = {0.0, 0.0}, TX[2] = {0.0, 0.0}, TE[2] = {0.0, 0.0};
  double Q = 0.0, QX = 0.0, QE = 0.0, QT = 0.0;

  const int d0 = blockIdx.y * kLagChunk;
  const int d1 = min(nt, d0 + kLagChunk);
  for (int d = d0; d < d1; ++d) {
    if (d >= 2) {
      __syncthreads();
      build_lag_nodes<double>(LN, d, ht, alpha);
      __syncthreads();
    }
    if (!live || skip || (d < 2 && singular01)) continue;
    const size_t cb = (size_t)d * N * N;
    double W0, W1;
    if (OP == STBEM_OP_V) {
      W0 = i == j ? C[cb + (size_t)i * N + i] : C[cb + (size_t)i * N + j] + C[cb + (size_t)j * N + i];
      W1 = W0;
    } else {
      W0 = C[cb + (size_t)i * N + j];
      W1 = C[cb + (size_t)i * N + jn];
    }
    const int n = d >= 2 ? space_order(d) : (cls == kRegular ? kRegular01 : kNear01);
    const int o = gauss_offset(n);
    for (int a = 0; a < n; ++a) {
      const double xi = c_tab.gx[o + a], wa = c_tab.gw[o + a];
      for (int b = 0; b < n; ++b) {
        const double eta = c_tab.gx[o + b];
        const double dx = (abx + xi * eax) - eta * ebx;
        const double dy = (aby + xi * eay) - eta * eby;
        const double r2 = dx * dx + dy * dy;
        const double c = 0.25 * alpha * r2;
        double k, dk;
        if (d < 2) dlag01<OP == STBEM_OP_V ? kV : kKq>(c, d, ht, alpha, &k, &dk);
        else dlag2<OP == STBEM_OP_V ? kV : kKq>(c, d, alpha, LN, &k, &dk);
        const double phi = W0 * (1.0 - eta) + W1 * eta;
        const double wpt = wa * c_tab.gw[o + b] * phi;
        double gc;
        if (OP == STBEM_OP_V) {
          val += wpt * k;
          gc = wpt * dk;
        } else {
          const double qn = qab + xi * qea;
          val += wpt * qn * k;
          gc = wpt * qn * dk;
          const double gq = wpt * k;
          const double tau = (dx * tbx + dy * tby) * inv_lb;
          Q += gq;
          QX += gq * xi;
          QE += gq * eta;
          QT += gq * tau;
        }
        TA[0] += gc * dx;
        TA[1] += gc * dy;
        TX[0] += gc * xi * dx;
        TX[1] += gc * xi * dy;
        TE[0] += gc * eta * dx;
        TE[1] += gc * eta * dy;
        al += gc * r2;
      }
    }
  }
  if (!live) return;
  double* o = out + ((size_t)blockIdx.y * npair + p) * kVals;
  if (skip) {
    for (int q = 0; q < kVals; ++q) o[q] = 0.0;
    return;
  }
  // roles: c_r = (1 - xi, xi, -(1 - eta), -eta); K: dq coefficients
  // (1 - xi, xi, -(1 - eta) + tau, -eta - tau) times n_B
  const double T[4][2] = {{TA[0] - TX[0], TA[1] - TX[1]}, {TX[0], TX[1]},
                          {-TA[0] + TE[0], -TA[1] + TE[1]}, {-TE[0], -TE[1]}};
  const double Qr[4] = {Q - QX, QX, -Q + QE + QT, -QE - QT};
  finish_roles<OP>(A, B, alpha, val, T, Qr, al, o);
}

// ---- identical / shared-vertex pairs, lags 0 and 1 ---------------------------------
// Slot s = kind N + i: kind 0 (i, i) [V], kind 1 (i, i+1) [V (each unordered
// pair once) and K], kind 2 (i, i-1) [K].
template <int OP>
__global__ void __launch_bounds__(kGradThreads) k_grad_singular(DevMesh M, const double* __restrict__ C,
                                                                double* __restrict__ out) {
  constexpr int NV = 14;
  __shared__ double red[NV][kGradThreads];
  const int N = M.N;
  const double ht = M.ht, alpha = M.alpha;
  const int slot = blockIdx.x, kind = slot / N, i = slot % N;
  const bool active = OP == STBEM_OP_V ? kind < 2 : kind > 0;
  const int j = kind == 0 ? i : (kind == 1 ? (i + 1) % N : (i - 1 + N) % N);
  const int cls = kind == 0 ? kIdentical : (kind == 1 ? kAdjNext : kAdjPrev);
  const Piece A = seg_piece(M, i), B = seg_piece(M, j);
  const double tbx = (B.x1 - B.x0) / B.len, tby = (B.y1 - B.y0) / B.len;
  double val = 0.0, al = 0.0, T[4][2] = {}, Q[4] = {};
  if (active) {
    const int np = singular_points(cls);
    for (int d = 0; d < 2 && d < M.n_t; ++d) {
      const size_t cb = (size_t)d * N * N;
      double W0, W1;
      if (OP == STBEM_OP_V) {
        W0 = kind == 0 ? C[cb + (size_t)i * N + i] : C[cb + (size_t)i * N + j] + C[cb + (size_t)j * N + i];
        W1 = W0;
      } else {
        W0 = C[cb + (size_t)i * N + j];
        W1 = C[cb + (size_t)i * N + (j + 1) % N];
      }
      for (int p = threadIdx.x; p < np; p += kGradThreads) {
        double xi, eta, w, dx, dy, cr[4];
        singular_point_coef(cls, p, A, B, &xi, &eta, &w, &dx, &dy, cr);
        const double r2 = dx * dx + dy * dy;
        const double c = 0.25 * alpha * r2;
        double k, dk;
        dlag01<OP == STBEM_OP_V ? kV : kKq>(c, d, ht, alpha, &k, &dk);
        const double wpt = w * (W0 * (1.0 - eta) + W1 * eta);
        double gc;
        if (OP == STBEM_OP_V) {
          val += wpt * k;
          gc = wpt * dk;
        } else {
          const double qn = dx * B.nx + dy * B.ny;
          val += wpt * qn * k;
          gc = wpt * qn * dk;
          const double gq = wpt * k;
          const double tau = (dx * tbx + dy * tby) / B.len;
          Q[0] += gq * cr[0];
          Q[1] += gq * cr[1];
          Q[2] += gq * (cr[2] + tau);
          Q[3] += gq * (cr[3] - tau);
        }
        for (int r = 0; r < 4; ++r) {
          T[r][0] += gc * cr[r] * dx;
          T[r][1] += gc * cr[r] * dy;
        }
        al += gc * r2;
      }
    }
  }
  double v[NV] = {val, al, T[0][0], T[0][1], T[1][0], T[1][1], T[2][0], T[2][1], T[3][0], T[3][1],
                  Q[0], Q[1], Q[2], Q[3]};
  for (int q = 0; q < NV; ++q) red[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int s = kGradThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < NV; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* o = out + (size_t)slot * kVals;
    if (!active) {
      for (int q = 0; q < kVals; ++q) o[q] = 0.0;
      return;
    }
    const double TT[4][2] = {{red[2][0], red[3][0]}, {red[4][0], red[5][0]},
                             {red[6][0], red[7][0]}, {red[8][0], red[9][0]}};
    const double QQ[4] = {red[10][0], red[11][0], red[12][0], red[13][0]};
    finish_roles<OP>(A, B, alpha, red[0][0], TT, QQ, red[1][0], o);
  }
}

// ---- datum and mass terms ---------------------------------------------------------
// gbar[m][p] += (1/2 M_h)^T lambda = ht (h_p lam_p + h_{p-1} lam_{p-1}) / 4
__global__ void k_half_mass_T_add(DevMesh M, const double* __restrict__ lam, double* __restrict__ gbar) {
  const int N = M.N;
  const size_t total = (size_t)M.n_t * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % N);
    const size_t row = e - p;
    const int pm = (p - 1 + N) % N;
    gbar[e] += 0.25 * M.ht * (M.slen[p] * lam[e] + M.slen[pm] * lam[row + pm]);
  }
}

// per vertex p: gbar^T dg with a_p = alpha |x_p - y*|^2 / 4 and
// dg[n][p]/da = alpha / (4 pi ht) (e^{-a/t_n} - e^{-a/t_{n+1}}) / a,
// dg/dx_p = dg/da (alpha/2)(x_p - y*),  dg/dalpha = g / alpha + dg/da |x_p - y*|^2 / 4
__global__ void k_grad_datum(DevMesh M, double ysx, double ysy, const double* __restrict__ g,
                             const double* __restrict__ gbar, double* __restrict__ gv) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = M.N;
  if (p >= N) return;
  const double rx = M.vx[p] - ysx, ry = M.vy[p] - ysy;
  const double rho2 = rx * rx + ry * ry;
  const double a = M.alpha * rho2 / 4.0;
  const double pre = M.alpha / (kFourPi * M.ht) / a;
  double s = 0.0, sg = 0.0, e0 = 0.0;
  for (int n = 0; n < M.n_t; ++n) {
    const double e1 = exp_neg_fast(a / ((double)(n + 1) * M.ht));
    const double gb = gbar[(size_t)n * N + p];
    s += gb * pre * (e0 - e1);
    sg += gb * g[(size_t)n * N + p];
    e0 = e1;
  }
  gv[3 * p] = s * 0.5 * M.alpha * rx;
  gv[3 * p + 1] = s * 0.5 * M.alpha * ry;
  gv[3 * p + 2] = sg / M.alpha + s * rho2 / 4.0;
}

// per segment i: sum_m lam[m][i] ht (g[m][i] + g[m][i+1]) / 4 (times dh_i)
__global__ void k_grad_mass(DevMesh M, const double* __restrict__ lam, const double* __restrict__ g,
                            double* __restrict__ sm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = M.N;
  if (i >= N) return;
  const int ip = (i + 1) % N;
  double s = 0.0;
  for (int m = 0; m < M.n_t; ++m)
    s += lam[(size_t)m * N + i] * 0.25 * M.ht * (g[(size_t)m * N + i] + g[(size_t)m * N + ip]);
  sm[i] = s;
}

// ---- per-vertex gather ---------------------------------------------------------------
__global__ void __launch_bounds__(kGradThreads) k_grad_gather(DevMesh M, int nchunks, const double* __restrict__ tV,
                                                              const double* __restrict__ tK,
                                                              const double* __restrict__ sV,
                                                              const double* __restrict__ sK,
                                                              const double* __restrict__ gv,
                                                              const double* __restrict__ sm,
                                                              double* __restrict__ dxy) {
  __shared__ double red[2][kGradThreads];
  const int N = M.N, k = blockIdx.x;
  const int kp = (k - 1 + N) % N;
  const long long nV = (long long)N * (N + 1) / 2, nK = (long long)N * N;
  double sx = 0.0, sy = 0.0;
  // V tensor pairs (i <= j): A0 (k, j >= k), A1 (kp, j >= kp), B0 (i <= k, k), B1 (i <= kp, kp)
  const int cnt[4] = {N - k, N - kp, k + 1, kp + 1};
  for (int r = 0; r < 4; ++r) {
    for (int e = threadIdx.x; e < cnt[r] * nchunks; e += kGradThreads) {
      const int c = e / cnt[r], u = e % cnt[r];
      long long p;
      if (r == 0) p = tri_start(k, N) + u;
      else if (r == 1) p = tri_start(kp, N) + u;
      else if (r == 2) p = tri_start(u, N) + (k - u);
      else p = tri_start(u, N) + (kp - u);
      const double* o = tV + ((size_t)c * nV + p) * kVals + 2 * r;
      sx -= o[0];
      sy -= o[1];
    }
  }
  // K tensor pairs (all ordered): A0 (k, j), A1 (kp, j), B0 (i, k), B1 (i, kp)
  for (int r = 0; r < 4; ++r) {
    for (int e = threadIdx.x; e < N * nchunks; e += kGradThreads) {
      const int c = e / N, u = e % N;
      const long long p = r == 0 ? (long long)k * N + u
                          : r == 1 ? (long long)kp * N + u
                          : r == 2 ? (long long)u * N + k
                                   : (long long)u * N + kp;
      const double* o = tK + ((size_t)c * nK + p) * kVals + 2 * r;
      sx += o[0];
      sy += o[1];
    }
  }
  // singular slots: every slot and role whose vertex is k
  for (int e = threadIdx.x; e < 3 * N; e += kGradThreads) {
    const int kind = e / N, i = e % N;
    const int j = kind == 0 ? i : (kind == 1 ? (i + 1) % N : (i - 1 + N) % N);
    const int node[4] = {i, (i + 1) % N, j, (j + 1) % N};
    for (int r = 0; r < 4; ++r) {
      if (node[r] != k) continue;
      sx += sK[(size_t)e * kVals + 2 * r] - sV[(size_t)e * kVals + 2 * r];
      sy += sK[(size_t)e * kVals + 2 * r + 1] - sV[(size_t)e * kVals + 2 * r + 1];
    }
  }
  red[0][threadIdx.x] = sx;
  red[1][threadIdx.x] = sy;
  __syncthreads();
  for (int s = kGradThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // datum and mass: h_{k-1} grows with x_k along t_{k-1}, h_k shrinks along t_k
    const double tpx = (M.sx1[kp] - M.sx0[kp]) / M.slen[kp], tpy = (M.sy1[kp] - M.sy0[kp]) / M.slen[kp];
    const double tkx = (M.sx1[k] - M.sx0[k]) / M.slen[k], tky = (M.sy1[k] - M.sy0[k]) / M.slen[k];
    dxy[2 * k] = red[0][0] + gv[3 * k] + sm[kp] * tpx - sm[k] * tkx;
    dxy[2 * k + 1] = red[1][0] + gv[3 * k + 1] + sm[kp] * tpy - sm[k] * tky;
  }
}

__global__ void __launch_bounds__(1024) k_grad_alpha(int N, int nchunks, const double* __restrict__ tV,
                                                     const double* __restrict__ tK, const double* __restrict__ sV,
                                                     const double* __restrict__ sK, const double* __restrict__ gv,
                                                     double* __restrict__ dalpha) {
  __shared__ double red[1024];
  const long long nV = (long long)nchunks * N * (N + 1) / 2, nK = (long long)nchunks * N * N;
  double s = 0.0;
  for (long long e = threadIdx.x; e < nV; e += blockDim.x) s -= tV[e * kVals + 8];
  for (long long e = threadIdx.x; e < nK; e += blockDim.x) s += tK[e * kVals + 8];
  for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) s += sK[(size_t)e * kVals + 8] - sV[(size_t)e * kVals + 8];
  for (int e = threadIdx.x; e < N; e += blockDim.x) s += gv[3 * e + 2];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *dalpha = red[0];
}

struct GradWork {
  double *CV, *CK, *gbar, *tV, *tK, *sV, *sK, *gv, *sm;
  void* apply;
};

size_t carve_grad(int nt, int N, void* base, GradWork* w) {
  const int nchunks = (nt + kLagChunk - 1) / kLagChunk;
  const size_t nn = (size_t)nt * N * N, v = (size_t)nt * N;
  const size_t nV = (size_t)N * (N + 1) / 2, nK = (size_t)N * N;
  size_t off = 0;
  auto take = [&](size_t count) {
    double* p = base ? reinterpret_cast<double*>(static_cast<char*>(base) + off) : nullptr;
    off += ((count * sizeof(double) + 255) / 256) * 256;
    return p;
  };
  GradWork g;
  g.CV = take(nn);
  g.CK = take(nn);
  g.gbar = take(v);
  g.tV = take((size_t)nchunks * nV * kVals);
  g.tK = take((size_t)nchunks * nK * kVals);
  g.sV = take((size_t)3 * N * kVals);
  g.sK = take((size_t)3 * N * kVals);
  g.gv = take((size_t)3 * N);
  g.sm = take((size_t)N);
  g.apply = base ? static_cast<char*>(base) + off : nullptr;
  off += apply_workspace_bytes(nt, N, 1);
  if (w) *w = g;
  return off;
}

}  // namespace

size_t grad_workspace_bytes(int nt, int N) { return carve_grad(nt, N, nullptr, nullptr); }

cudaError_t upload_grad_rule_tables(const RuleTables& t, cudaStream_t s) {
  cudaError_t e = cudaMemcpyToSymbolAsync(c_tab, &t, sizeof(RuleTables), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

cudaError_t grad_launch(const DevMesh& M, const double* K, double ysx, double ysy, const double* g,
                        const double* w, const double* lam, double* dxy, double* dalpha, void* work,
                        cudaStream_t s) {
  const int N = M.N, nt = M.n_t;
  GradWork W;
  carve_grad(nt, N, work, &W);
  const int nchunks = (nt + kLagChunk - 1) / kLagChunk;
  const dim3 cgrid((N + kCT - 1) / kCT, (N + kCT - 1) / kCT, nt);
  k_corr<<<cgrid, 256, 0, s>>>(nt, N, lam, w, W.CV);
  k_corr<<<cgrid, 256, 0, s>>>(nt, N, lam, g, W.CK);
  count_launches(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // gbar = K^T lambda + (1/2 M)^T lambda
  e = apply_launch(STBEM_F64, true, nt, N, K, 1, lam, W.gbar, W.apply, s);
  if (e != cudaSuccess) return e;
  const size_t v = (size_t)nt * N;
  const int vb = (int)((v + 255) / 256 < 4096 ? (v + 255) / 256 : 4096);
  k_half_mass_T_add<<<vb, 256, 0, s>>>(M, lam, W.gbar);
  k_grad_datum<<<(N + 127) / 128, 128, 0, s>>>(M, ysx, ysy, g, W.gbar, W.gv);
  k_grad_mass<<<(N + 127) / 128, 128, 0, s>>>(M, lam, g, W.sm);
  k_grad_singular<STBEM_OP_V><<<3 * N, kGradThreads, 0, s>>>(M, W.CV, W.sV);
  k_grad_singular<STBEM_OP_K><<<3 * N, kGradThreads, 0, s>>>(M, W.CK, W.sK);
  const long long nV = (long long)N * (N + 1) / 2, nK = (long long)N * N;
  k_grad_tensor<STBEM_OP_V><<<dim3((unsigned)((nV + kGradThreads - 1) / kGradThreads), nchunks), kGradThreads, 0,
                              s>>>(M, W.CV, W.tV);
  k_grad_tensor<STBEM_OP_K><<<dim3((unsigned)((nK + kGradThreads - 1) / kGradThreads), nchunks), kGradThreads, 0,
                              s>>>(M, W.CK, W.tK);
  k_grad_gather<<<N, kGradThreads, 0, s>>>(M, nchunks, W.tV, W.tK, W.sV, W.sK, W.gv, W.sm, dxy);
  k_grad_alpha<<<1, 1024, 0, s>>>(N, nchunks, W.tV, W.tK, W.sV, W.sK, W.gv, dalpha);
  count_launches(9);
  return cudaGetLastError();
}

}  // namespace stbem
