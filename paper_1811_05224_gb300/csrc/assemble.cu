// Assembly of the block-Toeplitz lag blocks of V_h, K_h and D_h (FP64).
//
// Entries (Section 1 eq. (4); Section 2 Theorem and dual space Y_h):
//   V^(d)[i][j] = int_{g_i} int_{g_j} D2_d F_V
//   K^(d)[i][p] = sum_{j in {p, p-1}} int_{g_i} int_{g_j} D2_d F_K phi_p(y)
//   D^(d)[l][k] = sum_{a in supp psi_l, b in supp psi_k}
//                   psi_l'(a) psi_k'(b) int_a int_b D2_d F_V
//                 + (n_a . n_b) int_a int_b psi_l psi_k D2_d F_1
// (D in the integrated-by-parts form of the hypersingular operator, Section 2
// citing Costabel 1990 Thm 6.1; a, b half-segments on which psi is linear).
//
// Two kernels per operator:
//   * lags d >= 2: one thread per entry; tensor Gauss-Legendre of order
//     space_order(d) on every piece pair; time by closed form or Peano form.
//   * lags 0 and 1: one CTA per entry; pair classes select the regular, near,
//     identical (graded diagonal) or shared-vertex (Duffy, graded) rule; the
//     rule's points are strided over the threads and reduced in a fixed tree.
// V^(d) and D^(d) are symmetric: the entry with the smaller index first is
// evaluated and written to both triangles.
#include <cuda_runtime.h>

#include "assemble.h"
#include "rule.cuh"
#include "timeint.cuh"

namespace stbem {

__constant__ RuleTables c_tab;

// ---- piece access -----------------------------------------------------------
struct Piece {
  double x0, y0, x1, y1, len, nx, ny;
};

__device__ __forceinline__ Piece seg_piece(const DevMesh& M, int i) {
  Piece p;
  p.x0 = M.sx0[i]; p.y0 = M.sy0[i]; p.x1 = M.sx1[i]; p.y1 = M.sy1[i];
  p.len = M.slen[i]; p.nx = M.snx[i]; p.ny = M.sny[i];
  return p;
}
__device__ __forceinline__ Piece half_piece(const DevMesh& M, int i) {
  Piece p;
  p.x0 = M.hx0[i]; p.y0 = M.hy0[i]; p.x1 = M.hx1[i]; p.y1 = M.hy1[i];
  p.len = M.hlen[i]; p.nx = M.hnx[i]; p.ny = M.hny[i];
  return p;
}

// ---- fused time kernels for D (share E1/E2 and exp between F_V and F_1) ------
__device__ __forceinline__ void lag_kernel_D(double c, int d, double ht, double alpha,
                                             double* outv, double* out1) {
  const double* gx = c_tab.gx;
  const double* gw = c_tab.gw;
  if (d == 0) {
    double a, b;
    e1e2(c / ht, &a, &b);
    *outv = ht / kFourPi * (a - b);
    *out1 = alpha / kFourPi * a;
    return;
  }
  if (d == 1) {
    const double z = c / ht;
    if (z < 1.0) {
      *outv = lag1_series<kV>(z, ht, alpha);
      *out1 = lag1_series<k1>(z, ht, alpha);
      return;
    }
    double a2, b2, a1, b1;
    e1e2(c / (2.0 * ht), &a2, &b2);
    e1e2(c / ht, &a1, &b1);
    *outv = (2.0 * ht) / kFourPi * (a2 - b2) - 2.0 * (ht / kFourPi * (a1 - b1));
    *out1 = alpha / kFourPi * a2 - 2.0 * (alpha / kFourPi * a1);
    return;
  }
  const double zd = c / ((double)d * ht);
  if (zd > 0.5 * (double)d) {
    const double s3 = (double)(d + 1) * ht, s2 = (double)d * ht, s1 = (double)(d - 1) * ht;
    double a3, b3, a2, b2, a1, b1;
    e1e2(c / s3, &a3, &b3);
    e1e2(c / s2, &a2, &b2);
    e1e2(c / s1, &a1, &b1);
    *outv = (s3 / kFourPi * (a3 - b3) - 2.0 * (s2 / kFourPi * (a2 - b2))) + s1 / kFourPi * (a1 - b1);
    *out1 = (alpha / kFourPi * a3 - 2.0 * (alpha / kFourPi * a2)) + alpha / kFourPi * a1;
    return;
  }
  const int nl = peano_order(d - 1), nr = peano_order(d);
  const int ol = gauss_offset(nl), orr = gauss_offset(nr);
  double lv = 0.0, rv = 0.0, l1 = 0.0, r1 = 0.0;
  for (int g = 0; g < nl; ++g) {
    const double t = gx[ol + g];
    const double s = ((double)(d - 1) + t) * ht;
    const double e = exp(-c / s);
    const double wt = gw[ol + g] * t;
    lv += wt * (e / (kFourPi * s));
    l1 += wt * (alpha / kFourPi * e * (c / (s * s * s) - 1.0 / (s * s)));
  }
  for (int g = 0; g < nr; ++g) {
    const double t = gx[orr + g];
    const double s = ((double)d + t) * ht;
    const double e = exp(-c / s);
    const double wt = gw[orr + g] * (1.0 - t);
    rv += wt * (e / (kFourPi * s));
    r1 += wt * (alpha / kFourPi * e * (c / (s * s * s) - 1.0 / (s * s)));
  }
  *outv = ht * ht * (lv + rv);
  *out1 = ht * ht * (l1 + r1);
}

// ---- tensor rule on a piece pair (lags >= 2) -----------------------------------
// Returns int_a int_b k(x,y) fa(xi) fb(eta) for kernel K (V or K/q*q).
template <int K>
__device__ double tensor_pair(const Piece& A, const Piece& B, double fa0, double fa1,
                              double fb0, double fb1, int d, int n, double ht, double alpha) {
  const int o = gauss_offset(n);
  const double eax = A.x1 - A.x0, eay = A.y1 - A.y0;
  const double ebx = B.x1 - B.x0, eby = B.y1 - B.y0;
  const double abx = A.x0 - B.x0, aby = A.y0 - B.y0;
  double acc = 0.0;
  for (int a = 0; a < n; ++a) {
    const double xi = c_tab.gx[o + a];
    const double wa = c_tab.gw[o + a];
    const double fa = fa0 + (fa1 - fa0) * xi;
    for (int b = 0; b < n; ++b) {
      const double eta = c_tab.gx[o + b];
      const double w = wa * c_tab.gw[o + b];
      const double dx = (abx + xi * eax) - eta * ebx;
      const double dy = (aby + xi * eay) - eta * eby;
      const double r2 = dx * dx + dy * dy;
      const double c = 0.25 * alpha * r2;
      double k = lag_kernel<K>(c, d, ht, alpha, c_tab.gx, c_tab.gw);
      if (K == kKq) k = (dx * B.nx + dy * B.ny) * k;
      const double fb = fb0 + (fb1 - fb0) * eta;
      acc += w * k * fa * fb;
    }
  }
  return acc * A.len * B.len;
}

// Fused V-kernel and F_1-kernel integrals on a half-segment pair (D operator).
__device__ void tensor_pair_D(const Piece& A, const Piece& B, double fa0, double fa1,
                              double fb0, double fb1, int d, int n, double ht, double alpha,
                              double* IV, double* I1) {
  const int o = gauss_offset(n);
  const double eax = A.x1 - A.x0, eay = A.y1 - A.y0;
  const double ebx = B.x1 - B.x0, eby = B.y1 - B.y0;
  const double abx = A.x0 - B.x0, aby = A.y0 - B.y0;
  double accv = 0.0, acc1 = 0.0;
  for (int a = 0; a < n; ++a) {
    const double xi = c_tab.gx[o + a];
    const double wa = c_tab.gw[o + a];
    const double fa = fa0 + (fa1 - fa0) * xi;
    for (int b = 0; b < n; ++b) {
      const double eta = c_tab.gx[o + b];
      const double w = wa * c_tab.gw[o + b];
      const double dx = (abx + xi * eax) - eta * ebx;
      const double dy = (aby + xi * eay) - eta * eby;
      const double c = 0.25 * alpha * (dx * dx + dy * dy);
      double kv, k1v;
      lag_kernel_D(c, d, ht, alpha, &kv, &k1v);
      const double fb = fb0 + (fb1 - fb0) * eta;
      accv += w * kv * 1.0 * 1.0;
      acc1 += w * k1v * fa * fb;
    }
  }
  *IV = accv * A.len * B.len;
  *I1 = acc1 * A.len * B.len;
}

// ---- lags >= 2: one thread per entry ------------------------------------------
template <int OP, typename T>
__global__ void k_lag2(DevMesh M, int d_begin, int d_end, T* __restrict__ out) {
  const int N = M.N;
  const long long total = (long long)(d_end - d_begin) * N * N;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= total) return;
  const int j = (int)(tid % N);
  const int i = (int)((tid / N) % N);
  const int d = d_begin + (int)(tid / ((long long)N * N));
  const double ht = M.ht, alpha = M.alpha;
  const int n = space_order(d);
  double val = 0.0;
  if (OP == STBEM_OP_V) {
    if (i > j) return;
    val = tensor_pair<kV>(seg_piece(M, i), seg_piece(M, j), 1.0, 1.0, 1.0, 1.0, d, n, ht, alpha);
  } else if (OP == STBEM_OP_K) {
    const Piece A = seg_piece(M, i);
    const int jp = j, jm = (j - 1 + N) % N;
    if (jp != i) val += tensor_pair<kKq>(A, seg_piece(M, jp), 1.0, 1.0, 1.0, 0.0, d, n, ht, alpha);
    if (jm != i) val += tensor_pair<kKq>(A, seg_piece(M, jm), 1.0, 1.0, 0.0, 1.0, d, n, ht, alpha);
  } else {
    if (i > j) return;
    for (int ia = 0; ia < 4; ++ia) {
      const int pa = M.dpiece[4 * i + ia];
      const double a0 = M.dv0[4 * i + ia], a1 = M.dv1[4 * i + ia], ca = M.dcurl[4 * i + ia];
      const Piece A = half_piece(M, pa);
      for (int ib = 0; ib < 4; ++ib) {
        const int pb = M.dpiece[4 * j + ib];
        const double b0 = M.dv0[4 * j + ib], b1 = M.dv1[4 * j + ib], cb = M.dcurl[4 * j + ib];
        const Piece B = half_piece(M, pb);
        double IV, I1;
        tensor_pair_D(A, B, a0, a1, b0, b1, d, n, ht, alpha, &IV, &I1);
        const double nn = A.nx * B.nx + A.ny * B.ny;
        val += ca * cb * IV + nn * I1;
      }
    }
  }
  const size_t base = (size_t)d * N * N;
  out[base + (size_t)i * N + j] = (T)val;
  if ((OP == STBEM_OP_V || OP == STBEM_OP_D) && i != j) out[base + (size_t)j * N + i] = (T)val;
}

// ---- lags >= 2, K and D: tile kernels on piece-pair moments -------------------
// D: a CTA owns a kDT x kDT tile of entries (l, k); the pieces of the dual
// functions of its rows are the 2 kDT + 2 consecutive half-segments starting at
// 2 l0 - 1 (likewise for the columns).  Per lag it integrates every half-pair
// once into five moments -- the V kernel with weight 1 and the D time kernel
// with the bilinear basis (1-xi)(1-eta), (1-xi)eta, xi(1-eta), xi eta -- and
// then sums the 16 piece pairs of each entry from shared memory.
constexpr int kDT = 16;
constexpr int kDP = 2 * kDT + 2;          // half-segments per tile side
constexpr int kTileThreads = 256;

__device__ void pair_moments_D(const Piece& A, const Piece& B, int d, int n, double ht, double alpha,
                               double* mom) {
  const int o = gauss_offset(n);
  const double eax = A.x1 - A.x0, eay = A.y1 - A.y0;
  const double ebx = B.x1 - B.x0, eby = B.y1 - B.y0;
  const double abx = A.x0 - B.x0, aby = A.y0 - B.y0;
  double sv = 0.0, s00 = 0.0, s01 = 0.0, s10 = 0.0, s11 = 0.0;
  for (int a = 0; a < n; ++a) {
    const double xi = c_tab.gx[o + a];
    const double wa = c_tab.gw[o + a];
    for (int b = 0; b < n; ++b) {
      const double eta = c_tab.gx[o + b];
      const double w = wa * c_tab.gw[o + b];
      const double dx = (abx + xi * eax) - eta * ebx;
      const double dy = (aby + xi * eay) - eta * eby;
      const double c = 0.25 * alpha * (dx * dx + dy * dy);
      double kv, k1v;
      lag_kernel_D(c, d, ht, alpha, &kv, &k1v);
      sv += w * kv;
      const double wk = w * k1v;
      s00 += wk * (1.0 - xi) * (1.0 - eta);
      s01 += wk * (1.0 - xi) * eta;
      s10 += wk * xi * (1.0 - eta);
      s11 += wk * xi * eta;
    }
  }
  const double L = A.len * B.len;
  mom[0] = sv * L; mom[1] = s00 * L; mom[2] = s01 * L; mom[3] = s10 * L; mom[4] = s11 * L;
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_lag2_D(DevMesh M, int d_begin, int d_end, T* __restrict__ out) {
  __shared__ double mom[kDP * kDP][5];
  const int N = M.N, H = 2 * N;
  // upper-triangular tile pair from the linear block index
  int lt = 0, rem = blockIdx.x;
  const int nT = (N + kDT - 1) / kDT;
  while (rem >= nT - lt) { rem -= nT - lt; ++lt; }
  const int kt = lt + rem;
  const int l0 = lt * kDT, k0 = kt * kDT;
  const int tid = threadIdx.x;
  const double ht = M.ht, alpha = M.alpha;
  for (int d = d_begin + blockIdx.y; d < d_end; d += gridDim.y) {
    const int n = space_order(d);
    for (int p = tid; p < kDP * kDP; p += kTileThreads) {
      const int u = p / kDP, v = p % kDP;
      const int ga = ((2 * l0 - 1 + u) % H + H) % H;
      const int gb = ((2 * k0 - 1 + v) % H + H) % H;
      pair_moments_D(half_piece(M, ga), half_piece(M, gb), d, n, ht, alpha, mom[p]);
    }
    __syncthreads();
    if (tid < kDT * kDT) {
      const int s = tid / kDT, t = tid % kDT;
      const int l = l0 + s, k = k0 + t;
      // evaluate the smaller index first (symmetric block): on the diagonal
      // tile both ranges coincide, so (lo, hi) local offsets exist
      const int lo = l < k ? l : k, hi = l < k ? k : l;
      const int so = lo - l0, to = hi - k0;
      if (l < N && k < N && so >= 0 && to >= 0 && so < kDT && to < kDT) {
        double val = 0.0;
        for (int ia = 0; ia < 4; ++ia) {
          const int qa = 4 * lo + ia;
          const double ca = M.dcurl[qa], a0 = M.dv0[qa], a1 = M.dv1[qa];
          const int u = 2 * so + ia;
          const int ga = M.dpiece[qa];
          const double nax = M.hnx[ga], nay = M.hny[ga];
          for (int ib = 0; ib < 4; ++ib) {
            const int qb = 4 * hi + ib;
            const double cb = M.dcurl[qb], b0 = M.dv0[qb], b1 = M.dv1[qb];
            const int v = 2 * to + ib;
            const int gb = M.dpiece[qb];
            const double nn = nax * M.hnx[gb] + nay * M.hny[gb];
            const double* m = mom[u * kDP + v];
            const double I1 = a0 * (b0 * m[1] + b1 * m[2]) + a1 * (b0 * m[3] + b1 * m[4]);
            val += ca * cb * m[0] + nn * I1;
          }
        }
        const size_t base = (size_t)d * N * N;
        out[base + (size_t)l * N + k] = (T)val;
        if (lt != kt) out[base + (size_t)k * N + l] = (T)val;
      }
    }
    __syncthreads();
  }
}

// K: a CTA owns kKI x kKP entries (i, p); the trial segments are p0-1 .. p0+kKP-1.
// Moments per segment pair (i, j): int k (1 - eta) and int k eta, so that
// K[i][p] = Ma(i, p) + Mb(i, p-1) (identical pairs contribute 0).
constexpr int kKI = 16, kKP = 15, kKJ = kKP + 1;

template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_lag2_K(DevMesh M, int d_begin, int d_end, T* __restrict__ out) {
  __shared__ double mom[kKI * kKJ][2];
  const int N = M.N;
  const int nP = (N + kKP - 1) / kKP;
  const int it = blockIdx.x / nP, pt = blockIdx.x % nP;
  const int i0 = it * kKI, p0 = pt * kKP;
  const int tid = threadIdx.x;
  const double ht = M.ht, alpha = M.alpha;
  for (int d = d_begin + blockIdx.y; d < d_end; d += gridDim.y) {
    const int n = space_order(d);
    const int o = gauss_offset(n);
    for (int p = tid; p < kKI * kKJ; p += kTileThreads) {
      const int si = p / kKJ, sj = p % kKJ;
      const int i = i0 + si;
      const int j = ((p0 - 1 + sj) % N + N) % N;
      double ma = 0.0, mb = 0.0;
      if (i < N && j != i) {
        const Piece A = seg_piece(M, i), B = seg_piece(M, j);
        const double eax = A.x1 - A.x0, eay = A.y1 - A.y0;
        const double ebx = B.x1 - B.x0, eby = B.y1 - B.y0;
        const double abx = A.x0 - B.x0, aby = A.y0 - B.y0;
        for (int a = 0; a < n; ++a) {
          const double xi = c_tab.gx[o + a];
          const double wa = c_tab.gw[o + a];
          for (int b = 0; b < n; ++b) {
            const double eta = c_tab.gx[o + b];
            const double w = wa * c_tab.gw[o + b];
            const double dx = (abx + xi * eax) - eta * ebx;
            const double dy = (aby + xi * eay) - eta * eby;
            const double c = 0.25 * alpha * (dx * dx + dy * dy);
            const double k = (dx * B.nx + dy * B.ny) * lag_kernel<kKq>(c, d, ht, alpha, c_tab.gx, c_tab.gw);
            const double wk = w * k;
            ma += wk * (1.0 - eta);
            mb += wk * eta;
          }
        }
        ma *= A.len * B.len;
        mb *= A.len * B.len;
      }
      mom[p][0] = ma;
      mom[p][1] = mb;
    }
    __syncthreads();
    if (tid < kKI * kKP) {
      const int si = tid / kKP, sp = tid % kKP;
      const int i = i0 + si, p = p0 + sp;
      if (i < N && p < N) {
        const double val = mom[si * kKJ + sp + 1][0] + mom[si * kKJ + sp][1];
        out[(size_t)d * N * N + (size_t)i * N + p] = (T)val;
      }
    }
    __syncthreads();
  }
}

// ---- lags 0, 1: one CTA per entry -----------------------------------------------
constexpr int kLag01Threads = 128;

__device__ double point_seg_dist(double px, double py, double sx0, double sy0, double sx1, double sy1) {
  const double ex = sx1 - sx0, ey = sy1 - sy0;
  const double L2 = ex * ex + ey * ey;
  double t = ((px - sx0) * ex + (py - sy0) * ey) / L2;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  const double qx = sx0 + t * ex, qy = sy0 + t * ey;
  return sqrt((px - qx) * (px - qx) + (py - qy) * (py - qy));
}

// Pair class on a closed ring of R pieces (piece k ends where k+1 starts).
__device__ int pair_class(int R, int ia, int ib, const Piece& A, const Piece& B) {
  const int diff = ((ib - ia) % R + R) % R;
  if (diff == 0) return kIdentical;
  if (diff == 1) return kAdjNext;
  if (diff == R - 1) return kAdjPrev;
  const int rd = diff < R - diff ? diff : R - diff;
  if (rd == 2) return kNear;
  double g = point_seg_dist(A.x0, A.y0, B.x0, B.y0, B.x1, B.y1);
  g = fmin(g, point_seg_dist(A.x1, A.y1, B.x0, B.y0, B.x1, B.y1));
  g = fmin(g, point_seg_dist(B.x0, B.y0, A.x0, A.y0, A.x1, A.y1));
  g = fmin(g, point_seg_dist(B.x1, B.y1, A.x0, A.y0, A.x1, A.y1));
  return g < kNearGapRatio * fmax(A.len, B.len) ? kNear : kRegular;
}

__device__ __forceinline__ int class_points(int cls) {
  if (cls == kRegular) return kRegular01 * kRegular01;
  if (cls == kNear) return kNear01 * kNear01;
  if (cls == kIdentical) return 2 * kGradedN * kSingularInner;
  return 2 * kGradedN * kDuffyAngular;
}

// Point `p` of the class rule: local parameters (xi, eta), weight, and x - y.
__device__ __forceinline__ void class_point(int cls, int p, const Piece& A, const Piece& B,
                                            const double* grx, const double* grw,
                                            double* xi, double* eta, double* w, double* dx, double* dy) {
  const double eax = A.x1 - A.x0, eay = A.y1 - A.y0;
  const double ebx = B.x1 - B.x0, eby = B.y1 - B.y0;
  if (cls == kRegular || cls == kNear) {
    const int n = cls == kRegular ? kRegular01 : kNear01;
    const int o = gauss_offset(n);
    const int a = p / n, b = p % n;
    *xi = c_tab.gx[o + a];
    *eta = c_tab.gx[o + b];
    *w = c_tab.gw[o + a] * c_tab.gw[o + b];
    *dx = ((A.x0 - B.x0) + *xi * eax) - *eta * ebx;
    *dy = ((A.y0 - B.y0) + *xi * eay) - *eta * eby;
    return;
  }
  if (cls == kIdentical) {
    const int per = kGradedN * kSingularInner;
    const int tri = p / per, rem = p % per;
    const int iu = rem / kSingularInner, it = rem % kSingularInner;
    const int o4 = gauss_offset(kSingularInner);
    const double U = grx[iu], WU = grw[iu];
    const double TA = c_tab.gx[o4 + it], WT = c_tab.gw[o4 + it];
    const double lo = (1.0 - U) * TA;
    *w = WU * WT * (1.0 - U);
    const double u = tri == 0 ? U : -U;
    *xi = tri == 0 ? lo + U : lo;
    *eta = tri == 0 ? lo : lo + U;
    *dx = u * eax;
    *dy = u * eay;
    return;
  }
  const int per = kGradedN * kDuffyAngular;
  const int tri = p / per, rem = p % per;
  const int ir = rem / kDuffyAngular, it = rem % kDuffyAngular;
  const int o16 = gauss_offset(kDuffyAngular);
  const double R = grx[ir], WR = grw[ir];
  const double T = c_tab.gx[o16 + it], WT = c_tab.gw[o16 + it];
  *w = WR * WT * R;
  const double xp = tri == 0 ? R : R * T;
  const double ep = tri == 0 ? R * T : R;
  if (cls == kAdjNext) {   // end of A == start of B
    *xi = 1.0 - xp;
    *eta = ep;
    *dx = -xp * eax - ep * ebx;
    *dy = -xp * eay - ep * eby;
  } else {                 // start of A == end of B
    *xi = xp;
    *eta = 1.0 - ep;
    *dx = xp * eax + ep * ebx;
    *dy = xp * eay + ep * eby;
  }
}

__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = kLag01Threads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Integral of the lag-0/1 kernel(s) over one piece pair with class rules.
template <int K>
__device__ void class_pair(const Piece& A, const Piece& B, int cls, double fa0, double fa1,
                           double fb0, double fb1, int d, double ht, double alpha,
                           const double* grx, const double* grw, double* red,
                           double* out0, double* out1) {
  const int np = class_points(cls);
  double s0 = 0.0, s1 = 0.0;
  for (int p = threadIdx.x; p < np; p += kLag01Threads) {
    double xi, eta, w, dx, dy;
    class_point(cls, p, A, B, grx, grw, &xi, &eta, &w, &dx, &dy);
    const double c = 0.25 * alpha * (dx * dx + dy * dy);
    const double fa = fa0 + (fa1 - fa0) * xi;
    const double fb = fb0 + (fb1 - fb0) * eta;
    if (K == k1) {   // D: both kernels
      double kv, k1v;
      lag_kernel_D(c, d, ht, alpha, &kv, &k1v);
      s0 += w * kv * 1.0 * 1.0;
      s1 += w * k1v * fa * fb;
    } else {
      double k = lag_kernel<K>(c, d, ht, alpha, c_tab.gx, c_tab.gw);
      if (K == kKq) k = (dx * B.nx + dy * B.ny) * k;
      s0 += w * k * fa * fb;
    }
  }
  *out0 = block_sum(s0, red) * A.len * B.len;
  if (K == k1) *out1 = block_sum(s1, red) * A.len * B.len;
}

template <int OP, typename T>
__global__ void __launch_bounds__(kLag01Threads) k_lag01(DevMesh M, T* __restrict__ out) {
  __shared__ double grx[kGradedN], grw[kGradedN];
  __shared__ double red[kLag01Threads];
  const int N = M.N;
  const int e = blockIdx.x;
  const int i = e / N, j = e % N;
  const int d = blockIdx.y;
  if ((OP == STBEM_OP_V || OP == STBEM_OP_D) && i > j) return;
  for (int t = threadIdx.x; t < kGradedN; t += kLag01Threads) {
    grx[t] = c_tab.grx[t];
    grw[t] = c_tab.grw[t];
  }
  __syncthreads();
  const double ht = M.ht, alpha = M.alpha;
  double val = 0.0, dummy;
  if (OP == STBEM_OP_V) {
    const Piece A = seg_piece(M, i), B = seg_piece(M, j);
    const int cls = pair_class(N, i, j, A, B);
    class_pair<kV>(A, B, cls, 1.0, 1.0, 1.0, 1.0, d, ht, alpha, grx, grw, red, &val, &dummy);
  } else if (OP == STBEM_OP_K) {
    const Piece A = seg_piece(M, i);
    const int js[2] = {j, (j - 1 + N) % N};
    const double w0[2] = {1.0, 0.0}, w1[2] = {0.0, 1.0};
    for (int t = 0; t < 2; ++t) {
      if (js[t] == i) continue;
      const Piece B = seg_piece(M, js[t]);
      const int cls = pair_class(N, i, js[t], A, B);
      double v;
      class_pair<kKq>(A, B, cls, 1.0, 1.0, w0[t], w1[t], d, ht, alpha, grx, grw, red, &v, &dummy);
      val += v;
    }
  } else {
    for (int ia = 0; ia < 4; ++ia) {
      const int pa = M.dpiece[4 * i + ia];
      const double a0 = M.dv0[4 * i + ia], a1 = M.dv1[4 * i + ia], ca = M.dcurl[4 * i + ia];
      const Piece A = half_piece(M, pa);
      for (int ib = 0; ib < 4; ++ib) {
        const int pb = M.dpiece[4 * j + ib];
        const double b0 = M.dv0[4 * j + ib], b1 = M.dv1[4 * j + ib], cb = M.dcurl[4 * j + ib];
        const Piece B = half_piece(M, pb);
        const int cls = pair_class(2 * N, pa, pb, A, B);
        double IV, I1;
        class_pair<k1>(A, B, cls, a0, a1, b0, b1, d, ht, alpha, grx, grw, red, &IV, &I1);
        const double nn = A.nx * B.nx + A.ny * B.ny;
        val += ca * cb * IV + nn * I1;
      }
    }
  }
  if (threadIdx.x == 0) {
    const size_t base = (size_t)d * N * N;
    out[base + (size_t)i * N + j] = (T)val;
    if ((OP == STBEM_OP_V || OP == STBEM_OP_D) && i != j) out[base + (size_t)j * N + i] = (T)val;
  }
}

// ---- host side ----------------------------------------------------------------
cudaError_t upload_rule_tables(const RuleTables& t, cudaStream_t s) {
  return cudaMemcpyToSymbolAsync(c_tab, &t, sizeof(RuleTables), 0, cudaMemcpyHostToDevice, s);
}

template <int OP, typename T>
static cudaError_t launch_op(const DevMesh& M, T* out, cudaStream_t s) {
  const int N = M.N, nt = M.n_t;
  const int nl = nt < 2 ? nt : 2;
  k_lag01<OP, T><<<dim3(N * N, nl), kLag01Threads, 0, s>>>(M, out);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (nt > 2) {
    // chunk the lag range so that one launch stays well below a second
    const int chunk = 64;
    for (int d0 = 2; d0 < nt; d0 += chunk) {
      const int d1 = d0 + chunk < nt ? d0 + chunk : nt;
      if (OP == STBEM_OP_V) {
        const long long total = (long long)(d1 - d0) * N * N;
        const int threads = 128;
        const long long blocks = (total + threads - 1) / threads;
        k_lag2<OP, T><<<(unsigned)blocks, threads, 0, s>>>(M, d0, d1, out);
      } else if (OP == STBEM_OP_K) {
        const int tiles = ((N + kKI - 1) / kKI) * ((N + kKP - 1) / kKP);
        k_lag2_K<T><<<dim3(tiles, d1 - d0), kTileThreads, 0, s>>>(M, d0, d1, out);
      } else {
        const int nT = (N + kDT - 1) / kDT;
        const int tiles = nT * (nT + 1) / 2;
        k_lag2_D<T><<<dim3(tiles, d1 - d0), kTileThreads, 0, s>>>(M, d0, d1, out);
      }
      count_launches(1);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t assemble_launch(const DevMesh& M, int op, int prec, void* out, cudaStream_t s) {
  if (prec == STBEM_F64) {
    double* o = static_cast<double*>(out);
    if (op == STBEM_OP_V) return launch_op<STBEM_OP_V>(M, o, s);
    if (op == STBEM_OP_K) return launch_op<STBEM_OP_K>(M, o, s);
    return launch_op<STBEM_OP_D>(M, o, s);
  }
  float* o = static_cast<float*>(out);
  if (op == STBEM_OP_V) return launch_op<STBEM_OP_V>(M, o, s);
  if (op == STBEM_OP_K) return launch_op<STBEM_OP_K>(M, o, s);
  return launch_op<STBEM_OP_D>(M, o, s);
}

}  // namespace stbem
