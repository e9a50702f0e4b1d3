// Device pieces shared by the assembly and its derivative (gradient) kernels:
// the boundary pieces, the pair classes of the quadrature rule, the points of
// the identical / shared-vertex rules and the per-lag Peano node tables.
// Each translation unit that includes this header owns a copy of the rule
// tables in constant memory (c_tab) and uploads it itself.
#pragma once
#include <cuda_runtime.h>

#include "assemble.h"
#include "rule.cuh"
#include "timeint.cuh"

namespace stbem {

static __constant__ RuleTables c_tab;

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

// ---- pair classes (lags 0 and 1) ----------------------------------------------
static __device__ double point_seg_dist(double px, double py, double sx0, double sy0, double sx1, double sy1) {
  const double ex = sx1 - sx0, ey = sy1 - sy0;
  const double L2 = ex * ex + ey * ey;
  double t = ((px - sx0) * ex + (py - sy0) * ey) / L2;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  const double qx = sx0 + t * ex, qy = sy0 + t * ey;
  return sqrt((px - qx) * (px - qx) + (py - qy) * (py - qy));
}

// Pair class on a closed ring of Rl pieces (piece k ends where k+1 starts).
static __device__ int pair_class(int Rl, int ia, int ib, const Piece& A, const Piece& B) {
  const int diff = ((ib - ia) % Rl + Rl) % Rl;
  if (diff == 0) return kIdentical;
  if (diff == 1) return kAdjNext;
  if (diff == Rl - 1) return kAdjPrev;
  const int rd = diff < Rl - diff ? diff : Rl - diff;
  if (rd == 2) return kNear;
  double g = point_seg_dist(A.x0, A.y0, B.x0, B.y0, B.x1, B.y1);
  g = fmin(g, point_seg_dist(A.x1, A.y1, B.x0, B.y0, B.x1, B.y1));
  g = fmin(g, point_seg_dist(B.x0, B.y0, A.x0, A.y0, A.x1, A.y1));
  g = fmin(g, point_seg_dist(B.x1, B.y1, A.x0, A.y0, A.x1, A.y1));
  return g < kNearGapRatio * fmax(A.len, B.len) ? kNear : kRegular;
}

__device__ __forceinline__ int singular_points(int cls) {
  return cls == kIdentical ? 2 * kGradedN * kSingularInner : 2 * kGradedN * kDuffyAngular;
}

// Point p of the identical / shared-vertex rule: (xi, eta), weight, x - y.
__device__ __forceinline__ void singular_point(int cls, int p, const Piece& A, const Piece& B,
                                               double* xi, double* eta, double* w, double* dx, double* dy) {
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
  const double Rr = c_tab.grx[ir], WR = c_tab.grw[ir];
  const double T = c_tab.gx[o16 + it], WT = c_tab.gw[o16 + it];
  *w = WR * WT * Rr;
  const double xp = tri == 0 ? Rr : Rr * T;
  const double ep = tri == 0 ? Rr * T : Rr;
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

// ---- per-lag time-node tables (lags >= 2) ----------------------------------------
// For one lag d every Peano node s_g and its weight are shared by all points
// and pairs, so they are tabulated once per CTA with sigma = 1/s folded into
// the weights; a node then costs one exp and a few multiply-adds:
//   Peano V  = sum_g wv_g e_g,           wv = ht^2 wt sigma / (4 pi)
//   Peano K/q= sum_g wk_g e_g,           wk = ht^2 wt alpha sigma^2 / (8 pi)
//   Peano D1 = sum_g e_g (w3_g c - w2_g), w3 = ht^2 wt alpha sigma^3/(4 pi), w2 = .. sigma^2
// with e_g = exp(-c sigma_g), wt = Gauss weight x hat (tau on the left interval,
// 1 - tau on the right).  The closed form uses the node reciprocals 1/s too.
// Tables are computed in FP64 and stored in the compute precision R.
constexpr int kMaxNodes = 32;
template <typename R>
struct LagNodes {
  int n;                      // total nodes (left + right interval)
  R inv_dht;                  // 1 / (d ht): the closed/Peano switch
  R s[3], inv_s[3];           // (d+1) ht, d ht, (d-1) ht and reciprocals
  R sig[kMaxNodes], wv[kMaxNodes], wk[kMaxNodes], w3[kMaxNodes], w2[kMaxNodes];
};

template <typename R>
static __device__ void build_lag_nodes(LagNodes<R>& L, int d, double ht, double alpha) {
  const int nl = peano_order(d - 1), nr = peano_order(d);
  const int ol = gauss_offset(nl), orr = gauss_offset(nr);
  for (int g = threadIdx.x; g < nl + nr; g += blockDim.x) {
    double t, wt, s;
    if (g < nl) {
      t = c_tab.gx[ol + g];
      wt = c_tab.gw[ol + g] * t;
      s = ((double)(d - 1) + t) * ht;
    } else {
      t = c_tab.gx[orr + g - nl];
      wt = c_tab.gw[orr + g - nl] * (1.0 - t);
      s = ((double)d + t) * ht;
    }
    const double sig = 1.0 / s;
    const double base = ht * ht * wt;
    L.sig[g] = (R)sig;
    L.wv[g] = (R)(base * sig / kFourPi);
    L.wk[g] = (R)(base * alpha * sig * sig / (2.0 * kFourPi));
    L.w3[g] = (R)(base * alpha * sig * sig * sig / kFourPi);
    L.w2[g] = (R)(base * alpha * sig * sig / kFourPi);
  }
  if (threadIdx.x == 0) {
    L.n = nl + nr;
    L.inv_dht = (R)(1.0 / ((double)d * ht));
    const double s3[3] = {(double)(d + 1) * ht, (double)d * ht, (double)(d - 1) * ht};
    for (int k = 0; k < 3; ++k) {
      L.s[k] = (R)s3[k];
      L.inv_s[k] = (R)(1.0 / s3[k]);
    }
  }
}

// ---- time-node tables for L consecutive lags (lags >= 2) ----------------------------
// The Peano form of lag d integrates over the time intervals d - 1 (hat tau)
// and d (hat 1 - tau), so lags d0 .. d0 + L - 1 use the L + 1 intervals
// d0 - 1 .. d0 + L - 1 and each interior interval serves two lags; the closed
// form of those lags needs F at the L + 2 times (d0 - 1 + j) ht.  One table
// per CTA holds every node of those intervals with its weights for the left
// role (hat tau, the interval is lag k + 1's left) and the right role
// (hat 1 - tau, lag k's right).  Factors as in LagNodes.
constexpr int kMaxLagsML = 8;
constexpr int kMaxNodesML = 16 + 8 * kMaxLagsML;
template <typename R>
struct MLNodes {
  int d0, L;
  int off[kMaxLagsML + 2];            // interval i = 0..L starts at off[i]; off[L + 1] = total
  R inv_dht[kMaxLagsML];              // 1 / (d ht) of each lag (closed / Peano switch)
  R s[kMaxLagsML + 2], inv_s[kMaxLagsML + 2];   // (d0 - 1 + j) ht, j = 0..L+1
  R cthr[kMaxLagsML];                 // lag d0 + l uses the closed form where c > d^2 ht / 2
  R sig[kMaxNodesML];                 // 1 / s at the nodes (FP32 e^{-c sig}; FP64 fallback)
  R sigk[kMaxNodesML];                // (2048 / ln2) / s: FP64 e^{-c sig} = exp_prod_fast(c, sigk)
  R sigk_max;                         // the largest sigk (first node): c sigk_max < kExpProdMax
  R lv[kMaxNodesML], rv[kMaxNodesML], lk[kMaxNodesML], rk[kMaxNodesML];
  R l3[kMaxNodesML], r3[kMaxNodesML], l2[kMaxNodesML], r2[kMaxNodesML];
  double etab[sizeof(R) == 8 ? 2048 : 1];  // FP64: copy of the 2^{-j/2048} table (divergent reads)
};

template <typename R>
static __device__ void build_ml_nodes(MLNodes<R>& T, int d0, int L, double ht, double alpha) {
  int off[kMaxLagsML + 2];
  off[0] = 0;
  for (int i = 0; i <= L; ++i) off[i + 1] = off[i] + peano_order(d0 - 1 + i);
  const int total = off[L + 1];
  for (int g = threadIdx.x; g < total; g += blockDim.x) {
    int i = 0;
    while (off[i + 1] <= g) ++i;
    const int k = d0 - 1 + i, n = peano_order(k), o = gauss_offset(n);
    const double t = c_tab.gx[o + g - off[i]], w = c_tab.gw[o + g - off[i]];
    const double sv = ((double)k + t) * ht;
    const double sig = 1.0 / sv;
    const double base = ht * ht * w;
    const double fv = base * sig / kFourPi, fk = base * alpha * sig * sig / (2.0 * kFourPi);
    const double f3 = base * alpha * sig * sig * sig / kFourPi, f2 = base * alpha * sig * sig / kFourPi;
    T.sig[g] = (R)sig;
    T.sigk[g] = (R)(kInvLn2x2048 / sv);
    T.lv[g] = (R)(fv * t);
    T.rv[g] = (R)(fv * (1.0 - t));
    T.lk[g] = (R)(fk * t);
    T.rk[g] = (R)(fk * (1.0 - t));
    T.l3[g] = (R)(f3 * t);
    T.r3[g] = (R)(f3 * (1.0 - t));
    T.l2[g] = (R)(f2 * t);
    T.r2[g] = (R)(f2 * (1.0 - t));
  }
  if (sizeof(R) == 8)
    for (int j = threadIdx.x; j < 2048; j += blockDim.x) T.etab[j] = kExp2Tab2048[j];
  if (threadIdx.x == 0) {
    T.d0 = d0;
    T.L = L;
    // the nodes' s increase with g, so node 0 has the largest sigma
    T.sigk_max = (R)(kInvLn2x2048 / (((double)(d0 - 1) + c_tab.gx[gauss_offset(peano_order(d0 - 1))]) * ht));
    for (int l = 0; l < L; ++l) {
      const double d = (double)(d0 + l);
      T.cthr[l] = (R)(0.5 * d * (d * ht));
    }
    for (int i = 0; i <= L + 1; ++i) T.off[i] = off[i];
    for (int l = 0; l < L; ++l) T.inv_dht[l] = (R)(1.0 / ((double)(d0 + l) * ht));
    for (int j = 0; j <= L + 1; ++j) {
      const double sj = (double)(d0 - 1 + j) * ht;
      T.s[j] = (R)sj;
      T.inv_s[j] = (R)(1.0 / sj);
    }
  }
}

}  // namespace stbem
