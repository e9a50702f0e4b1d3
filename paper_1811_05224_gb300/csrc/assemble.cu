// Assembly of the block-Toeplitz lag blocks of V_h, K_h and D_h.
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
// One tile kernel per operator.  A CTA owns a tile of entries at one lag and
// first integrates every piece pair the tile needs into moments in shared
// memory, then sums the moments of each entry:
//   V: 16 x 16 entries = the segment pairs themselves (symmetric tiles only);
//   K: 16 x 15 entries from 16 x 16 segment pairs, moments int k (1 - eta)
//      and int k eta, so K[i][p] = Ma(i, p) + Mb(i, p-1);
//   D: 16 x 16 entries from 34 x 34 half-segment pairs, moments int k_V and
//      int k_1 times (1-xi)(1-eta), (1-xi)eta, xi(1-eta), xi eta.
// Phase 1 gives each thread whole pairs (tensor Gauss-Legendre) in the compute
// precision R; at lags 0 and 1 identical pieces and pieces sharing a vertex are
// deferred to phase 2, where one warp integrates one pair with the graded /
// Duffy rules in FP64 (the small-z E1 terms cancel there) and reduces with
// shuffles.  V^(d) and D^(d) are symmetric: the entry with the smaller index
// first is evaluated and written to both triangles.
//
// Precisions: R = double, T = double (STBEM_F64); R = float, T = float
// (STBEM_F32: FP32 arithmetic everywhere except the deferred FP64 pairs).
#include <cuda_runtime.h>

#include <algorithm>

#include "assemble.h"
#include "pairs.cuh"
#include "rule.cuh"
#include "timeint.cuh"
#include "nonuniform_time.cuh"

namespace stbem {

__constant__ float c_gxf[kGaussTotal];
__constant__ float c_gwf[kGaussTotal];

template <typename R> __device__ __forceinline__ R gxr(int i);
template <> __device__ __forceinline__ double gxr<double>(int i) { return c_tab.gx[i]; }
template <> __device__ __forceinline__ float gxr<float>(int i) { return c_gxf[i]; }
template <typename R> __device__ __forceinline__ R gwr(int i);
template <> __device__ __forceinline__ double gwr<double>(int i) { return c_tab.gw[i]; }
template <> __device__ __forceinline__ float gwr<float>(int i) { return c_gwf[i]; }

__device__ __forceinline__ double exp_neg(double x) { return exp_neg_fast(x); }
__device__ __forceinline__ float exp_neg(float x) { return exp_neg_f(x); }
// e^{-c sigma_g} at node g of a multi-lag table: FP64 from the pre-scaled
// nodes and the table copy in shared memory (`fast`: c sigk_max is below the
// table method's range, tested once per point), FP32 by the MUFU exponential
template <typename T>
__device__ __forceinline__ double ml_exp(double c, const T& tab, int g, bool fast) {
  return fast ? exp_prod_fast(c, tab.sigk[g], tab.etab) : exp_neg_fast(c * tab.sig[g]);
}
template <typename T>
__device__ __forceinline__ float ml_exp(float c, const T& tab, int g, bool) {
  return exp_neg_f(c * tab.sig[g]);
}
__device__ __forceinline__ void e12(double z, double* a, double* b) { e1e2(z, a, b); }
__device__ __forceinline__ void e12(float z, float* a, float* b) { e1e2_f(z, a, b); }

// ---- FP64 lag-0/1 kernels for D (share E1/E2 between F_V and F_1) ----------------
__device__ __forceinline__ void lag01_D64(double c, int d, double ht, double alpha, double* outv, double* out1) {
  if (d == 0) {
    double a, b;
    e1e2(c / ht, &a, &b);
    *outv = ht / kFourPi * (a - b);
    *out1 = alpha / kFourPi * a;
    return;
  }
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
}

// ---- FP32 lag-0/1 kernels (regular and near pairs of the mixed precision) --------
template <int K>
__device__ __forceinline__ float lag01_f(float c, int d, float ht, float alpha) {
  const float four_pi = (float)kFourPi;
  const float z = c * (1.0f / ht);
  if (d == 0) {
    float a, b;
    e1e2_f(z, &a, &b);
    if (K == kV) return ht / four_pi * (a - b);
    if (K == kKq) return alpha / (2.0f * four_pi * z) * b;
    return alpha / four_pi * a;
  }
  if (z < 1.0f) {
    const float eh = ein_series_f(0.5f * z), ef = ein_series_f(z);
    const float g = (float)kEulerGamma, l2z = logf(2.0f * z);
    const float em = exp_neg_f(0.5f * z) * expm1f(-0.5f * z);
    if (K == kV) return ht / (2.0f * (float)kPi) * (0.69314718f + eh - ef + 0.5f * z * (g + l2z + eh - 2.0f * ef) + em);
    if (K == kKq) return alpha / four_pi * (-em / z - 0.5f * (g + l2z) - 0.5f * eh + ef);
    return alpha / four_pi * (g + l2z + eh - 2.0f * ef);
  }
  float a2, b2, a1, b1;
  e1e2_f(0.5f * z, &a2, &b2);
  e1e2_f(z, &a1, &b1);
  if (K == kV) return (2.0f * ht) / four_pi * (a2 - b2) - 2.0f * (ht / four_pi * (a1 - b1));
  if (K == kKq) return alpha / (four_pi * z) * (b2 - b1);   // 2 ht alpha / (8 pi c)
  return alpha / four_pi * a2 - 2.0f * (alpha / four_pi * a1);
}

// precision-generic lag-0/1 evaluation
template <typename R, int K>
__device__ __forceinline__ R lag01(R c, int d, double ht, double alpha) {
  if constexpr (sizeof(R) == 8) return lag_kernel<K>(c, d, ht, alpha, c_tab.gx, c_tab.gw);
  else return lag01_f<K>(c, d, (float)ht, (float)alpha);
}
template <typename R>
__device__ __forceinline__ void lag01D(R c, int d, double ht, double alpha, R* kv, R* k1v) {
  if constexpr (sizeof(R) == 8) {
    lag01_D64(c, d, ht, alpha, kv, k1v);
  } else {
    *kv = lag01_f<kV>(c, d, (float)ht, (float)alpha);
    *k1v = lag01_f<k1>(c, d, (float)ht, (float)alpha);
  }
}

// Lags 0 and 1 together at one c (FP64): lag 0 is F(ht) and the closed form of
// lag 1 is F(2 ht) - 2 F(ht), so F(ht) is evaluated once for both.  Same
// operations in the same order as the one-lag evaluation (lag_kernel,
// lag01_D64), so both give identical results.
template <int K>
__device__ __forceinline__ void lag01_pair(double c, double ht, double alpha, double* k0, double* k1) {
  const double z = c / ht;
  double a1, b1;
  e1e2(z, &a1, &b1);
  const double F1 = K == kV ? ht / kFourPi * (a1 - b1) : alpha / (2.0 * kFourPi * c) * ht * b1;
  *k0 = F1;
  if (z < 1.0) {
    *k1 = lag1_series<K>(z, ht, alpha);
    return;
  }
  double a2, b2;
  e1e2(c / (2.0 * ht), &a2, &b2);
  const double F2 = K == kV ? (2.0 * ht) / kFourPi * (a2 - b2) : alpha / (2.0 * kFourPi * c) * (2.0 * ht) * b2;
  *k1 = F2 - 2.0 * F1;
}

__device__ __forceinline__ void lag01_D64_pair(double c, double ht, double alpha, double* v0, double* o0, double* v1,
                                               double* o1) {
  const double z = c / ht;
  double a1, b1;
  e1e2(z, &a1, &b1);
  const double fv = ht / kFourPi * (a1 - b1), f1 = alpha / kFourPi * a1;
  *v0 = fv;
  *o0 = f1;
  if (z < 1.0) {
    *v1 = lag1_series<kV>(z, ht, alpha);
    *o1 = lag1_series<k1>(z, ht, alpha);
    return;
  }
  double a2, b2;
  e1e2(c / (2.0 * ht), &a2, &b2);
  *v1 = (2.0 * ht) / kFourPi * (a2 - b2) - 2.0 * fv;
  *o1 = alpha / kFourPi * a2 - 2.0 * f1;
}

// D2_d F_V (K = kV) or D2_d F_K / q (K = kKq) at lag d >= 2 from the tables.
template <typename R, int K>
__device__ __forceinline__ R lag2_kernel(R c, int d, R alpha, const LagNodes<R>& L) {
  const R four_pi = (R)kFourPi;
  if (c * L.inv_dht > (R)0.5 * (R)d) {
    R f[3];
    for (int k = 0; k < 3; ++k) {
      R a, b;
      e12(c * L.inv_s[k], &a, &b);
      f[k] = K == kV ? L.s[k] / four_pi * (a - b) : alpha / ((R)2 * four_pi * c) * L.s[k] * b;
    }
    return (f[0] - (R)2 * f[1]) + f[2];
  }
  R acc = (R)0;
  for (int g = 0; g < L.n; ++g) {
    const R e = exp_neg(c * L.sig[g]);
    acc = fma(K == kV ? L.wv[g] : L.wk[g], e, acc);
  }
  return acc;
}

template <typename R>
__device__ __forceinline__ void lag2_kernel_D(R c, int d, R alpha, const LagNodes<R>& L, R* outv, R* out1) {
  const R four_pi = (R)kFourPi;
  if (c * L.inv_dht > (R)0.5 * (R)d) {
    R fv[3], f1[3];
    for (int k = 0; k < 3; ++k) {
      R a, b;
      e12(c * L.inv_s[k], &a, &b);
      fv[k] = L.s[k] / four_pi * (a - b);
      f1[k] = alpha / four_pi * a;
    }
    *outv = (fv[0] - (R)2 * fv[1]) + fv[2];
    *out1 = (f1[0] - (R)2 * f1[1]) + f1[2];
    return;
  }
  R av = (R)0, a1 = (R)0;
  for (int g = 0; g < L.n; ++g) {
    const R e = exp_neg(c * L.sig[g]);
    av = fma(L.wv[g], e, av);
    a1 = fma(e, fma(L.w3[g], c, -L.w2[g]), a1);
  }
  *outv = av;
  *out1 = a1;
}

// ---- moments of one piece pair with a tensor Gauss rule (phase 1) ----------------
template <int OP> struct NMom { static constexpr int n = OP == STBEM_OP_V ? 1 : (OP == STBEM_OP_K ? 2 : 5); };

template <typename R, int OP, bool LAG01>
__device__ void tensor_moments_impl(const Piece& A, const Piece& B, int d, int n, double ht, double alpha,
                                    const LagNodes<R>* LN, double* mom) {
  const int o = gauss_offset(n);
  const R eax = (R)(A.x1 - A.x0), eay = (R)(A.y1 - A.y0);
  const R ebx = (R)(B.x1 - B.x0), eby = (R)(B.y1 - B.y0);
  const R abx = (R)(A.x0 - B.x0), aby = (R)(A.y0 - B.y0);
  // q = (x - y) . n_b = (A0 - B0) . n_b + xi (e_a . n_b): the trial edge is
  // orthogonal to its own normal, so the eta term drops out exactly
  const R qab = (R)((A.x0 - B.x0) * B.nx + (A.y0 - B.y0) * B.ny);
  const R qea = (R)((A.x1 - A.x0) * B.nx + (A.y1 - A.y0) * B.ny);
  const R qa = (R)(0.25 * alpha);
  const R al = (R)alpha;
  R s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
  for (int a = 0; a < n; ++a) {
    const R xi = gxr<R>(o + a);
    const R wa = gwr<R>(o + a);
    for (int b = 0; b < n; ++b) {
      const R eta = gxr<R>(o + b);
      const R w = wa * gwr<R>(o + b);
      const R dx = (abx + xi * eax) - eta * ebx;
      const R dy = (aby + xi * eay) - eta * eby;
      const R c = qa * (dx * dx + dy * dy);
      if constexpr (OP == STBEM_OP_V) {
        R k;
        if constexpr (LAG01) k = lag01<R, kV>(c, d, ht, alpha);
        else k = lag2_kernel<R, kV>(c, d, al, *LN);
        s0 += w * k;
      } else if constexpr (OP == STBEM_OP_K) {
        R kq;
        if constexpr (LAG01) kq = lag01<R, kKq>(c, d, ht, alpha);
        else kq = lag2_kernel<R, kKq>(c, d, al, *LN);
        const R wk = w * ((qab + xi * qea) * kq);
        s0 += wk * ((R)1 - eta);
        s1 += wk * eta;
      } else {
        R kv, k1v;
        if constexpr (LAG01) lag01D<R>(c, d, ht, alpha, &kv, &k1v);
        else lag2_kernel_D<R>(c, d, al, *LN, &kv, &k1v);
        s0 += w * kv;
        const R wk = w * k1v;
        s1 += wk * ((R)1 - xi) * ((R)1 - eta);
        s2 += wk * ((R)1 - xi) * eta;
        s3 += wk * xi * ((R)1 - eta);
        s4 += wk * xi * eta;
      }
    }
  }
  const double L = A.len * B.len;
  mom[0] = (double)s0 * L;
  if (NMom<OP>::n > 1) mom[1] = (double)s1 * L;
  if (NMom<OP>::n > 2) {
    mom[2] = (double)s2 * L;
    mom[3] = (double)s3 * L;
    mom[4] = (double)s4 * L;
  }
}

// ---- several consecutive lags at once (lags >= 2) ----------------------------------
// Values of D2_d F (K = kV or kKq) for the T.L lags d0.. of the table at one c.
// The closed form applies to a prefix of the lags (its switch c / (d ht) > d/2
// moves to larger c as d grows); F at the shared times is evaluated once.  The
// Peano lags use intervals lc .. L, each evaluated once: its left-role sum
// serves lag i, its right-role sum lag i - 1.
template <typename R, int K, int NL>
__device__ __forceinline__ void ml_kernel(R c, R alpha, const MLNodes<R>& T, R (&out)[NL]) {
  const int L = T.L;
  const R four_pi = (R)kFourPi;
  int lc = 0;
  while (lc < L && c > T.cthr[lc]) ++lc;
  const bool fast = c * T.sigk_max < (R)kExpProdMax;
  if (lc > 0) {
    R F[NL + 2];
#pragma unroll
    for (int j = 0; j < NL + 2; ++j) {
      if (j >= lc + 2) break;
      R a, b;
      e12(c * T.inv_s[j], &a, &b);
      F[j] = K == kV ? T.s[j] / four_pi * (a - b) : alpha / ((R)2 * four_pi * c) * T.s[j] * b;
    }
#pragma unroll
    for (int l = 0; l < NL; ++l)
      if (l < lc) out[l] = (F[l + 2] - (R)2 * F[l + 1]) + F[l];
  }
  if (lc < L) {
    const R* lw = K == kV ? T.lv : T.lk;
    const R* rw = K == kV ? T.rv : T.rk;
    R carry = (R)0;
    for (int i = lc; i <= L; ++i) {
      R sl = (R)0, sr = (R)0;
      const int g0 = T.off[i], g1 = T.off[i + 1];
      if (i < L && i > lc) {
        for (int g = g0; g < g1; ++g) {
          const R e = ml_exp(c, T, g, fast);
          sl = fma(lw[g], e, sl);
          sr = fma(rw[g], e, sr);
        }
      } else if (i < L) {
        for (int g = g0; g < g1; ++g) sl = fma(lw[g], ml_exp(c, T, g, fast), sl);
      } else {
        for (int g = g0; g < g1; ++g) sr = fma(rw[g], ml_exp(c, T, g, fast), sr);
      }
#pragma unroll
      for (int l = 0; l < NL; ++l)
        if (l == i - 1 && i > lc) out[l] = carry + sr;
      carry = sl;
    }
  }
}

// D_h's two kernels (F_V and F_1) for the lags of the table at one c.
template <typename R, int NL>
__device__ __forceinline__ void ml_kernel_D(R c, R alpha, const MLNodes<R>& T, R (&ov)[NL], R (&o1)[NL]) {
  const int L = T.L;
  const R four_pi = (R)kFourPi;
  int lc = 0;
  while (lc < L && c > T.cthr[lc]) ++lc;
  const bool fast = c * T.sigk_max < (R)kExpProdMax;
  if (lc > 0) {
    R Fv[NL + 2], F1[NL + 2];
#pragma unroll
    for (int j = 0; j < NL + 2; ++j) {
      if (j >= lc + 2) break;
      R a, b;
      e12(c * T.inv_s[j], &a, &b);
      Fv[j] = T.s[j] / four_pi * (a - b);
      F1[j] = alpha / four_pi * a;
    }
#pragma unroll
    for (int l = 0; l < NL; ++l)
      if (l < lc) {
        ov[l] = (Fv[l + 2] - (R)2 * Fv[l + 1]) + Fv[l];
        o1[l] = (F1[l + 2] - (R)2 * F1[l + 1]) + F1[l];
      }
  }
  if (lc < L) {
    R cv = (R)0, c1 = (R)0;
    for (int i = lc; i <= L; ++i) {
      R slv = (R)0, srv = (R)0, sl1 = (R)0, sr1 = (R)0;
      const int g0 = T.off[i], g1 = T.off[i + 1];
      const bool wl = i < L, wr = i > lc;
      for (int g = g0; g < g1; ++g) {
        const R e = ml_exp(c, T, g, fast);
        if (wl) {
          slv = fma(T.lv[g], e, slv);
          sl1 = fma(e, fma(T.l3[g], c, -T.l2[g]), sl1);
        }
        if (wr) {
          srv = fma(T.rv[g], e, srv);
          sr1 = fma(e, fma(T.r3[g], c, -T.r2[g]), sr1);
        }
      }
#pragma unroll
      for (int l = 0; l < NL; ++l)
        if (l == i - 1 && wr) {
          ov[l] = cv + srv;
          o1[l] = c1 + sr1;
        }
      cv = slv;
      c1 = sl1;
    }
  }
}

// Moments of one piece pair for the lags of the table, tensor Gauss rule of
// order n; mom[l * ls + q] for lag l and moment q (as tensor_moments_impl).
template <typename R, int OP, int NL>
__device__ void tensor_moments_ml(const Piece& A, const Piece& B, int n, double alpha, const MLNodes<R>& T,
                                  double* mom, int ls) {
  const int o = gauss_offset(n);
  const R eax = (R)(A.x1 - A.x0), eay = (R)(A.y1 - A.y0);
  const R ebx = (R)(B.x1 - B.x0), eby = (R)(B.y1 - B.y0);
  const R abx = (R)(A.x0 - B.x0), aby = (R)(A.y0 - B.y0);
  const R qab = (R)((A.x0 - B.x0) * B.nx + (A.y0 - B.y0) * B.ny);
  const R qea = (R)((A.x1 - A.x0) * B.nx + (A.y1 - A.y0) * B.ny);
  const R qa = (R)(0.25 * alpha);
  const R al = (R)alpha;
  constexpr int NM = NMom<OP>::n;
  R acc[NL][NM];
#pragma unroll
  for (int l = 0; l < NL; ++l)
#pragma unroll
    for (int q = 0; q < NM; ++q) acc[l][q] = (R)0;
  for (int a = 0; a < n; ++a) {
    const R xi = gxr<R>(o + a);
    const R wa = gwr<R>(o + a);
    for (int b = 0; b < n; ++b) {
      const R eta = gxr<R>(o + b);
      const R w = wa * gwr<R>(o + b);
      const R dx = (abx + xi * eax) - eta * ebx;
      const R dy = (aby + xi * eay) - eta * eby;
      const R c = qa * (dx * dx + dy * dy);
      if constexpr (OP == STBEM_OP_V) {
        R k[NL];
        ml_kernel<R, kV, NL>(c, al, T, k);
#pragma unroll
        for (int l = 0; l < NL; ++l)
          if (l < T.L) acc[l][0] += w * k[l];
      } else if constexpr (OP == STBEM_OP_K) {
        R k[NL];
        ml_kernel<R, kKq, NL>(c, al, T, k);
        const R wq = w * (qab + xi * qea);
#pragma unroll
        for (int l = 0; l < NL; ++l)
          if (l < T.L) {
            const R wk = wq * k[l];
            acc[l][0] += wk * ((R)1 - eta);
            acc[l][1] += wk * eta;
          }
      } else {
        R kv[NL], k1[NL];
        ml_kernel_D<R, NL>(c, al, T, kv, k1);
        const R b11 = ((R)1 - xi) * ((R)1 - eta), b10 = ((R)1 - xi) * eta;
        const R b01 = xi * ((R)1 - eta), b00 = xi * eta;
#pragma unroll
        for (int l = 0; l < NL; ++l)
          if (l < T.L) {
            acc[l][0] += w * kv[l];
            const R wk = w * k1[l];
            acc[l][1] += wk * b11;
            acc[l][2] += wk * b10;
            acc[l][3] += wk * b01;
            acc[l][4] += wk * b00;
          }
      }
    }
  }
  const double LL = A.len * B.len;
#pragma unroll
  for (int l = 0; l < NL; ++l)
    if (l < T.L)
#pragma unroll
      for (int q = 0; q < NM; ++q) mom[l * ls + q] = (double)acc[l][q] * LL;
}

// Moments of one regular or near piece pair at lags 0 and 1 together (FP64):
// mom[q] for lag 0, mom[ls + q] for lag 1.
template <int OP>
__device__ void tensor_moments_01(const Piece& A, const Piece& B, int n, double ht, double alpha, double* mom,
                                  int ls) {
  const int o = gauss_offset(n);
  const double eax = A.x1 - A.x0, eay = A.y1 - A.y0;
  const double ebx = B.x1 - B.x0, eby = B.y1 - B.y0;
  const double abx = A.x0 - B.x0, aby = A.y0 - B.y0;
  const double qab = (A.x0 - B.x0) * B.nx + (A.y0 - B.y0) * B.ny;
  const double qea = (A.x1 - A.x0) * B.nx + (A.y1 - A.y0) * B.ny;
  const double qa = 0.25 * alpha;
  constexpr int NM = NMom<OP>::n;
  double acc[2][NM];
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int q = 0; q < NM; ++q) acc[l][q] = 0.0;
  for (int a = 0; a < n; ++a) {
    const double xi = c_tab.gx[o + a], wa = c_tab.gw[o + a];
    for (int b = 0; b < n; ++b) {
      const double eta = c_tab.gx[o + b];
      const double w = wa * c_tab.gw[o + b];
      const double dx = (abx + xi * eax) - eta * ebx;
      const double dy = (aby + xi * eay) - eta * eby;
      const double c = qa * (dx * dx + dy * dy);
      if constexpr (OP == STBEM_OP_V) {
        double k0, k1;
        lag01_pair<kV>(c, ht, alpha, &k0, &k1);
        acc[0][0] += w * k0;
        acc[1][0] += w * k1;
      } else if constexpr (OP == STBEM_OP_K) {
        double k0, k1;
        lag01_pair<kKq>(c, ht, alpha, &k0, &k1);
        const double q = qab + xi * qea;
        const double w0 = w * (q * k0), w1 = w * (q * k1);
        acc[0][0] += w0 * (1.0 - eta);
        acc[0][1] += w0 * eta;
        acc[1][0] += w1 * (1.0 - eta);
        acc[1][1] += w1 * eta;
      } else {
        double v0, o0, v1, o1;
        lag01_D64_pair(c, ht, alpha, &v0, &o0, &v1, &o1);
        const double wo0 = w * o0, wo1 = w * o1;
        acc[0][0] += w * v0;
        acc[1][0] += w * v1;
        acc[0][1] += wo0 * (1.0 - xi) * (1.0 - eta);
        acc[0][2] += wo0 * (1.0 - xi) * eta;
        acc[0][3] += wo0 * xi * (1.0 - eta);
        acc[0][4] += wo0 * xi * eta;
        acc[1][1] += wo1 * (1.0 - xi) * (1.0 - eta);
        acc[1][2] += wo1 * (1.0 - xi) * eta;
        acc[1][3] += wo1 * xi * (1.0 - eta);
        acc[1][4] += wo1 * xi * eta;
      }
    }
  }
  const double LL = A.len * B.len;
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int q = 0; q < NM; ++q) mom[l * ls + q] = acc[l][q] * LL;
}

// ---- moments of one singular pair, FP64 (lags 0 and 1) ------------------------------
// One CTA per identical or vertex-sharing pair at lag 0 or 1; the rule's
// points are strided over the threads and reduced in a fixed tree, so the
// moments do not depend on scheduling.  Slots: identical pairs (i, i) at
// [0, R), (i, i+1) at [R, 2R), (i, i-1) at [2R, 3R) of the ring of R pieces.
constexpr int kSingThreads = 128;

template <int OP>
__device__ void singular_body(const DevMesh& M, int slot, int d, double* __restrict__ buf,
                              double (*red)[kSingThreads]) {
  constexpr int NM = NMom<OP>::n;
  const int N = M.N;
  const int Rl = OP == STBEM_OP_D ? 2 * N : N;
  const int kind = slot / Rl, i = slot % Rl;
  const int cls = kind == 0 ? kIdentical : (kind == 1 ? kAdjNext : kAdjPrev);
  const int j = kind == 0 ? i : (kind == 1 ? (i + 1) % Rl : (i - 1 + Rl) % Rl);
  const double ht = M.ht, alpha = M.alpha;
  const Piece A = OP == STBEM_OP_D ? half_piece(M, i) : seg_piece(M, i);
  const Piece B = OP == STBEM_OP_D ? half_piece(M, j) : seg_piece(M, j);
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  // the identical pair of K contributes nothing (q = 0 on a straight segment)
  if (!(OP == STBEM_OP_K && kind == 0)) {
    const int np = singular_points(cls);
    for (int p = threadIdx.x; p < np; p += kSingThreads) {
      double xi, eta, w, dx, dy;
      singular_point(cls, p, A, B, &xi, &eta, &w, &dx, &dy);
      const double c = 0.25 * alpha * (dx * dx + dy * dy);
      if constexpr (OP == STBEM_OP_V) {
        s[0] += w * lag_kernel<kV>(c, d, ht, alpha, c_tab.gx, c_tab.gw);
      } else if constexpr (OP == STBEM_OP_K) {
        const double wk = w * ((dx * B.nx + dy * B.ny) * lag_kernel<kKq>(c, d, ht, alpha, c_tab.gx, c_tab.gw));
        s[0] += wk * (1.0 - eta);
        s[1] += wk * eta;
      } else {
        double kv, k1v;
        lag01_D64(c, d, ht, alpha, &kv, &k1v);
        s[0] += w * kv;
        const double wk = w * k1v;
        s[1] += wk * (1.0 - xi) * (1.0 - eta);
        s[2] += wk * (1.0 - xi) * eta;
        s[3] += wk * xi * (1.0 - eta);
        s[4] += wk * xi * eta;
      }
    }
  }
  for (int q = 0; q < NM; ++q) red[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int w = kSingThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < NM; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 5) {
    const double L = A.len * B.len;
    buf[((size_t)d * 3 * Rl + slot) * 5 + threadIdx.x] = (int)threadIdx.x < NM ? red[threadIdx.x][0] * L : 0.0;
  }
}

template <int OP>
__global__ void __launch_bounds__(kSingThreads) k_singular(DevMesh M, double* __restrict__ buf) {
  __shared__ double red[5][kSingThreads];
  singular_body<OP>(M, blockIdx.x, blockIdx.y, buf, red);
}

// V, lags >= 2: one thread per upper-triangle entry, one lag per block row.
template <typename R, typename T>
__global__ void __launch_bounds__(128) k_lag2_V(DevMesh M, int d_begin, T* __restrict__ out) {
  __shared__ LagNodes<R> LN;
  const int N = M.N;
  const int d = d_begin + blockIdx.y;
  build_lag_nodes<R>(LN, d, M.ht, M.alpha);
  __syncthreads();
  const long long npair = (long long)N * (N + 1) / 2;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npair) return;
  // row i of the upper triangle: rows < i hold S(i) = i N - i (i - 1) / 2 entries
  const double B2 = 2.0 * N + 1.0;
  int i = (int)floor((B2 - sqrt(B2 * B2 - 8.0 * (double)p)) * 0.5);
  auto S = [N](long long r) { return r * N - r * (r - 1) / 2; };
  while (i > 0 && S(i) > p) --i;
  while (S(i + 1) <= p) ++i;
  const int j = i + (int)(p - S(i));
  double m[1];
  tensor_moments_impl<R, STBEM_OP_V, false>(seg_piece(M, i), seg_piece(M, j), d, space_order(d), M.ht, M.alpha,
                                            &LN, m);
  const size_t base = (size_t)d * N * N;
  out[base + (size_t)i * N + j] = (T)m[0];
  if (i != j) out[base + (size_t)j * N + i] = (T)m[0];
}

// Lags >= 2 of one launch: up to three runs [lo, hi) of one space order each
// (split at d = 8 and 32), cut into chunks of at most L consecutive lags;
// chunk c of the launch (blockIdx.y) is the c-th in lag order, so the CTAs
// of the most expensive lags (highest space and Peano orders) start first.
struct MLSegs {
  int lo[3], hi[3], n[3];   // n: chunks of the run
};

__device__ __forceinline__ void ml_chunk(const MLSegs& S, int L, int c, int* d0, int* d1) {
  int sg = 0;
  while (sg < 2 && c >= S.n[sg]) c -= S.n[sg++];
  *d0 = S.lo[sg] + c * L;
  *d1 = min(*d0 + L, S.hi[sg]);
}

// V, lags >= 2, L consecutive lags per block row (one table per CTA).
template <typename R, typename T>
__global__ void __launch_bounds__(128) k_lag2_V_ml(DevMesh M, MLSegs segs, int L, T* __restrict__ out) {
  __shared__ MLNodes<R> TN;
  const int N = M.N;
  int d0, d_end;
  ml_chunk(segs, L, blockIdx.y, &d0, &d_end);
  const int nl = min(L, d_end - d0);
  build_ml_nodes<R>(TN, d0, nl, M.ht, M.alpha);
  __syncthreads();
  const long long npair = (long long)N * (N + 1) / 2;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npair) return;
  const double B2 = 2.0 * N + 1.0;
  int i = (int)floor((B2 - sqrt(B2 * B2 - 8.0 * (double)p)) * 0.5);
  auto S = [N](long long r) { return r * N - r * (r - 1) / 2; };
  while (i > 0 && S(i) > p) --i;
  while (S(i + 1) <= p) ++i;
  const int j = i + (int)(p - S(i));
  double m[kMaxLagsML];
  tensor_moments_ml<R, STBEM_OP_V, kMaxLagsML>(seg_piece(M, i), seg_piece(M, j), space_order(d0), M.alpha, TN, m, 1);
  for (int l = 0; l < nl; ++l) {
    const size_t base = (size_t)(d0 + l) * N * N;
    out[base + (size_t)i * N + j] = (T)m[l];
    if (i != j) out[base + (size_t)j * N + i] = (T)m[l];
  }
}

// ---- tile geometry -----------------------------------------------------------------
constexpr int kTileThreads = 256;
constexpr int kT = 16;                 // entries per tile side (V, D); K rows
constexpr int kKP = 15, kKJ = kKP + 1; // K: entry columns, trial segment columns
constexpr int kDP = 2 * kT + 2;        // D: half-segments per tile side

template <int OP> struct Tile {
  static constexpr int pairs = OP == STBEM_OP_V ? kT * kT : (OP == STBEM_OP_K ? kT * kKJ : kDP * kDP);
  static constexpr int nm = NMom<OP>::n;
};

template <int OP, typename R>
constexpr size_t tile_smem_bytes() {
  return (((size_t)Tile<OP>::pairs * Tile<OP>::nm * sizeof(double) + 15) / 16) * 16 + sizeof(LagNodes<R>);
}

// Decode the tile of block x: symmetric operators use upper-triangular tile pairs.
__device__ __forceinline__ void upper_tile(int bx, int nT, int* rt, int* ct) {
  int r = 0, rem = bx;
  while (rem >= nT - r) {
    rem -= nT - r;
    ++r;
  }
  *rt = r;
  *ct = r + rem;
}

// Pieces of tile pair p (phase 1 and 2 share this map); false if the pair
// contributes nothing.
template <int OP>
__device__ __forceinline__ bool tile_pair(const DevMesh& M, int r0, int c0, int p, Piece* A, Piece* B,
                                          int* ia, int* ib, int* ring) {
  const int N = M.N;
  if (OP == STBEM_OP_V) {
    const int i = r0 + p / kT, j = c0 + p % kT;
    if (i >= N || j >= N) return false;
    *ia = i < j ? i : j;
    *ib = i < j ? j : i;
    *A = seg_piece(M, *ia);
    *B = seg_piece(M, *ib);
    *ring = N;
    return true;
  } else if (OP == STBEM_OP_K) {
    const int i = r0 + p / kKJ;
    const int j = ((c0 - 1 + p % kKJ) % N + N) % N;
    if (i >= N || j == i) return false;       // identical pair: q = 0
    *ia = i;
    *ib = j;
    *A = seg_piece(M, i);
    *B = seg_piece(M, j);
    *ring = N;
    return true;
  } else {
    const int H = 2 * N;
    *ia = ((2 * r0 - 1 + p / kDP) % H + H) % H;
    *ib = ((2 * c0 - 1 + p % kDP) % H + H) % H;
    *A = half_piece(M, *ia);
    *B = half_piece(M, *ib);
    *ring = H;
    return true;
  }
}

// Slot of a singular pair in the lag-0/1 moment buffer: ring R pieces,
// identical pairs at [0, R), (i, i+1) at [R, 2R), (i, i-1) at [2R, 3R).
__device__ __forceinline__ int singular_slot(int cls, int ia, int Rl) {
  return cls == kIdentical ? ia : (cls == kAdjNext ? Rl + ia : 2 * Rl + ia);
}

// Number of tiles of one lag block of op on N segments.
template <int OP>
__host__ __device__ __forceinline__ int tiles_per_lag(int N) {
  if (OP == STBEM_OP_K) return ((N + kT - 1) / kT) * ((N + kKP - 1) / kKP);
  const int nT = (N + kT - 1) / kT;
  return nT * (nT + 1) / 2;
}

// Phase 3 of a tile: entries of one lag block from its pair moments.  With
// `mirrored` (D on a diagonal tile) only the half-pairs (u, v) with u <= v
// were integrated; (v, u) is the same pair with the roles exchanged, whose
// moments are those of (u, v) with the two mixed ones (1 - xi) eta and
// xi (1 - eta) swapped (both kernels depend on |x - y| only).
template <int OP, typename T>
__device__ __forceinline__ void tile_entries(const DevMesh& M, int rt, int ct, int r0, int c0,
                                             const double* __restrict__ mom, size_t base, T* __restrict__ out,
                                             bool mirrored = false) {
  constexpr int NM = Tile<OP>::nm;
  const int N = M.N;
  const int tid = threadIdx.x;
  if (OP == STBEM_OP_V) {
    const int i = r0 + tid / kT, j = c0 + tid % kT;
    if (i < N && j < N) {
      const T v = (T)mom[tid];
      out[base + (size_t)i * N + j] = v;
      if (rt != ct) out[base + (size_t)j * N + i] = v;
    }
  } else if (OP == STBEM_OP_K) {
    if (tid < kT * kKP) {
      const int si = tid / kKP, sp = tid % kKP;
      const int i = r0 + si, p = c0 + sp;
      if (i < N && p < N) {
        const double val = mom[(size_t)(si * kKJ + sp + 1) * NM + 0] + mom[(size_t)(si * kKJ + sp) * NM + 1];
        out[base + (size_t)i * N + p] = (T)val;
      }
    }
  } else {
    const int s = tid / kT, t = tid % kT;
    const int l = r0 + s, k = c0 + t;
    // evaluate with the smaller index first; on a diagonal tile both ranges coincide
    const int lo = l < k ? l : k, hi = l < k ? k : l;
    const int so = lo - r0, to = hi - c0;
    if (l < N && k < N && so >= 0 && to >= 0 && so < kT && to < kT) {
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
          const bool mir = mirrored && v < u;
          const double* mm = mom + (size_t)(mir ? v * kDP + u : u * kDP + v) * NM;
          const double m2 = mir ? mm[3] : mm[2], m3 = mir ? mm[2] : mm[3];
          const double I1 = a0 * (b0 * mm[1] + b1 * m2) + a1 * (b0 * m3 + b1 * mm[4]);
          val += ca * cb * mm[0] + nn * I1;
        }
      }
      out[base + (size_t)l * N + k] = (T)val;
      if (rt != ct) out[base + (size_t)k * N + l] = (T)val;
    }
  }
}

// One tile of one lag block: all threads of the CTA take part.
template <int OP, typename R, typename T, bool LAG01>
__device__ void tile_body(const DevMesh& M, int d, int tile, const double* __restrict__ sing, T* __restrict__ out,
                          unsigned char* smem_raw) {
  constexpr int P = Tile<OP>::pairs, NM = Tile<OP>::nm;
  double* mom = reinterpret_cast<double*>(smem_raw);
  LagNodes<R>* LN = reinterpret_cast<LagNodes<R>*>(smem_raw + (((size_t)P * NM * sizeof(double) + 15) / 16) * 16);

  const int N = M.N;
  const double ht = M.ht, alpha = M.alpha;
  int rt, ct;
  if (OP == STBEM_OP_K) {
    const int nP = (N + kKP - 1) / kKP;
    rt = tile / nP;
    ct = tile % nP;
  } else {
    upper_tile(tile, (N + kT - 1) / kT, &rt, &ct);
  }
  const int r0 = rt * kT, c0 = ct * (OP == STBEM_OP_K ? kKP : kT);
  const int tid = threadIdx.x;
  if (!LAG01) build_lag_nodes<R>(*LN, d, ht, alpha);
  __syncthreads();

  // phase 1: whole pairs per thread; at lags 0 and 1 the identical and
  // vertex-sharing pairs take their FP64 moments from k_singular's buffer
  for (int p = tid; p < P; p += kTileThreads) {
    Piece A, B;
    int ia, ib, ring;
    double* m = mom + (size_t)p * NM;
    if (!tile_pair<OP>(M, r0, c0, p, &A, &B, &ia, &ib, &ring)) {
      for (int q = 0; q < NM; ++q) m[q] = 0.0;
      continue;
    }
    int n;
    if (!LAG01) {
      n = space_order(d);
      tensor_moments_impl<R, OP, false>(A, B, d, n, ht, alpha, LN, m);
    } else {
      const int cls = pair_class(ring, ia, ib, A, B);
      if (cls == kIdentical || cls == kAdjNext || cls == kAdjPrev) {
        const double* src = sing + ((size_t)d * 3 * ring + singular_slot(cls, ia, ring)) * 5;
        for (int q = 0; q < NM; ++q) m[q] = src[q];
        continue;
      }
      n = cls == kRegular ? kRegular01 : kNear01;
      tensor_moments_impl<R, OP, true>(A, B, d, n, ht, alpha, (const LagNodes<R>*)nullptr, m);
    }
  }
  __syncthreads();
  // phase 3: entries
  tile_entries<OP, T>(M, rt, ct, r0, c0, mom, (size_t)d * N * N, out);
}

// L consecutive lags >= 2 of one tile: phase 1 integrates every pair for all
// L lags at once (shared Peano intervals and closed-form times), phase 3
// gathers each lag's entries.  Shared memory: L moment arrays + the table.
template <int OP, int LM>
struct TileML {
  static constexpr size_t mom_bytes = (((size_t)LM * Tile<OP>::pairs * Tile<OP>::nm * sizeof(double) + 15) / 16) * 16;
};
template <int OP, typename R, int LM>
constexpr size_t tile_ml_smem_bytes() {
  return TileML<OP, LM>::mom_bytes + sizeof(MLNodes<R>);
}

template <int OP, typename R, typename T, int LM>
__device__ void tile_body_ml(const DevMesh& M, int d0, int nl, int tile, T* __restrict__ out,
                             unsigned char* smem_raw) {
  constexpr int P = Tile<OP>::pairs, NM = Tile<OP>::nm;
  double* mom = reinterpret_cast<double*>(smem_raw);
  MLNodes<R>* TN = reinterpret_cast<MLNodes<R>*>(smem_raw + TileML<OP, LM>::mom_bytes);
  const int N = M.N;
  int rt, ct;
  if (OP == STBEM_OP_K) {
    const int nP = (N + kKP - 1) / kKP;
    rt = tile / nP;
    ct = tile % nP;
  } else {
    upper_tile(tile, (N + kT - 1) / kT, &rt, &ct);
  }
  const int r0 = rt * kT, c0 = ct * (OP == STBEM_OP_K ? kKP : kT);
  build_ml_nodes<R>(*TN, d0, nl, M.ht, M.alpha);
  __syncthreads();
  const int n = space_order(d0);
  // D on a diagonal tile: the half-pair block is symmetric, integrate u <= v only
  const bool mirrored = OP == STBEM_OP_D && rt == ct;
  for (int p = threadIdx.x; p < P; p += kTileThreads) {
    if (mirrored && p % kDP < p / kDP) continue;
    Piece A, B;
    int ia, ib, ring;
    double* m = mom + (size_t)p * NM;
    if (!tile_pair<OP>(M, r0, c0, p, &A, &B, &ia, &ib, &ring)) {
      for (int l = 0; l < nl; ++l)
        for (int q = 0; q < NM; ++q) m[(size_t)l * P * NM + q] = 0.0;
      continue;
    }
    tensor_moments_ml<R, OP, LM>(A, B, n, M.alpha, *TN, m, P * NM);
  }
  __syncthreads();
  for (int l = 0; l < nl; ++l)
    tile_entries<OP, T>(M, rt, ct, r0, c0, mom + (size_t)l * P * NM, (size_t)(d0 + l) * N * N, out, mirrored);
}

// Lags 0 and 1 of one tile together (FP64 compute): regular and near pairs
// integrated once for both lags, identical and vertex-sharing pairs from the
// singular-pair buffer; then each lag's entries.
template <int OP, typename T>
__device__ void tile_body_01(const DevMesh& M, int tile, const double* __restrict__ sing, T* __restrict__ out,
                             unsigned char* smem_raw) {
  constexpr int P = Tile<OP>::pairs, NM = Tile<OP>::nm;
  double* mom = reinterpret_cast<double*>(smem_raw);
  const int N = M.N;
  int rt, ct;
  if (OP == STBEM_OP_K) {
    const int nP = (N + kKP - 1) / kKP;
    rt = tile / nP;
    ct = tile % nP;
  } else {
    upper_tile(tile, (N + kT - 1) / kT, &rt, &ct);
  }
  const int r0 = rt * kT, c0 = ct * (OP == STBEM_OP_K ? kKP : kT);
  for (int p = threadIdx.x; p < P; p += kTileThreads) {
    Piece A, B;
    int ia, ib, ring;
    double* m = mom + (size_t)p * NM;
    if (!tile_pair<OP>(M, r0, c0, p, &A, &B, &ia, &ib, &ring)) {
      for (int l = 0; l < 2; ++l)
        for (int q = 0; q < NM; ++q) m[(size_t)l * P * NM + q] = 0.0;
      continue;
    }
    const int cls = pair_class(ring, ia, ib, A, B);
    if (cls == kIdentical || cls == kAdjNext || cls == kAdjPrev) {
      for (int l = 0; l < 2; ++l) {
        const double* src = sing + ((size_t)l * 3 * ring + singular_slot(cls, ia, ring)) * 5;
        for (int q = 0; q < NM; ++q) m[(size_t)l * P * NM + q] = src[q];
      }
      continue;
    }
    tensor_moments_01<OP>(A, B, cls == kRegular ? kRegular01 : kNear01, M.ht, M.alpha, m, P * NM);
  }
  __syncthreads();
  for (int l = 0; l < 2; ++l)
    tile_entries<OP, T>(M, rt, ct, r0, c0, mom + (size_t)l * P * NM, (size_t)l * N * N, out);
}

template <int OP, typename T>
__global__ void __launch_bounds__(kTileThreads) k_tile_01(DevMesh M, const double* __restrict__ sing,
                                                          T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_body_01<OP, T>(M, blockIdx.x, sing, out, smem_raw);
}

template <int OP>
constexpr size_t tile_01_smem_bytes() {
  return (((size_t)2 * Tile<OP>::pairs * Tile<OP>::nm * sizeof(double) + 15) / 16) * 16;
}

template <int OP, typename R, typename T, int LM>
__global__ void __launch_bounds__(kTileThreads) k_tile_ml(DevMesh M, MLSegs S, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int d0, d_end;
  ml_chunk(S, LM, blockIdx.y, &d0, &d_end);
  tile_body_ml<OP, R, T, LM>(M, d0, min(LM, d_end - d0), blockIdx.x, out, smem_raw);
}

// Lag groups of one operator on n_t steps: lags 0 and 1 one at a time, then
// runs of up to LM consecutive lags that never cross the space-order changes
// at d = 8 and 32 (the same runs as the single-problem launches).
// (FP32 D keeps one lag per tile: its exponentials are cheap MUFU operations,
// so sharing intervals saves little and the doubled moment storage costs
// occupancy.)
template <int OP, typename R>
__host__ __device__ constexpr int lag_group_len() {
  return OP == STBEM_OP_D ? (sizeof(R) == 4 ? 1 : 4) : kMaxLagsML;   // D: 4 moment arrays fill shared memory
}

// (FP64: lags 0 and 1 form one group; FP32: one each, pair01 = false.)
__host__ __device__ inline int lag_groups(int nt, int LM, bool pair01) {
  int g = nt < 2 ? nt : (pair01 ? 1 : 2);
  const int seg[4] = {2, 8, 32, 1 << 30};
  for (int k = 0; k < 3; ++k) {
    const int lo = seg[k], hi = nt < seg[k + 1] ? nt : seg[k + 1];
    if (hi > lo) g += (hi - lo + LM - 1) / LM;
  }
  return g;
}

__host__ __device__ inline void lag_group(int nt, int LM, bool pair01, int g, int* d0, int* nl) {
  const int l01 = nt < 2 ? nt : (pair01 ? 1 : 2);
  if (g < l01) {
    *d0 = g;
    *nl = (pair01 && nt >= 2) ? 2 : 1;
    return;
  }
  g -= l01;
  const int seg[4] = {2, 8, 32, 1 << 30};
  for (int k = 0; k < 3; ++k) {
    const int lo = seg[k], hi = nt < seg[k + 1] ? nt : seg[k + 1];
    if (hi <= lo) continue;
    const int n = (hi - lo + LM - 1) / LM;
    if (g < n) {
      *d0 = lo + g * LM;
      *nl = (hi - *d0) < LM ? (hi - *d0) : LM;
      return;
    }
    g -= n;
  }
  *d0 = 0;
  *nl = 0;
}

template <int OP, typename R, typename T, bool LAG01>
__global__ void __launch_bounds__(kTileThreads) k_tile(DevMesh M, int d_begin, const double* __restrict__ sing,
                                                       T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_body<OP, R, T, LAG01>(M, d_begin + blockIdx.y, blockIdx.x, sing, out, smem_raw);
}

// ---- ragged batches: one persistent launch over the tiles of many problems --------
// Work items are (problem, lag, tile) in the order of the host's item table
// (largest problems first); CTAs take the next item from an atomic counter, so
// uneven problems balance dynamically.  Item k of the table belongs to the
// problem slot s with prefix[s] <= k < prefix[s + 1].
__device__ __forceinline__ int ragged_slot(const long long* __restrict__ prefix, int P, long long item) {
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int OP>
__global__ void __launch_bounds__(kSingThreads) k_ragged_singular(const RaggedProblem* __restrict__ probs,
                                                                  const int* __restrict__ order,
                                                                  const long long* __restrict__ prefix, int P,
                                                                  unsigned long long* __restrict__ counter) {
  __shared__ double red[5][kSingThreads];
  __shared__ long long item_s;
  const long long total = prefix[P];
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ULL);
    __syncthreads();
    const long long item = item_s;
    __syncthreads();
    if (item >= total) break;
    const int s = ragged_slot(prefix, P, item);
    const RaggedProblem& pr = probs[order[s]];
    const long long local = item - prefix[s];
    const int Rl = OP == STBEM_OP_D ? 2 * pr.M.N : pr.M.N;
    const int d = (int)(local / (3 * Rl)), slot = (int)(local % (3 * Rl));
    singular_body<OP>(pr.M, slot, d, pr.M.sing, red);
    __syncthreads();
  }
}

template <int OP, typename R, typename T>
__global__ void __launch_bounds__(kTileThreads) k_ragged_tile(const RaggedProblem* __restrict__ probs,
                                                              const int* __restrict__ order,
                                                              const long long* __restrict__ prefix, int P,
                                                              unsigned long long* __restrict__ counter,
                                                              T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long item_s;
  const long long total = prefix[P];
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ULL);
    __syncthreads();
    const long long item = item_s;
    __syncthreads();
    if (item >= total) break;
    const int s = ragged_slot(prefix, P, item);
    const RaggedProblem& pr = probs[order[s]];
    const long long local = item - prefix[s];
    const int nt_tiles = tiles_per_lag<OP>(pr.M.N);
    const int g = (int)(local / nt_tiles), t = (int)(local % nt_tiles);
    int d0, nl;
    constexpr int LM = lag_group_len<OP, R>();
    constexpr bool P01 = sizeof(R) == 8;
    lag_group(pr.M.n_t, LM, P01, g, &d0, &nl);
    T* o = out + pr.op_off;
    if (d0 == 0 && nl == 2) tile_body_01<OP, T>(pr.M, t, pr.M.sing, o, smem_raw);
    else if (d0 < 2) tile_body<OP, R, T, true>(pr.M, d0, t, pr.M.sing, o, smem_raw);
    else if (LM == 1) tile_body<OP, R, T, false>(pr.M, d0, t, pr.M.sing, o, smem_raw);
    else tile_body_ml<OP, R, T, LM>(pr.M, d0, nl, t, o, smem_raw);
    __syncthreads();
  }
}

// ---- non-uniform time grids -------------------------------------------------------
// Section 1 allows any decomposition 0 = t_0 < .. < t_{n_t} = T of (0, T).  The
// Galerkin block of test step m and trial step n <= m then depends on (m, n),
// not on m - n alone: blocks are stored packed, p = m (m + 1) / 2 + n.  Time:
// with s1 = t_{m+1} - t_n, s2 = t_{m+1} - t_{n+1}, s3 = t_m - t_n,
// s4 = t_m - t_{n+1} the integral over tau_m x tau_n is
// F(s1) - F(s2) - F(s3) + F(s4) (F = 0 for s <= 0); branches as the host-checked
// nonuniform_time.cuh: d = m - n = 0 closed; d = 1 the series form for
// z = c / s_c < 1 (s_c = (s1 + s4) / 2), else closed; d >= 2 closed when
// z > d / 2, else the Peano form over the trapezoid of the overlap length,
// whose nodes and weights (up to three linear pieces, peano_order nodes each)
// are tabulated per block as the uniform lag tables are.  Space: the uniform
// rule with the lag d (classes, orders, singular rules at d <= 1).
constexpr int kMaxNodesNU = 48;
struct BlockTime {
  int d, n;
  double s[4], inv_sc;
  double sig[kMaxNodesNU], wv[kMaxNodesNU], wk[kMaxNodesNU], w3[kMaxNodesNU], w2[kMaxNodesNU];
  // e^{-c sig} = exp_prod_fast(c, sigk) with sigk = sig 2048 / ln 2 while
  // c sigk_max < kExpProdMax; etab: the 2048-entry table in shared memory
  double sigk[kMaxNodesNU], sigk_max;
  const double* etab;
};

// e^{-c sig_g} of a block's Peano node g (fast: the table form applies to every node)
__device__ __forceinline__ double nu_exp(double c, const BlockTime& B, int g, bool fast) {
  return fast ? exp_prod_fast(c, B.sigk[g], B.etab) : exp_neg_fast(c * B.sig[g]);
}

__device__ __forceinline__ void nu_block_index(long long p, int* m, int* n) {
  int mm = (int)floor((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
  while ((long long)mm * (mm + 1) / 2 > p) --mm;
  while ((long long)(mm + 1) * (mm + 2) / 2 <= p) ++mm;
  *m = mm;
  *n = (int)(p - (long long)mm * (mm + 1) / 2);
}

// thread 0 builds the block's table (a few dozen nodes)
__device__ void build_block_time(BlockTime& B, const double* __restrict__ tn, int m, int n, double alpha) {
  if (threadIdx.x != 0) return;
  B.d = m - n;
  B.s[0] = tn[m + 1] - tn[n];
  B.s[1] = tn[m + 1] - tn[n + 1];
  B.s[2] = tn[m] - tn[n];
  B.s[3] = tn[m] - tn[n + 1];
  B.inv_sc = 1.0 / (0.5 * (B.s[0] + B.s[3]));
  int g = 0;
  if (B.d >= 2) {
    const double pt[4] = {B.s[3], fmin(B.s[1], B.s[2]), fmax(B.s[1], B.s[2]), B.s[0]};
    const double plateau = pt[1] - pt[0];
    for (int piece = 0; piece < 3; ++piece) {
      const double lo = pt[piece], L = pt[piece + 1] - pt[piece];
      if (!(L > 0.0)) continue;
      const int q = peano_order((int)rint(lo / L)), o = gauss_offset(q);
      for (int k = 0; k < q && g < kMaxNodesNU; ++k, ++g) {
        const double x = c_tab.gx[o + k];
        const double wt = piece == 0 ? x * L : (piece == 1 ? plateau : (1.0 - x) * L);
        const double sv = lo + x * L, sig = 1.0 / sv;
        const double W = L * c_tab.gw[o + k] * wt;
        B.sig[g] = sig;
        B.wv[g] = W * sig / kFourPi;
        B.wk[g] = W * alpha * sig * sig / (2.0 * kFourPi);
        B.w3[g] = W * alpha * sig * sig * sig / kFourPi;
        B.w2[g] = W * alpha * sig * sig / kFourPi;
      }
    }
  }
  B.n = g;
  B.sigk_max = 0.0;
  for (int k = 0; k < g; ++k) {
    B.sigk[k] = B.sig[k] * kInvLn2x2048;
    B.sigk_max = fmax(B.sigk_max, B.sigk[k]);
  }
}

template <int K>
__device__ __forceinline__ double nu_closed(double c, const BlockTime& B, double alpha) {
  const double a = Fk<K>(c, B.s[0], alpha) - Fk<K>(c, B.s[1], alpha);
  if (B.d == 1) return a - Fk<K>(c, B.s[2], alpha);
  return (a - Fk<K>(c, B.s[2], alpha)) + Fk<K>(c, B.s[3], alpha);
}

// kernel K (kV, kKq = K / q, k1) of the block at c = alpha r^2 / 4
template <int K>
__device__ double nu_kernel(double c, const BlockTime& B, double alpha) {
  if (B.d == 0) return Fk<K>(c, B.s[0], alpha);
  const double z = c * B.inv_sc;
  if (B.d == 1) return z < 1.0 ? nu_lag1_series<K>(c, B.s[0], B.s[1], B.s[2], alpha) : nu_closed<K>(c, B, alpha);
  if (z > 0.5 * (double)B.d) return nu_closed<K>(c, B, alpha);
  double acc = 0.0;
  const bool fast = c * B.sigk_max < kExpProdMax;
  for (int g = 0; g < B.n; ++g) {
    const double e = nu_exp(c, B, g, fast);
    if (K == kV) acc = fma(B.wv[g], e, acc);
    else if (K == kKq) acc = fma(B.wk[g], e, acc);
    else acc = fma(e, fma(B.w3[g], c, -B.w2[g]), acc);
  }
  return acc;
}

// D's two kernels (kV and k1) of the block: one exponential per Peano node
__device__ __forceinline__ void nu_kernel_D(double c, const BlockTime& B, double alpha, double* kv, double* k1v) {
  if (B.d >= 2 && !(c * B.inv_sc > 0.5 * (double)B.d)) {
    double av = 0.0, a1 = 0.0;
    const bool fast = c * B.sigk_max < kExpProdMax;
    for (int g = 0; g < B.n; ++g) {
      const double e = nu_exp(c, B, g, fast);
      av = fma(B.wv[g], e, av);
      a1 = fma(e, fma(B.w3[g], c, -B.w2[g]), a1);
    }
    *kv = av;
    *k1v = a1;
    return;
  }
  *kv = nu_kernel<kV>(c, B, alpha);
  *k1v = nu_kernel<k1>(c, B, alpha);
}

// moments of one regular / near pair (tensor Gauss rule of order n) of the block
template <int OP>
__device__ void nu_tensor_moments(const Piece& A, const Piece& Bp, int n, const BlockTime& B, double alpha,
                                  double* mom) {
  const int o = gauss_offset(n);
  const double eax = A.x1 - A.x0, eay = A.y1 - A.y0;
  const double ebx = Bp.x1 - Bp.x0, eby = Bp.y1 - Bp.y0;
  const double abx = A.x0 - Bp.x0, aby = A.y0 - Bp.y0;
  const double qab = (A.x0 - Bp.x0) * Bp.nx + (A.y0 - Bp.y0) * Bp.ny;
  const double qea = (A.x1 - A.x0) * Bp.nx + (A.y1 - A.y0) * Bp.ny;
  const double qa = 0.25 * alpha;
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
  for (int a = 0; a < n; ++a) {
    const double xi = c_tab.gx[o + a], wa = c_tab.gw[o + a];
    for (int b = 0; b < n; ++b) {
      const double eta = c_tab.gx[o + b];
      const double w = wa * c_tab.gw[o + b];
      const double dx = (abx + xi * eax) - eta * ebx;
      const double dy = (aby + xi * eay) - eta * eby;
      const double c = qa * (dx * dx + dy * dy);
      if constexpr (OP == STBEM_OP_V) {
        s0 += w * nu_kernel<kV>(c, B, alpha);
      } else if constexpr (OP == STBEM_OP_K) {
        const double wk = w * ((qab + xi * qea) * nu_kernel<kKq>(c, B, alpha));
        s0 += wk * (1.0 - eta);
        s1 += wk * eta;
      } else {
        double kv, k1v;
        nu_kernel_D(c, B, alpha, &kv, &k1v);
        s0 += w * kv;
        const double wk = w * k1v;
        s1 += wk * (1.0 - xi) * (1.0 - eta);
        s2 += wk * (1.0 - xi) * eta;
        s3 += wk * xi * (1.0 - eta);
        s4 += wk * xi * eta;
      }
    }
  }
  const double L = A.len * Bp.len;
  const double sv[5] = {s0, s1, s2, s3, s4};
  for (int q = 0; q < NMom<OP>::n; ++q) mom[q] = sv[q] * L;
}

// moments of one identical / vertex-sharing pair (d <= 1), the whole CTA
// striding over the rule's points, fixed-order tree reduction
template <int OP>
__device__ void nu_singular_moments(const Piece& A, const Piece& Bp, int cls, const BlockTime& B, double alpha,
                                    double* mom, double (*red)[kTileThreads]) {
  constexpr int NM = NMom<OP>::n;
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int np = singular_points(cls);
  for (int p = threadIdx.x; p < np; p += kTileThreads) {
    double xi, eta, w, dx, dy;
    singular_point(cls, p, A, Bp, &xi, &eta, &w, &dx, &dy);
    const double c = 0.25 * alpha * (dx * dx + dy * dy);
    if constexpr (OP == STBEM_OP_V) {
      s[0] += w * nu_kernel<kV>(c, B, alpha);
    } else if constexpr (OP == STBEM_OP_K) {
      const double wk = w * ((dx * Bp.nx + dy * Bp.ny) * nu_kernel<kKq>(c, B, alpha));
      s[0] += wk * (1.0 - eta);
      s[1] += wk * eta;
    } else {
      s[0] += w * nu_kernel<kV>(c, B, alpha);
      const double wk = w * nu_kernel<k1>(c, B, alpha);
      s[1] += wk * (1.0 - xi) * (1.0 - eta);
      s[2] += wk * (1.0 - xi) * eta;
      s[3] += wk * xi * (1.0 - eta);
      s[4] += wk * xi * eta;
    }
  }
  for (int q = 0; q < NM; ++q) red[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int h = kTileThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int q = 0; q < NM; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if ((int)threadIdx.x < NM) mom[threadIdx.x] = red[threadIdx.x][0] * (A.len * Bp.len);
  __syncthreads();
}

template <int OP>
constexpr size_t nu_tile_smem_bytes() {
  return (((size_t)Tile<OP>::pairs * Tile<OP>::nm * sizeof(double) + 15) / 16) * 16 + 2048 * sizeof(double) +
         sizeof(BlockTime);
}

// One tile of one block (m, n) = packed index p0 + blockIdx.y.
template <int OP>
__global__ void __launch_bounds__(kTileThreads) k_nu_tile(DevMesh M, const double* __restrict__ tn, long long p0,
                                                          double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[5][kTileThreads];
  __shared__ int sing[Tile<OP>::pairs];
  __shared__ int n_sing;
  constexpr int P = Tile<OP>::pairs, NM = Tile<OP>::nm;
  double* mom = reinterpret_cast<double*>(smem_raw);
  double* etab = reinterpret_cast<double*>(smem_raw + ((P * NM * sizeof(double) + 15) / 16) * 16);
  BlockTime* BT = reinterpret_cast<BlockTime*>(etab + 2048);
  const long long p = p0 + blockIdx.y;
  int m, n;
  nu_block_index(p, &m, &n);
  const int d = m - n;
  const int N = M.N;
  int rt, ct;
  if (OP == STBEM_OP_K) {
    const int nP = (N + kKP - 1) / kKP;
    rt = blockIdx.x / nP;
    ct = blockIdx.x % nP;
  } else {
    upper_tile(blockIdx.x, (N + kT - 1) / kT, &rt, &ct);
  }
  const int r0 = rt * kT, c0 = ct * (OP == STBEM_OP_K ? kKP : kT);
  build_block_time(*BT, tn, m, n, M.alpha);
  for (int k = threadIdx.x; k < 2048; k += kTileThreads) etab[k] = kExp2Tab2048[k];
  if (threadIdx.x == 0) {
    n_sing = 0;
    BT->etab = etab;
  }
  __syncthreads();
  // D at d >= 2 on a diagonal tile: the half-pair block is symmetric, integrate u <= v only
  const bool mirrored = OP == STBEM_OP_D && rt == ct && d >= 2;
  for (int q = threadIdx.x; q < P; q += kTileThreads) {
    if (mirrored && q % kDP < q / kDP) continue;
    Piece A, B;
    int ia, ib, ring;
    double* mq = mom + (size_t)q * NM;
    if (!tile_pair<OP>(M, r0, c0, q, &A, &B, &ia, &ib, &ring)) {
      for (int k = 0; k < NM; ++k) mq[k] = 0.0;
      continue;
    }
    int order = space_order(d);
    if (d <= 1) {
      const int cls = pair_class(ring, ia, ib, A, B);
      if (cls == kIdentical || cls == kAdjNext || cls == kAdjPrev) {
        sing[atomicAdd(&n_sing, 1)] = q;       // the whole CTA integrates it below
        continue;
      }
      order = cls == kRegular ? kRegular01 : kNear01;
    }
    nu_tensor_moments<OP>(A, B, order, *BT, M.alpha, mq);
  }
  __syncthreads();
  const int ns = n_sing;
  for (int k = 0; k < ns; ++k) {
    const int q = sing[k];
    Piece A, B;
    int ia, ib, ring;
    tile_pair<OP>(M, r0, c0, q, &A, &B, &ia, &ib, &ring);
    nu_singular_moments<OP>(A, B, pair_class(ring, ia, ib, A, B), *BT, M.alpha, mom + (size_t)q * NM, red);
  }
  __syncthreads();
  tile_entries<OP, double>(M, rt, ct, r0, c0, mom, (size_t)p * N * N, out, mirrored);
}

// y[m][i] = sum_{n <= m} sum_j A[p(m, n)][i][j] x[n][j]: one warp per (m, i)
// row, rows of the latest steps (the longest) first; coalesced row reads,
// lane partial sums reduced by shuffles in a fixed order.
__global__ void __launch_bounds__(256) k_nu_apply(int nt, int nx, const double* __restrict__ A,
                                                  const double* __restrict__ x, double* __restrict__ y) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long long)nt * nx) return;
  const int m = nt - 1 - (int)(warp / nx), i = (int)(warp % nx);
  double acc = 0.0;
  const size_t base_m = (size_t)m * (m + 1) / 2;
  for (int n = 0; n <= m; ++n) {
    const double* row = A + ((base_m + n) * nx + i) * (size_t)nx;
    const double* xn = x + (size_t)n * nx;
    for (int j = lane; j < nx; j += 32) acc = fma(row[j], xn[j], acc);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) y[(size_t)m * nx + i] = acc;
}

cudaError_t nu_assemble_launch(const DevMesh& M, const double* tn, int op, double* out, cudaStream_t s) {
  const int N = M.N, nt = M.n_t;
  const long long blocks = (long long)nt * (nt + 1) / 2;
  auto run = [&](auto kern, size_t smem, int tiles) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (long long p0 = 0; p0 < blocks; p0 += 65535) {
      const unsigned nb = (unsigned)std::min<long long>(65535, blocks - p0);
      kern<<<dim3(tiles, nb), kTileThreads, smem, s>>>(M, tn, p0, out);
      count_launches(1);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (op == STBEM_OP_V) return run(k_nu_tile<STBEM_OP_V>, nu_tile_smem_bytes<STBEM_OP_V>(), tiles_per_lag<STBEM_OP_V>(N));
  if (op == STBEM_OP_K) return run(k_nu_tile<STBEM_OP_K>, nu_tile_smem_bytes<STBEM_OP_K>(), tiles_per_lag<STBEM_OP_K>(N));
  return run(k_nu_tile<STBEM_OP_D>, nu_tile_smem_bytes<STBEM_OP_D>(), tiles_per_lag<STBEM_OP_D>(N));
}

cudaError_t nu_apply_launch(int nt, int nx, const double* A, const double* x, double* y, cudaStream_t s) {
  const long long threads = (long long)nt * nx * 32;
  const unsigned blocks = (unsigned)((threads + 255) / 256);
  k_nu_apply<<<blocks, 256, 0, s>>>(nt, nx, A, x, y);
  count_launches(1);
  return cudaGetLastError();
}

// ---- host side ----------------------------------------------------------------
cudaError_t upload_rule_tables(const RuleTables& t, cudaStream_t s) {
  cudaError_t e = cudaMemcpyToSymbolAsync(c_tab, &t, sizeof(RuleTables), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  float gxf[kGaussTotal], gwf[kGaussTotal];
  for (int i = 0; i < kGaussTotal; ++i) {
    gxf[i] = (float)t.gx[i];
    gwf[i] = (float)t.gw[i];
  }
  e = cudaMemcpyToSymbolAsync(c_gxf, gxf, sizeof(gxf), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbolAsync(c_gwf, gwf, sizeof(gwf), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);   // the host arrays above go out of scope
}

template <int OP, typename R, typename T>
static cudaError_t launch_op(const DevMesh& M, int lag_begin, int lag_end, T* out, cudaStream_t s) {
  const int N = M.N;
  const size_t smem = tile_smem_bytes<OP, R>();
  cudaError_t e = cudaFuncSetAttribute(k_tile<OP, R, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tile<OP, R, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int tiles;
  if (OP == STBEM_OP_K) {
    tiles = ((N + kT - 1) / kT) * ((N + kKP - 1) / kKP);
  } else {
    const int nT = (N + kT - 1) / kT;
    tiles = nT * (nT + 1) / 2;
  }
  // lags 0 and 1: FP64 singular pairs spread over the GPU, then the tiles
  const int l01 = lag_begin, u01 = lag_end < 2 ? lag_end : 2;
  if (l01 < u01) {
    const int Rl = OP == STBEM_OP_D ? 2 * N : N;
    k_singular<OP><<<dim3(3 * Rl, u01), kSingThreads, 0, s>>>(M, M.sing);
    if (sizeof(R) == 8 && l01 == 0 && u01 == 2) {
      // FP64: both lags in one pass (shared closed-form evaluations)
      const size_t smem01 = tile_01_smem_bytes<OP>();
      e = cudaFuncSetAttribute(k_tile_01<OP, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem01);
      if (e != cudaSuccess) return e;
      k_tile_01<OP, T><<<tiles, kTileThreads, smem01, s>>>(M, M.sing, out);
    } else {
      k_tile<OP, R, T, true><<<dim3(tiles, u01 - l01), kTileThreads, smem, s>>>(M, l01, M.sing, out);
    }
    count_launches(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // lags >= 2: L consecutive lags per CTA, each chunk within one space order
  // (runs split at the order changes d = 8 and 32), all chunks in one launch
  constexpr int LM = lag_group_len<OP, R>();
  const size_t smem_ml = tile_ml_smem_bytes<OP, R, LM>();
  if (OP != STBEM_OP_V && LM > 1) {
    e = cudaFuncSetAttribute(k_tile_ml<OP, R, T, LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ml);
    if (e != cudaSuccess) return e;
  }
  const int seg[4] = {2, 8, 32, 1 << 30};
  MLSegs S{};
  int chunks = 0;
  for (int sg = 0; sg < 3; ++sg) {
    S.lo[sg] = std::max(std::max(lag_begin, 2), seg[sg]);
    S.hi[sg] = std::min(lag_end, seg[sg + 1]);
    S.n[sg] = S.hi[sg] > S.lo[sg] ? (S.hi[sg] - S.lo[sg] + LM - 1) / LM : 0;
    chunks += S.n[sg];
  }
  if (chunks == 0) return cudaSuccess;
  if (chunks > 65535) return cudaErrorInvalidConfiguration;
  if (OP == STBEM_OP_V) {
    const long long npair = (long long)N * (N + 1) / 2;
    k_lag2_V_ml<R, T><<<dim3((unsigned)((npair + 127) / 128), chunks), 128, 0, s>>>(M, S, LM, out);
    count_launches(1);
    return cudaGetLastError();
  }
  if (LM > 1) {
    k_tile_ml<OP, R, T, LM><<<dim3(tiles, chunks), kTileThreads, smem_ml, s>>>(M, S, out);
    count_launches(1);
    return cudaGetLastError();
  }
  for (int sg = 0; sg < 3; ++sg) {   // one lag per CTA
    if (S.n[sg] == 0) continue;
    k_tile<OP, R, T, false><<<dim3(tiles, S.hi[sg] - S.lo[sg]), kTileThreads, smem, s>>>(M, S.lo[sg], M.sing, out);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int assembly_lag_groups(int op, int prec, int nt) {
  if (prec == STBEM_F64)
    return lag_groups(nt, op == STBEM_OP_V   ? lag_group_len<STBEM_OP_V, double>()
                          : op == STBEM_OP_K ? lag_group_len<STBEM_OP_K, double>()
                                             : lag_group_len<STBEM_OP_D, double>(), true);
  return lag_groups(nt, op == STBEM_OP_V   ? lag_group_len<STBEM_OP_V, float>()
                        : op == STBEM_OP_K ? lag_group_len<STBEM_OP_K, float>()
                                           : lag_group_len<STBEM_OP_D, float>(), false);
}

int assembly_tiles_per_lag(int op, int N) {
  if (op == STBEM_OP_V) return tiles_per_lag<STBEM_OP_V>(N);
  if (op == STBEM_OP_K) return tiles_per_lag<STBEM_OP_K>(N);
  return tiles_per_lag<STBEM_OP_D>(N);
}

template <int OP, typename R, typename T>
static cudaError_t ragged_op(const RaggedProblem* probs, int P, RaggedItems si, RaggedItems ti,
                             unsigned long long* counters, T* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ragged_singular<OP>, kSingThreads, 0);
  if (e != cudaSuccess) return e;
  k_ragged_singular<OP><<<sms * (occ > 0 ? occ : 1), kSingThreads, 0, s>>>(probs, si.order, si.prefix, P, counters);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = std::max(std::max(tile_smem_bytes<OP, R>(), tile_ml_smem_bytes<OP, R, lag_group_len<OP, R>()>()),
                               sizeof(R) == 8 ? tile_01_smem_bytes<OP>() : (size_t)0);
  e = cudaFuncSetAttribute(k_ragged_tile<OP, R, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ragged_tile<OP, R, T>, kTileThreads, smem);
  if (e != cudaSuccess) return e;
  k_ragged_tile<OP, R, T><<<sms * (occ > 0 ? occ : 1), kTileThreads, smem, s>>>(probs, ti.order, ti.prefix, P,
                                                                                  counters + 1, out);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t ragged_assemble_launch(int op, int prec, const RaggedProblem* probs, int P, RaggedItems si,
                                   RaggedItems ti, unsigned long long* counters, void* out, cudaStream_t s) {
  if (prec == STBEM_F64) {
    double* o = static_cast<double*>(out);
    if (op == STBEM_OP_V) return ragged_op<STBEM_OP_V, double>(probs, P, si, ti, counters, o, s);
    if (op == STBEM_OP_K) return ragged_op<STBEM_OP_K, double>(probs, P, si, ti, counters, o, s);
    return ragged_op<STBEM_OP_D, double>(probs, P, si, ti, counters, o, s);
  }
  float* o = static_cast<float*>(out);
  if (op == STBEM_OP_V) return ragged_op<STBEM_OP_V, float>(probs, P, si, ti, counters, o, s);
  if (op == STBEM_OP_K) return ragged_op<STBEM_OP_K, float>(probs, P, si, ti, counters, o, s);
  return ragged_op<STBEM_OP_D, float>(probs, P, si, ti, counters, o, s);
}

cudaError_t assemble_launch(const DevMesh& M, int op, int prec, int lag_begin, int lag_end, void* out,
                            cudaStream_t s) {
  if (prec == STBEM_F64) {
    double* o = static_cast<double*>(out);
    if (op == STBEM_OP_V) return launch_op<STBEM_OP_V, double>(M, lag_begin, lag_end, o, s);
    if (op == STBEM_OP_K) return launch_op<STBEM_OP_K, double>(M, lag_begin, lag_end, o, s);
    return launch_op<STBEM_OP_D, double>(M, lag_begin, lag_end, o, s);
  }
  float* o = static_cast<float*>(out);
  if (op == STBEM_OP_V) return launch_op<STBEM_OP_V, float>(M, lag_begin, lag_end, o, s);
  if (op == STBEM_OP_K) return launch_op<STBEM_OP_K, float>(M, lag_begin, lag_end, o, s);
  return launch_op<STBEM_OP_D, float>(M, lag_begin, lag_end, o, s);
}

}  // namespace stbem
