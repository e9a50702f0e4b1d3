// Double time integrals of the heat kernels over two steps of a non-uniform
// time grid (Section 1 allows any decomposition of (0, T)).  For test step
// tau_m and trial step tau_n (n <= m, d = m - n) and a kernel G with second
// antiderivative F (timeint.cuh; F = 0 for s <= 0):
//   int_{tau_m} int_{tau_n} G(t - tau) = F(s1) - F(s2) - F(s3) + F(s4),
//   s1 = t_{m+1} - t_n, s2 = t_{m+1} - t_{n+1}, s3 = t_m - t_n, s4 = t_m - t_{n+1}.
// Branches (on a uniform grid they are timeint.cuh's, s_c = d ht):
//   d = 0: F(s1);
//   d = 1 (s4 = 0, s1 = s2 + s3), z = c / s_c < 1 with s_c = (s1 + s4) / 2:
//     the ln c terms of the closed form combined analytically, with
//     E1 = -gamma - ln z + Ein(z), E2 = e^{-z} - z E1 and s1 - s2 - s3 = 0;
//   d >= 2: the closed form when c / s_c > d / 2, else the Peano form
//     int w(s) G(s) ds over the overlap length w (a trapezoid on [s4, s1],
//     breaks at min(s2, s3) and max(s2, s3)), peano_order(k) Gauss nodes
//     per linear piece, k = rint(start / length).
#pragma once
#include "hd.cuh"
#include "rule.cuh"
#include "special.cuh"
#include "timeint.cuh"

namespace stbem {

// d = 1, z < 1: sum over (s1, +1), (s2, -1), (s3, -1) of the rearranged terms
template <int K>
STB_HD double nu_lag1_series(double c, double s1, double s2, double s3, double alpha) {
  const double s[3] = {s1, s2, s3};
  const double sg[3] = {1.0, -1.0, -1.0};
  const double lc = kEulerGamma + log(c);
  if (K == kV) {
    double acc = c * lc;
    for (int k = 0; k < 3; ++k) {
      const double z = c / s[k];
      acc += sg[k] * ((s[k] + c) * (log(s[k]) + ein_series(z)) - s[k] * expm1(-z));
    }
    return acc / kFourPi;
  }
  if (K == kKq) {
    double acc = -lc;
    for (int k = 0; k < 3; ++k) {
      const double z = c / s[k];
      acc += sg[k] * (s[k] * expm1(-z) / c - log(s[k]) - ein_series(z));
    }
    return alpha / (2.0 * kFourPi) * acc;
  }
  double acc = lc;
  for (int k = 0; k < 3; ++k) acc += sg[k] * (log(s[k]) + ein_series(c / s[k]));
  return alpha / kFourPi * acc;
}

// Peano form over the trapezoid of the overlap length; gx/gw: Gauss tables
template <int K>
STB_HD double nu_peano(double c, double s1, double s2, double s3, double s4, double alpha, const double* gx,
                       const double* gw) {
  const double p[4] = {s4, fmin(s2, s3), fmax(s2, s3), s1};
  const double plateau = p[1] - p[0];
  double out = 0.0;
  for (int piece = 0; piece < 3; ++piece) {
    const double lo = p[piece], L = p[piece + 1] - p[piece];
    if (!(L > 0.0)) continue;
    const int n = peano_order((int)rint(lo / L));
    const int o = gauss_offset(n);
    double acc = 0.0;
    for (int g = 0; g < n; ++g) {
      const double x = gx[o + g];
      const double wt = piece == 0 ? x * L : (piece == 1 ? plateau : (1.0 - x) * L);
      acc += gw[o + g] * wt * Gk<K>(c, lo + x * L, alpha);
    }
    out += L * acc;
  }
  return out;
}

// The block (m, n) time integral for kernel K at c = alpha r^2 / 4 (K: / q).
template <int K>
STB_HD double nu_time_integral(double c, int d, double s1, double s2, double s3, double s4, double alpha,
                               const double* gx, const double* gw) {
  if (d == 0) return Fk<K>(c, s1, alpha);
  const double z = c / (0.5 * (s1 + s4));
  if (d == 1) {
    if (z < 1.0) return nu_lag1_series<K>(c, s1, s2, s3, alpha);
    return (Fk<K>(c, s1, alpha) - Fk<K>(c, s2, alpha)) - Fk<K>(c, s3, alpha);
  }
  if (z > 0.5 * (double)d)
    return ((Fk<K>(c, s1, alpha) - Fk<K>(c, s2, alpha)) - Fk<K>(c, s3, alpha)) + Fk<K>(c, s4, alpha);
  return nu_peano<K>(c, s1, s2, s3, s4, alpha, gx, gw);
}

}  // namespace stbem
