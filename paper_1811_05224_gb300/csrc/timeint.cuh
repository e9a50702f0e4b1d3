// Double time integrals of the heat kernels over two uniform time steps at lag
// d (Section 1: fundamental solution U*; eq. (2)/(3) scalings).  With
// c = alpha r^2 / 4 and second antiderivatives F (F'' = G, F = 0 for s <= 0):
//   V: G = (1/alpha) U*            F_V = s/(4 pi) [E1(c/s) - E2(c/s)]
//   K: G = (1/alpha) d_{n_y} U*/q  F_K = alpha/(8 pi c) s E2(c/s)      (q = (x-y).n_y)
//   D: G = d_s U*                  F_1 = alpha/(4 pi) E1(c/s)          (time term of D_h)
// the exact integral over tau_m x tau_n is F((d+1)ht) - 2F(d ht) + F((d-1)ht).
// Branches: d = 0 closed; d = 1: z = c/ht < 1 uses the series form in which the
// log c terms cancel analytically, else closed; d >= 2: closed if
// c/(d ht) > d/2, else the Peano form
//   int_{(d-1)ht}^{(d+1)ht} (ht - |s - d ht|) G(s) ds
// with Gauss nodes on each of the two intervals.
#pragma once
#include "hd.cuh"
#include "rule.cuh"
#include "special.cuh"

namespace stbem {

enum Kern { kV = 0, kKq = 1, k1 = 2 };

STB_HD double F_V(double c, double s) {
  double a, b;
  e1e2(c / s, &a, &b);
  return s / kFourPi * (a - b);
}
STB_HD double F_Kq(double c, double s, double alpha) {
  double a, b;
  e1e2(c / s, &a, &b);
  return alpha / (2.0 * kFourPi * c) * s * b;
}
STB_HD double F_1(double c, double s, double alpha) {
  return alpha / kFourPi * e1_only(c / s);
}

template <int K>
STB_HD double Fk(double c, double s, double alpha) {
  return K == kV ? F_V(c, s) : (K == kKq ? F_Kq(c, s, alpha) : F_1(c, s, alpha));
}

template <int K>
STB_HD double Gk(double c, double s, double alpha) {
  const double e = exp_neg_fast(c / s);
  if (K == kV) return e / (kFourPi * s);
  if (K == kKq) return alpha * e / (2.0 * kFourPi * s * s);
  return alpha / kFourPi * e * (c / (s * s * s) - 1.0 / (s * s));
}

// Peano form at lag d >= 2; gx/gw: Gauss tables (rule.cuh layout).
template <int K>
STB_HD double peano(double c, int d, double ht, double alpha, const double* gx, const double* gw) {
  const int nl = peano_order(d - 1), nr = peano_order(d);
  const int ol = gauss_offset(nl), orr = gauss_offset(nr);
  double left = 0.0, right = 0.0;
  for (int g = 0; g < nl; ++g) {
    const double t = gx[ol + g];
    left += gw[ol + g] * t * Gk<K>(c, ((double)(d - 1) + t) * ht, alpha);
  }
  for (int g = 0; g < nr; ++g) {
    const double t = gx[orr + g];
    right += gw[orr + g] * (1.0 - t) * Gk<K>(c, ((double)d + t) * ht, alpha);
  }
  return ht * ht * (left + right);
}

// Series forms at lag 1 for z = c / ht < 1.
template <int K>
STB_HD double lag1_series(double z, double ht, double alpha) {
  const double eh = ein_series(0.5 * z), ef = ein_series(z);
  if (K == kV)
    return ht / (2.0 * kPi) *
           (log(2.0) + eh - ef + 0.5 * z * (kEulerGamma + log(2.0 * z) + eh - 2.0 * ef) +
            exp_neg_fast(0.5 * z) * expm1(-0.5 * z));
  if (K == kKq)
    return alpha / kFourPi *
           (-exp_neg_fast(0.5 * z) * expm1(-0.5 * z) / z - 0.5 * (kEulerGamma + log(2.0 * z)) - 0.5 * eh + ef);
  return alpha / kFourPi * (kEulerGamma + log(2.0 * z) + eh - 2.0 * ef);
}

// D2_d F for kernel K at c = alpha r^2 / 4 (for K: divided by q).
template <int K>
STB_HD double lag_kernel(double c, int d, double ht, double alpha, const double* gx, const double* gw) {
  if (d == 0) return Fk<K>(c, ht, alpha);
  if (d == 1) {
    const double z = c / ht;
    if (z < 1.0) return lag1_series<K>(z, ht, alpha);
    return Fk<K>(c, 2.0 * ht, alpha) - 2.0 * Fk<K>(c, ht, alpha);
  }
  const double zd = c / ((double)d * ht);
  if (zd > 0.5 * (double)d) {
    const double f = Fk<K>(c, (double)(d + 1) * ht, alpha) - 2.0 * Fk<K>(c, (double)d * ht, alpha);
    return f + Fk<K>(c, (double)(d - 1) * ht, alpha);
  }
  return peano<K>(c, d, ht, alpha, gx, gw);
}

}  // namespace stbem
