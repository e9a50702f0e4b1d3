// Values and c-derivatives of the double time integrals of the V and K kernels
// (timeint.cuh), for the shape and alpha gradients.  Every entry depends on the
// geometry and on alpha through c = alpha r^2 / 4 (and for K also through q and
// an explicit factor alpha), so each branch is differentiated in c.  With
// E1' = -e^{-z}/z and E2' = -E1, z = c / s:
//   d/dc F_V(c, s)  = -E2(z) / (4 pi z)
//   d/dc F_Kq(c, s) = -alpha / (8 pi c) (E2(z)/z + E1(z))
//   d/dc G(c, s)    = -G(c, s) / s          (Peano form, G = e^{-c/s} x f(s))
// Lag 1, z = c / ht (d/dc = (1/ht) d/dz):
//   V, z < 1: (1/(4 pi)) [gamma + ln(2z) + Ein(z/2) - 2 Ein(z) + (2/z) e^{-z/2} expm1(-z/2)]
//             (the log terms of E1(z/2) - 2 E1(z) combined analytically);
//   K, every z: D2_1 F_Kq = alpha (E2(z/2) - E2(z)) / (4 pi z), whose z-derivative
//             simplifies to -alpha (e^{-z/2} - e^{-z}) / (4 pi z^2), and
//             e^{-z/2} - e^{-z} = -e^{-z/2} expm1(-z/2) has no cancellation.
#pragma once
#include "hd.cuh"
#include "special.cuh"
#include "timeint.cuh"

namespace stbem {

// value (D2_d F) and d/dc at lags 0 and 1, FP64; K = kV or kKq (divided by q)
template <int K>
STB_HD void dlag01(double c, int d, double ht, double alpha, double* k, double* dk) {
  if (d == 0) {
    const double z = c / ht;
    double a, b;
    e1e2(z, &a, &b);
    if (K == kV) {
      *k = ht / kFourPi * (a - b);
      *dk = -b / (kFourPi * z);
    } else {
      *k = alpha / (2.0 * kFourPi * c) * ht * b;
      *dk = -alpha / (2.0 * kFourPi * c) * (b / z + a);
    }
    return;
  }
  const double z = c / ht;
  if (K == kV) {
    if (z < 1.0) {
      const double eh = ein_series(0.5 * z), ef = ein_series(z);
      const double ex = exp_neg_fast(0.5 * z), em = expm1(-0.5 * z);
      const double lg = kEulerGamma + log(2.0 * z);
      *k = ht / (2.0 * kPi) * (log(2.0) + eh - ef + 0.5 * z * (lg + eh - 2.0 * ef) + ex * em);
      *dk = (lg + eh - 2.0 * ef + 2.0 / z * ex * em) / kFourPi;
    } else {
      double a2, b2, a1, b1;
      e1e2(0.5 * z, &a2, &b2);
      e1e2(z, &a1, &b1);
      *k = 2.0 * ht / kFourPi * (a2 - b2) - 2.0 * (ht / kFourPi * (a1 - b1));
      *dk = -(b2 - b1) / (2.0 * kPi * z);
    }
  } else {
    *k = lag_kernel<kKq>(c, 1, ht, alpha, nullptr, nullptr);
    *dk = alpha / (kFourPi * ht) * exp_neg_fast(0.5 * z) * expm1(-0.5 * z) / (z * z);
  }
}

// closed-form value and d/dc of F at one time s (lags >= 2)
template <int K>
STB_HD void dF_closed(double c, double s, double inv_s, double alpha, double* f, double* df) {
  const double z = c * inv_s;
  double a, b;
  e1e2(z, &a, &b);
  if (K == kV) {
    *f = s / kFourPi * (a - b);
    *df = -b / (kFourPi * z);
  } else {
    const double pre = alpha / (2.0 * kFourPi * c);
    *f = pre * s * b;
    *df = -pre * (b / z + a);
  }
}

}  // namespace stbem
