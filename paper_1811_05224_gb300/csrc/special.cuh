// Exponential integrals E1, E2 and the entire function Ein, written from their
// definitions: E_n(z) = int_1^inf e^{-zt} t^{-n} dt.
//  * z < 1: E1(z) = -gamma - ln z + Ein(z), Ein(z) = sum_{k>=1} (-1)^{k+1} z^k/(k k!)
//    (Abramowitz & Stegun 5.1.11), and E2(z) = e^{-z} - z E1(z) (A&S 5.1.14);
//  * 1 <= z < 16: e^z E1 and e^z E2 from 26-term Chebyshev expansions on
//    [1,2], [2,4], [4,8], [8,16] (coefficients in expint_cheb.inc, generated
//    by gen_expint_tables.py in 40-digit arithmetic), Clenshaw summation;
//  * z >= 16: the continued fraction of A&S 5.1.22 in its even (contracted)
//    form, E_n(z) = e^{-z} / (z + n - 1 n / (z + n + 2 - 2 (n+1) / (z + n + 4 - ...))),
//    evaluated backward at a fixed depth of 14 (converged to < 1e-16 there).
//    The Lentz evaluation (Lentz, Appl. Opt. 15, 1976) of the same fraction is
//    kept as cf_e1e2 for checks.
// exp and log are the platform's; nothing here reproduces their internals.
#pragma once
#include "hd.cuh"
#include "expint_cheb.inc"

namespace stbem {

constexpr double kEulerGamma = 0.577215664901532860606512090082402431;
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kFourPi = 4.0 * 3.141592653589793238462643383279502884;

STB_HD double ein_series(double z) {
  double term = 1.0, acc = 0.0;
  for (int k = 1; k <= 30; ++k) {
    term = term * z / k;
    acc = acc + ((k & 1) ? term : -term) / k;
  }
  return acc;
}

// Lentz evaluation of the contracted continued fraction for E_n, n = 1 and 2
// together; returns the fractions without the e^{-z} factor.
STB_HD void cf_e1e2(double z, double* f1, double* f2) {
  const double tiny = 1e-300;
  double b1 = z + 1.0, b2 = z + 2.0;
  double c1 = 1.0 / tiny, c2 = 1.0 / tiny;
  double d1 = 1.0 / b1, d2 = 1.0 / b2;
  double h1 = d1, h2 = d2;
  bool done1 = false, done2 = false;
  for (int i = 1; i <= 400 && !(done1 && done2); ++i) {
    if (!done1) {
      const double an = -(double)i * (double)i;          // -i (n - 1 + i), n = 1
      b1 += 2.0;
      d1 = 1.0 / (an * d1 + b1);
      c1 = b1 + an / c1;
      const double del = c1 * d1;
      h1 *= del;
      done1 = fabs(del - 1.0) < 1e-16;
    }
    if (!done2) {
      const double an = -(double)i * (double)(i + 1);    // n = 2
      b2 += 2.0;
      d2 = 1.0 / (an * d2 + b2);
      c2 = b2 + an / c2;
      const double del = c2 * d2;
      h2 *= del;
      done2 = fabs(del - 1.0) < 1e-16;
    }
  }
  *f1 = h1;
  *f2 = h2;
}

// Backward evaluation of the contracted fraction at fixed depth (z >= 16).
STB_HD double cf_backward(double z, int n) {
  constexpr int K = 14;
  double f = z + (double)n + 2.0 * K;
  for (int k = K; k >= 1; --k) {
    const double a = -(double)k * (double)(n - 1 + k);
    f = (z + (double)n + 2.0 * (double)(k - 1)) + a / f;
  }
  return 1.0 / f;
}

// Clenshaw sum of c0/2 + sum_{k>=1} c_k T_k(t).
STB_HD double cheb_sum(const double* c, double t) {
  double b1 = 0.0, b2 = 0.0;
  for (int k = kChebN - 1; k >= 1; --k) {
    const double b0 = c[k] + 2.0 * t * b1 - b2;
    b2 = b1;
    b1 = b0;
  }
  return 0.5 * c[0] + t * b1 - b2;
}

// E1(z), E2(z) for z > 0.
STB_HD void e1e2(double z, double* e1, double* e2) {
  if (z < 1.0) {
    const double E1 = -kEulerGamma - log(z) + ein_series(z);
    *e1 = E1;
    *e2 = exp(-z) - z * E1;
  } else if (z < 16.0) {
    const int k = z < 2.0 ? 0 : (z < 4.0 ? 1 : (z < 8.0 ? 2 : 3));
    const double a = (double)(1 << k);
    const double t = 2.0 * z / a - 3.0;
    const double ez = exp(-z);
    *e1 = cheb_sum(kChebE1[k], t) * ez;
    *e2 = cheb_sum(kChebE2[k], t) * ez;
  } else {
    const double ez = exp(-z);
    *e1 = cf_backward(z, 1) * ez;
    *e2 = cf_backward(z, 2) * ez;
  }
}

STB_HD double e1_only(double z) {
  double a, b;
  e1e2(z, &a, &b);
  return a;
}

}  // namespace stbem
