// Exponential integrals E1, E2 and the entire function Ein, written from their
// definitions: E_n(z) = int_1^inf e^{-zt} t^{-n} dt.
//  * z < 1: E1(z) = -gamma - ln z + Ein(z), Ein(z) = sum_{k>=1} (-1)^{k+1} z^k/(k k!)
//    (Abramowitz & Stegun 5.1.11), and E2(z) = e^{-z} - z E1(z) (A&S 5.1.14);
//  * z >= 1: the continued fraction of A&S 5.1.22 in its even (contracted)
//    form, E_n(z) = e^{-z} / (z + n - 1 n / (z + n + 2 - 2 (n+1) / (z + n + 4 - ...))),
//    evaluated by Lentz's method (Lentz, Appl. Opt. 15, 1976) to relative
//    convergence 1e-16.
// exp and log are the platform's; nothing here reproduces their internals.
#pragma once
#include "hd.cuh"

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

// E1(z), E2(z) for z > 0.
STB_HD void e1e2(double z, double* e1, double* e2) {
  if (z < 1.0) {
    const double E1 = -kEulerGamma - log(z) + ein_series(z);
    *e1 = E1;
    *e2 = exp(-z) - z * E1;
  } else {
    double f1, f2;
    cf_e1e2(z, &f1, &f2);
    const double ez = exp(-z);
    *e1 = f1 * ez;
    *e2 = f2 * ez;
  }
}

STB_HD double e1_only(double z) {
  double a, b;
  e1e2(z, &a, &b);
  return a;
}

}  // namespace stbem
