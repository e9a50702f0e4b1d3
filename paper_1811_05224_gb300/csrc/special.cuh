// Exponential integrals E1, E2 and the entire function Ein, written from their
// definitions: E_n(z) = int_1^inf e^{-zt} t^{-n} dt.
//  * z < 1: E1(z) = -gamma - ln z + Ein(z), Ein(z) = sum_{k>=1} (-1)^{k+1} z^k/(k k!)
//    (Abramowitz & Stegun 5.1.11), and E2(z) = e^{-z} - z E1(z) (A&S 5.1.14);
//    e^{-z} here and below from exp_neg_fast;
//  * 1 <= z < 16: e^z E1 and e^z E2 from 16-term Chebyshev fits on the
//    eight intervals [2^{k/2}, 2^{(k+1)/2}], converted to powers of the
//    interval variable (coefficients in expint_cheb.inc, generated by
//    gen_expint_tables.py in 40-digit arithmetic), Horner's rule;
//  * z >= 16: the continued fraction of A&S 5.1.22 in its even (contracted)
//    form, E_n(z) = e^{-z} / (z + n - 1 n / (z + n + 2 - 2 (n+1) / (z + n + 4 - ...))),
//    truncated at a fixed depth of 14 (converged to < 1e-16 there) and
//    evaluated by forward numerator / denominator recurrences (one division),
//    or backward from z = 700 on.
//    The Lentz evaluation (Lentz, Appl. Opt. 15, 1976) of the same fraction is
//    kept as cf_e1e2 for checks.
// exp and log are the platform's; nothing here reproduces their internals.
#pragma once
#include "hd.cuh"
#include <cstring>

#include "expint_cheb.inc"

namespace stbem {

constexpr double kEulerGamma = 0.577215664901532860606512090082402431;
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kFourPi = 4.0 * 3.141592653589793238462643383279502884;

// Ein(z) for |z| <= 1: Horner sum of the first 18 terms (the tail is below
// 1e-17 there); coefficients (-1)^{k+1} / (k k!) from expint_cheb.inc.
STB_HD double ein_series(double z) {
  double acc = kEinCoef[kEinTerms - 1];
  for (int k = kEinTerms - 2; k >= 0; --k) acc = fma(acc, z, kEinCoef[k]);
  return acc * z;
}

// e^{-x}, table-driven (Tang, ACM TOMS 15, 1989): x = n ln2/256 + r with
// |r| <= ln2/512 (two-part ln2/256 so that n ln2_hi is exact), then
// e^{-x} = 2^{-(n >> 8)} 2^{-(n & 255)/256} e^{-r}, the middle factor from a
// 256-entry table and e^{-r} from its Taylor polynomial of degree 4 (remainder
// |r|^5/120 < 4e-17).  The power of two is applied by subtracting n >> 8 from
// the exponent field (an integer operation): for x < 700 the table-times-
// polynomial value lies in [2^-2, 2) and the result stays a normal number.
// Results within 2 ulp of the correctly rounded value (checked on the host
// against the C library).  Arguments from 700 on go to the library exp.
STB_HD double exp_neg_fast(double x) {
  if (!(x < 700.0)) return exp(-x);
  const double nd = rint(x * kInvLn2x256);
  const int n = (int)nd;
  double r = fma(-nd, kLn2by256Hi, x);
  r = fma(-nd, kLn2by256Lo, r);
  double p = fma(r, 1.0 / 24.0, -1.0 / 6.0);
  p = fma(r, p, 0.5);
  p = fma(r, p, -1.0);
  p = fma(r, p, 1.0);
  const double t = kExp2Tab[n & 255] * p;
  long long bits;
#ifdef __CUDA_ARCH__
  bits = __double_as_longlong(t);
#else
  std::memcpy(&bits, &t, sizeof(bits));
#endif
  bits -= (long long)(n >> 8) << 52;
#ifdef __CUDA_ARCH__
  return __longlong_as_double(bits);
#else
  double out;
  std::memcpy(&out, &bits, sizeof(out));
  return out;
#endif
}

// e^{-c k} for the hot loops, k = sigma 2048/ln2 pre-scaled in a node table
// (the same table method with 2048 entries): t = fma(c, k, 1.5 2^52) rounds the
// exact product c k to the nearest integer n, the low word of t (no
// conversion instruction); r = fma(c, k, -n) is the exact remainder, |r| <= 1/2,
// rounded once; e^{-c k ln2/2048} = 2^{-(n >> 11)} 2^{-(n & 2047)/2048}
// e^{-r ln2/2048}, the last factor by its cubic Taylor polynomial (remainder
// below 4e-17).  The product c k is never rounded on its own, so only k's
// rounding (|x| eps, x = c sigma) enters besides the final 2 ulp; checked on
// the host.  Requires 0 <= c k < kExpProdMax (the caller tests it); tab: the
// 2048 values 2^{-j/2048} (kExp2Tab2048 or a copy in shared memory).
constexpr double kExpProdMax = 700.0 * kInvLn2x2048;
STB_HD double exp_prod_fast(double c, double k, const double* tab) {
  const double kRound = 6755399441055744.0;   // 1.5 2^52
  const double t = fma(c, k, kRound);
#ifdef __CUDA_ARCH__
  const double nd = __dsub_rn(t, kRound);
  const int n = __double2loint(t);
#else
  const double nd = t - kRound;
  long long tb;
  std::memcpy(&tb, &t, sizeof(tb));
  const int n = (int)(tb & 0xffffffffLL);
#endif
  const double r = fma(c, k, -nd);
  double p = fma(r, kExpProdC3, kExpProdC2);
  p = fma(r, p, kExpProdC1);
  p = fma(r, p, 1.0);
  const double v = tab[n & 2047] * p;
  long long bits;
#ifdef __CUDA_ARCH__
  bits = __double_as_longlong(v);
#else
  std::memcpy(&bits, &v, sizeof(bits));
#endif
  bits -= (long long)(n >> 11) << 52;
#ifdef __CUDA_ARCH__
  return __longlong_as_double(bits);
#else
  double out;
  std::memcpy(&out, &bits, sizeof(out));
  return out;
#endif
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

// The same depth-14 convergent by the forward recurrences of its numerators
// and denominators (the fundamental recurrence formulas), P_j = b_j P_{j-1} +
// a_j P_{j-2} and likewise Q_j, with one division at the end instead of one per
// level; both functions n = 1, 2 together.  For 16 <= z < 700 the P_j stay
// below (z + 28)^14 < 1e41.  Returns the reciprocals 1 / f (as cf_backward).
STB_HD void cf_forward12(double z, double* r1, double* r2) {
  constexpr int K = 14;
  double p1m = 1.0, q1m = 0.0, p1 = z + 1.0, q1 = 1.0;   // n = 1: b_j = z + 1 + 2 j
  double p2m = 1.0, q2m = 0.0, p2 = z + 2.0, q2 = 1.0;   // n = 2: b_j = z + 2 + 2 j
  for (int j = 1; j <= K; ++j) {
    const double b1 = z + 1.0 + 2.0 * (double)j, a1 = -(double)j * (double)j;
    const double b2 = z + 2.0 + 2.0 * (double)j, a2 = -(double)j * (double)(j + 1);
    const double np1 = fma(b1, p1, a1 * p1m), nq1 = fma(b1, q1, a1 * q1m);
    const double np2 = fma(b2, p2, a2 * p2m), nq2 = fma(b2, q2, a2 * q2m);
    p1m = p1; q1m = q1; p1 = np1; q1 = nq1;
    p2m = p2; q2m = q2; p2 = np2; q2 = nq2;
  }
  *r1 = q1 / p1;
  *r2 = q2 / p2;
}

// sum_j a_j t^j, j < kHornN, by Horner's rule
STB_HD double horner_sum(const double* a, double t) {
  double p = a[kHornN - 1];
  for (int j = kHornN - 2; j >= 0; --j) p = fma(p, t, a[j]);
  return p;
}


// Interval of the FP64 Chebyshev tables for 1 <= z < 16: [a_k, a_{k+1}],
// a_k = 2^{k/2} (the split inside each octave [2^e, 2^{e+1}) at sqrt 2 2^e).
STB_HD int cheb_interval(double z) {
  const int e = z < 2.0 ? 0 : (z < 4.0 ? 1 : (z < 8.0 ? 2 : 3));
  return 2 * e + (z >= kChebSplit[e] ? 1 : 0);
}

// E1(z), E2(z) for z > 0.
STB_HD void e1e2(double z, double* e1, double* e2) {
  if (z < 1.0) {
    const double E1 = -kEulerGamma - log(z) + ein_series(z);
    *e1 = E1;
    *e2 = exp_neg_fast(z) - z * E1;
  } else if (z < 16.0) {
    const int k = cheb_interval(z);
    const double t = fma(z, kChebS[k], kChebO[k]);
    const double ez = exp_neg_fast(z);
    *e1 = horner_sum(kHornE1[k], t) * ez;
    *e2 = horner_sum(kHornE2[k], t) * ez;
  } else if (z < 700.0) {
    const double ez = exp_neg_fast(z);
    double r1, r2;
    cf_forward12(z, &r1, &r2);
    *e1 = r1 * ez;
    *e2 = r2 * ez;
  } else {
    const double ez = exp_neg_fast(z);
    *e1 = cf_backward(z, 1) * ez;
    *e2 = cf_backward(z, 2) * ez;
  }
}

// E1 alone: the E1 half of e1e2, the same operations in the same order
// (bitwise the same value), without the E2 work.
STB_HD double e1_only(double z) {
  if (z < 1.0) return -kEulerGamma - log(z) + ein_series(z);
  if (z < 16.0) {
    const int k = cheb_interval(z);
    const double t = fma(z, kChebS[k], kChebO[k]);
    return horner_sum(kHornE1[k], t) * exp_neg_fast(z);
  }
  const double ez = exp_neg_fast(z);
  if (z < 700.0) {
    constexpr int K = 14;
    double pm = 1.0, qm = 0.0, p = z + 1.0, q = 1.0;
    for (int j = 1; j <= K; ++j) {
      const double b = z + 1.0 + 2.0 * (double)j, a = -(double)j * (double)j;
      const double np = fma(b, p, a * pm), nq = fma(b, q, a * qm);
      pm = p; qm = q; p = np; q = nq;
    }
    return (q / p) * ez;
  }
  return cf_backward(z, 1) * ez;
}

// ---- FP32 versions (mixed-precision assembly) ----------------------------------
// Same definitions in single precision: 12-term series for z < 1, the leading
// 12 Chebyshev coefficients on [1,16], a depth-9 continued fraction beyond.
// Relative accuracy about 1e-6, well inside the FP32 assembly tolerance.

STB_HD float ein_series_f(float z) {
  float term = 1.0f, acc = 0.0f;
  for (int k = 1; k <= 12; ++k) {
    term = term * z * (1.0f / (float)k);
    acc = acc + ((k & 1) ? term : -term) * (1.0f / (float)k);
  }
  return acc;
}

STB_HD float exp_neg_f(float x) {   // e^{-x}
#ifdef __CUDA_ARCH__
  return __expf(-x);
#else
  return expf(-x);
#endif
}

STB_HD float cheb_sum_f(const float* c, float t) {
  float b1 = 0.0f, b2 = 0.0f;
  for (int k = kChebNf - 1; k >= 1; --k) {
    const float b0 = c[k] + 2.0f * t * b1 - b2;
    b2 = b1;
    b1 = b0;
  }
  return 0.5f * c[0] + t * b1 - b2;
}

STB_HD float cf_backward_f(float z, int n) {
  constexpr int K = 9;
  float f = z + (float)n + 2.0f * K;
  for (int k = K; k >= 1; --k) {
    const float a = -(float)k * (float)(n - 1 + k);
    f = (z + (float)n + 2.0f * (float)(k - 1)) + a / f;
  }
  return 1.0f / f;
}

STB_HD void e1e2_f(float z, float* e1, float* e2) {
  if (z < 1.0f) {
    const float E1 = -(float)kEulerGamma - logf(z) + ein_series_f(z);
    *e1 = E1;
    *e2 = exp_neg_f(z) - z * E1;
  } else if (z < 16.0f) {
    const int k = z < 2.0f ? 0 : (z < 4.0f ? 1 : (z < 8.0f ? 2 : 3));
    const float t = 2.0f * z * (1.0f / (float)(1 << k)) - 3.0f;
    const float ez = exp_neg_f(z);
    *e1 = cheb_sum_f(kChebE1f[k], t) * ez;
    *e2 = cheb_sum_f(kChebE2f[k], t) * ez;
  } else {
    const float ez = exp_neg_f(z);
    *e1 = cf_backward_f(z, 1) * ez;
    *e2 = cf_backward_f(z, 2) * ez;
  }
}

}  // namespace stbem
