// Host generation of the quadrature tables of rule.cuh.
// Gauss-Legendre nodes: Newton iteration on P_n (three-term recurrence) from
// the Tricomi-type initial guess cos(pi (k - 1/4) / (n + 1/2)), weights
// 2 / ((1 - x^2) P_n'(x)^2), mapped to [0,1] and sorted ascending.
#include <algorithm>
#include <cmath>

#include "rule.cuh"

namespace stbem {

static void gauss_legendre01(int n, double* x01, double* w01) {
  for (int k = 0; k < n; ++k) {
    long double x = std::cos(3.14159265358979323846264338327950288L * (k + 0.75L) / (n + 0.5L));
    long double dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1.0L, p1 = x;
      for (int j = 2; j <= n; ++j) {
        const long double p2 = ((2.0L * j - 1.0L) * x * p1 - (j - 1.0L) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0L);
      const long double dx = p1 / dp;
      x -= dx;
      if (std::fabs((double)dx) < 1e-19) {
        // one more evaluation of the derivative at the converged node
        p0 = 1.0L; p1 = x;
        for (int j = 2; j <= n; ++j) {
          const long double p2 = ((2.0L * j - 1.0L) * x * p1 - (j - 1.0L) * p0) / j;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0L);
        break;
      }
    }
    x01[k] = (double)(0.5L * (x + 1.0L));
    w01[k] = (double)(1.0L / ((1.0L - x * x) * dp * dp));   // (2 / (...)) / 2 on [0,1]
  }
  // ascending order
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b)
      if (x01[b] < x01[a]) {
        std::swap(x01[a], x01[b]);
        std::swap(w01[a], w01[b]);
      }
}

void build_rule_tables(RuleTables* t) {
  for (int n : kGaussOrders) gauss_legendre01(n, t->gx + gauss_offset(n), t->gw + gauss_offset(n));
  // graded composite rule: breakpoints 0, s^L, s^(L-1), ..., s, 1
  double bps[kGradedLevels + 2];
  bps[0] = 0.0;
  for (int k = kGradedLevels, i = 1; k >= 1; --k, ++i) bps[i] = std::pow(kGradedSigma, (double)k);
  bps[kGradedLevels + 1] = 1.0;
  const double* g = t->gx + gauss_offset(kGradedPoints);
  const double* gw = t->gw + gauss_offset(kGradedPoints);
  int o = 0;
  for (int s = 0; s <= kGradedLevels; ++s) {
    const double a = bps[s], b = bps[s + 1];
    for (int q = 0; q < kGradedPoints; ++q, ++o) {
      t->grx[o] = a + (b - a) * g[q];
      t->grw[o] = (b - a) * gw[q];
    }
  }
}

}  // namespace stbem
