// Host build of the CUDA path's device numerics (special.cuh, timeint.cuh,
// rules_host.cpp) for CPU tests: the same source, compiled for the host.
#include "dtimeint.cuh"
#include "nonuniform_time.cuh"
namespace stbem { void build_rule_tables(RuleTables* t); }
static stbem::RuleTables T;
extern "C" {
void nc_init() { stbem::build_rule_tables(&T); }
void nc_exp_neg(const double* x, int n, double* out) { for (int i = 0; i < n; ++i) out[i] = stbem::exp_neg_fast(x[i]); }
void nc_exp_prod(const double* c, const double* k, int n, double* out) {
  for (int i = 0; i < n; ++i) out[i] = stbem::exp_prod_fast(c[i], k[i], stbem::kExp2Tab2048);
}
void nc_e1e2(const double* z, int n, double* e1, double* e2) { for (int i = 0; i < n; ++i) stbem::e1e2(z[i], e1 + i, e2 + i); }
void nc_e1only(const double* z, int n, double* e1) { for (int i = 0; i < n; ++i) e1[i] = stbem::e1_only(z[i]); }
void nc_e1e2f(const float* z, int n, float* e1, float* e2) { for (int i = 0; i < n; ++i) stbem::e1e2_f(z[i], e1 + i, e2 + i); }
void nc_ein(const double* z, int n, double* out) { for (int i = 0; i < n; ++i) out[i] = stbem::ein_series(z[i]); }
void nc_lag(int kind, const double* c, int n, int d, double ht, double alpha, double* out) {
  for (int i = 0; i < n; ++i)
    out[i] = kind == 0 ? stbem::lag_kernel<stbem::kV>(c[i], d, ht, alpha, T.gx, T.gw)
           : kind == 1 ? stbem::lag_kernel<stbem::kKq>(c[i], d, ht, alpha, T.gx, T.gw)
                       : stbem::lag_kernel<stbem::k1>(c[i], d, ht, alpha, T.gx, T.gw);
}
// lags 0, 1: dlag01 (value and c-derivative); lags >= 2, closed branch: the
// second difference of dF_closed
void nc_dlag(int kind, const double* c, int n, int d, double ht, double alpha, double* k, double* dk) {
  for (int i = 0; i < n; ++i) {
    if (d <= 1) {
      if (kind == 0) stbem::dlag01<stbem::kV>(c[i], d, ht, alpha, k + i, dk + i);
      else stbem::dlag01<stbem::kKq>(c[i], d, ht, alpha, k + i, dk + i);
      continue;
    }
    double f[3], df[3];
    for (int q = 0; q < 3; ++q) {
      const double s = (double)(d + 1 - q) * ht;
      if (kind == 0) stbem::dF_closed<stbem::kV>(c[i], s, 1.0 / s, alpha, &f[q], &df[q]);
      else stbem::dF_closed<stbem::kKq>(c[i], s, 1.0 / s, alpha, &f[q], &df[q]);
    }
    k[i] = (f[0] - 2.0 * f[1]) + f[2];
    dk[i] = (df[0] - 2.0 * df[1]) + df[2];
  }
}
void nc_nu_time(int kind, const double* c, int n, int d, double s1, double s2, double s3, double s4,
                double alpha, double* out) {
  for (int i = 0; i < n; ++i)
    out[i] = kind == 0 ? stbem::nu_time_integral<stbem::kV>(c[i], d, s1, s2, s3, s4, alpha, T.gx, T.gw)
           : kind == 1 ? stbem::nu_time_integral<stbem::kKq>(c[i], d, s1, s2, s3, s4, alpha, T.gx, T.gw)
                       : stbem::nu_time_integral<stbem::k1>(c[i], d, s1, s2, s3, s4, alpha, T.gx, T.gw);
}
void nc_gauss(int n, double* x, double* w) {
  const int o = stbem::gauss_offset(n);
  for (int i = 0; i < n; ++i) { x[i] = T.gx[o + i]; w[i] = T.gw[o + i]; }
}
}
