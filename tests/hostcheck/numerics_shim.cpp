// Host build of the CUDA path's device numerics (special.cuh, timeint.cuh,
// rules_host.cpp) for CPU tests: the same source, compiled for the host.
#include "timeint.cuh"
namespace stbem { void build_rule_tables(RuleTables* t); }
static stbem::RuleTables T;
extern "C" {
void nc_init() { stbem::build_rule_tables(&T); }
void nc_exp_neg(const double* x, int n, double* out) { for (int i = 0; i < n; ++i) out[i] = stbem::exp_neg_fast(x[i]); }
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
void nc_gauss(int n, double* x, double* w) {
  const int o = stbem::gauss_offset(n);
  for (int i = 0; i < n; ++i) { x[i] = T.gx[o + i]; w[i] = T.gw[o + i]; }
}
}
