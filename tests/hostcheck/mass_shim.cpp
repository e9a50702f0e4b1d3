// Host build of the mixed-mass numerics (mass_host.h) for CPU tests.
#include "mass_host.h"
extern "C" {
void mh_matrix(const double* h, int N, double ht, double* A) {
  const std::vector<double> M = stbem::mixed_mass_matrix(std::vector<double>(h, h + N), ht);
  for (size_t k = 0; k < M.size(); ++k) A[k] = M[k];
}
int mh_inverse(const double* h, int N, double ht, double* Inv) {
  std::vector<double> A = stbem::mixed_mass_matrix(std::vector<double>(h, h + N), ht), I;
  if (!stbem::gauss_jordan_inverse(A, N, I)) return 0;
  for (size_t k = 0; k < I.size(); ++k) Inv[k] = I[k];
  return 1;
}
}
