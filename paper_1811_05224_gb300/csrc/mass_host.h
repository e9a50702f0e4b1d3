// Host numerics of the consistent mixed mass M_h[l][k] = <phi^0_k, psi_l>
// (Section 2; the preconditioner M_h^{-1} D_h M_h^{-T} of Section 4): the
// cyclic tridiagonal matrix of one time step and its inverse.  Plain C++ (no
// CUDA), also compiled into the CPU tests.
#pragma once
#include <cmath>
#include <cstddef>
#include <utility>
#include <vector>

namespace stbem {

// M[l][k] = ht int_{gamma_k} psi_l: psi_l is linear on its four half-segments,
// with values a_l at x_l and b_l at x_{l+1} (the bends), 1 at the midpoint.
inline std::vector<double> mixed_mass_matrix(const std::vector<double>& h, double ht) {
  const int N = (int)h.size();
  std::vector<double> A((size_t)N * N, 0.0);
  for (int l = 0; l < N; ++l) {
    const int lm = (l - 1 + N) % N, lp = (l + 1) % N;
    const double a = h[lm] / (h[lm] + h[l]), b = h[lp] / (h[l] + h[lp]);
    A[(size_t)l * N + l] += ht * h[l] * (a + 2.0 + b) / 4.0;
    A[(size_t)l * N + lm] += ht * h[lm] * a / 4.0;
    A[(size_t)l * N + lp] += ht * h[lp] * b / 4.0;
  }
  return A;
}

// Inverse of the N x N row-major A by Gauss-Jordan elimination with partial
// pivoting (A is overwritten).  Returns false for a singular matrix.
inline bool gauss_jordan_inverse(std::vector<double>& A, int N, std::vector<double>& Inv) {
  Inv.assign((size_t)N * N, 0.0);
  for (int l = 0; l < N; ++l) Inv[(size_t)l * N + l] = 1.0;
  for (int c = 0; c < N; ++c) {
    int piv = c;
    for (int r = c + 1; r < N; ++r)
      if (std::fabs(A[(size_t)r * N + c]) > std::fabs(A[(size_t)piv * N + c])) piv = r;
    if (!(std::fabs(A[(size_t)piv * N + c]) > 0.0)) return false;
    if (piv != c)
      for (int k = 0; k < N; ++k) {
        std::swap(A[(size_t)c * N + k], A[(size_t)piv * N + k]);
        std::swap(Inv[(size_t)c * N + k], Inv[(size_t)piv * N + k]);
      }
    const double inv = 1.0 / A[(size_t)c * N + c];
    for (int k = 0; k < N; ++k) {
      A[(size_t)c * N + k] *= inv;
      Inv[(size_t)c * N + k] *= inv;
    }
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * N + c];
      if (f == 0.0) continue;
      for (int k = 0; k < N; ++k) {
        A[(size_t)r * N + k] -= f * A[(size_t)c * N + k];
        Inv[(size_t)r * N + k] -= f * Inv[(size_t)c * N + k];
      }
    }
  }
  return true;
}

}  // namespace stbem
