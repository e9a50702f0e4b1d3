#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace stbem {
// The block-Toeplitz product y_n = sum_{d<=n} A_d x_{n-d} (V_h, K_h, D_h are
// block lower triangular, Section 3, and on a uniform grid Toeplitz in time,
// the integrals of eq. (4) depending on t - s only) is a linear convolution
// in the time index.  With L the smallest power of two >= 2 n_t
// the zero-padded circular convolution of length L equals it on n < n_t, so
// with w = e^{-2 pi i / L} and the frequency blocks
//     Ahat_k = sum_{d < n_t} A_d w^{d k},   k = 0 .. L/2
// (the rest follow by Hermitian symmetry, the A_d being real) one product is
// a real FFT of x along time, one complex N_x x N_x matrix-vector product per
// frequency, and an inverse real FFT.
constexpr int kFftMaxSteps = 4096;    // n_t <= 4096 (L <= 8192)
constexpr int kFftMaxSpace = 8192;    // N_x <= 8192 (one frequency's x in shared memory)
int fft_len(int nt);                  // L: smallest power of two >= 2 n_t
inline int fft_freqs(int nt) { return fft_len(nt) / 2 + 1; }
// bytes of the frequency blocks: (L/2 + 1) N_x^2 complex doubles
size_t fft_operator_bytes(int nt, int nx);
// scratch of one product: the transforms of x and y, 2 n_rhs (L/2 + 1) N_x complex doubles
size_t fft_apply_bytes(int nt, int nx, int n_rhs);
// Ahat[k][i][j] from the lag blocks A[d][i][j] (FP64, or FP32 with prec STBEM_F32)
cudaError_t fft_operator_launch(int prec, int nt, int nx, const void* A, double2* Ahat, cudaStream_t s);
// y = A x (trans: A^T x, y_n = sum_d A_d^T x_{n+d}) for n_rhs right-hand sides
// x[r][n][j], through the frequency blocks; work: fft_apply_bytes, 16-byte aligned
cudaError_t fft_apply_launch(bool trans, int nt, int nx, int n_rhs, const double2* Ahat, const double* x,
                             double* y, void* work, cudaStream_t s);
}  // namespace stbem
