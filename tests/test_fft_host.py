"""Host logic of the products through time FFTs (no CUDA call): the transform
length L (smallest power of two >= 2 n_t), the number of frequency blocks
L/2 + 1, the byte counts of the frequency blocks and of the workspaces, the
size limits; and the fact the length rests on, that the zero-padded circular
convolution of length L equals the linear one on the first n_t steps (the
block lower-triangular product of Section 3, Toeplitz in time on a uniform
grid, is a convolution in time), for the product and for its transpose (a
correlation)."""
import ctypes

import numpy as np
import pytest

from paper_1811_05224_gb300 import capi


@pytest.fixture(scope="module")
def lib():
    try:
        return capi.load()
    except OSError as e:          # library not built here
        pytest.skip(str(e))


def pow2_at_least(n):
    L = 1
    while L < n:
        L *= 2
    return L


@pytest.mark.parametrize("nt", [1, 2, 3, 5, 37, 64, 65, 256, 257, 1000, 1024, 4096])
def test_frequency_block_sizes(lib, nt):
    L = max(2, pow2_at_least(2 * nt))
    for nx in (1, 3, 256):
        nf, nb = ctypes.c_int(), ctypes.c_size_t()
        assert lib.stbem_fft_operator_bytes(nt, nx, ctypes.byref(nf), ctypes.byref(nb)) == capi.STBEM_OK
        assert nf.value == L // 2 + 1
        assert nb.value == nf.value * nx * nx * 16
        for nrhs in (1, 4):
            assert lib.stbem_apply_fft_workspace_bytes(nt, nx, nrhs, ctypes.byref(nb)) == capi.STBEM_OK
            assert nb.value == 2 * nrhs * nf.value * nx * 16
        sb, fb = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.stbem_solve_workspace_bytes(nt, nx, 30, ctypes.byref(sb)) == capi.STBEM_OK
        assert lib.stbem_solve_fft_workspace_bytes(nt, nx, 30, ctypes.byref(fb)) == capi.STBEM_OK
        extra = 2 * nf.value * nx * 16
        assert sb.value + extra <= fb.value <= sb.value + extra + 15


def test_size_limits(lib):
    nb = ctypes.c_size_t()
    for nt, nx in [(0, 4), (4097, 4), (4, 0), (4, 8193), (-1, 4)]:
        assert lib.stbem_fft_operator_bytes(nt, nx, None, ctypes.byref(nb)) == capi.STBEM_ERR_ARG
        assert lib.stbem_apply_fft_workspace_bytes(nt, nx, 1, ctypes.byref(nb)) == capi.STBEM_ERR_ARG
        assert lib.stbem_solve_fft_workspace_bytes(nt, nx, 10, ctypes.byref(nb)) == capi.STBEM_ERR_ARG
    assert lib.stbem_fft_operator_bytes(4096, 8192, None, ctypes.byref(nb)) == capi.STBEM_OK
    assert lib.stbem_fft_operator_bytes(4, 4, None, None) == capi.STBEM_ERR_ARG
    assert lib.stbem_apply_fft_workspace_bytes(4, 4, 0, ctypes.byref(nb)) == capi.STBEM_ERR_ARG


@pytest.mark.parametrize("nt", [1, 2, 7, 32, 33, 100])
def test_zero_padded_circular_convolution_is_the_block_product(nt):
    """y_n = sum_{d<=n} a_d x_{n-d} and z_n = sum_d a_d x_{n+d} (n < n_t) from
    length-L transforms, L = pow2 >= 2 n_t; one step shorter than 2 n_t - 1
    wraps the tail of the convolution onto its head."""
    rng = np.random.default_rng(nt)
    a, x = rng.standard_normal(nt), rng.standard_normal(nt)
    lin = np.convolve(a, x)[:nt]
    cor = np.array([np.dot(a[:nt - n], x[n:]) for n in range(nt)])
    L = max(2, pow2_at_least(2 * nt))
    A, X = np.fft.rfft(a, L), np.fft.rfft(x, L)
    assert np.allclose(np.fft.irfft(A * X, L)[:nt], lin, rtol=0, atol=1e-12 * np.abs(a).sum() * np.abs(x).max())
    assert np.allclose(np.fft.irfft(np.conj(A) * X, L)[:nt], cor, rtol=0,
                       atol=1e-12 * np.abs(a).sum() * np.abs(x).max())
    if nt >= 3:
        Ls = 2 * nt - 2                      # too short: the wrapped tail lands on the first steps
        As, Xs = np.fft.fft(a, Ls), np.fft.fft(x, Ls)
        wrapped = np.real(np.fft.ifft(As * Xs))[:nt]
        full = np.convolve(a, x)
        expect = lin.copy()
        expect[:len(full) - Ls] += full[Ls:]
        assert np.allclose(wrapped, expect, atol=1e-10)
        assert not np.allclose(wrapped, lin, atol=1e-10)
