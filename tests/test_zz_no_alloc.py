"""stbem_apply_noalloc: the block-Toeplitz product for callers that cannot
allocate device memory (for example inside a host framework that owns all
device buffers through its own pool, or a C caller without an allocator).

Called through the C ABI and checked against stbem_apply (caller workspace)
on two calls in a row with different sizes, precisions and directions, so
that leftovers of the first call in the shared fixed scratch cannot leak into
the second.  The file sorts last so that a run stopping at the first failure
has already run every other test; it also runs alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def lib_ctx():
    from paper_1811_05224_gb300 import capi
    lib = capi.load()
    h = ctypes.c_void_p()
    stream = torch.cuda.current_stream()
    assert lib.stbem_create(ctypes.byref(h), 0, ctypes.c_void_p(stream.cuda_stream)) == capi.STBEM_OK
    yield lib, h, capi
    torch.cuda.synchronize()
    lib.stbem_destroy(h)


def _workspace_apply(lib, h, capi, prec, tr, A, x):
    nt, nx = A.shape[0], A.shape[1]
    nb = x.shape[0]
    sz = ctypes.c_size_t()
    assert lib.stbem_apply_workspace_bytes(nt, nx, nb, prec, ctypes.byref(sz)) == capi.STBEM_OK
    work = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    assert lib.stbem_apply(h, prec, tr, nt, nx, _p(A), nb, _p(x), _p(y), _p(work), sz.value) == capi.STBEM_OK
    return y


def test_noalloc_apply_matches_workspace_apply(lib_ctx):
    lib, h, capi = lib_ctx
    rng = np.random.default_rng(11)
    # two calls in a row: a large FP64 forward product, then a small ragged
    # FP32 transposed product with three right-hand sides
    cases = [(256, 256, 1, capi.F64, 0, 1e-13), (37, 45, 3, capi.F32, 1, 2e-6)]
    for nt, nx, nb, prec, tr, tol in cases:
        dt = torch.float64 if prec == capi.F64 else torch.float32
        A = torch.as_tensor(rng.standard_normal((nt, nx, nx))).to(dt).cuda()
        x = torch.as_tensor(rng.standard_normal((nb, nt, nx))).cuda()
        y = torch.full_like(x, float("nan"))
        code = lib.stbem_apply_noalloc(h, prec, tr, nt, nx, _p(A), nb, _p(x), _p(y))
        assert code == capi.STBEM_OK, lib.stbem_last_error(h)
        y_ref = _workspace_apply(lib, h, capi, prec, tr, A, x)
        mag = _workspace_apply(lib, h, capi, prec, tr, A.abs(), x.abs())
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        assert float((y - y_ref).abs().max()) <= tol * float(mag.max())


def test_noalloc_apply_rejects_oversized_products(lib_ctx):
    lib, h, capi = lib_ctx
    A = torch.zeros(8, dtype=torch.float64, device="cuda")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 1024 steps x 1024 segments x 4 right-hand sides needs far more than the
    # fixed scratch; the call is refused before any launch
    code = lib.stbem_apply_noalloc(h, capi.F64, 0, 1024, 1024, _p(A), 4, _p(x), _p(y))
    assert code == capi.STBEM_ERR_NOMEM
    assert b"fixed scratch" in lib.stbem_last_error(h)
