"""stbem_apply_noalloc: the block-Toeplitz product for callers that cannot
allocate device memory (for example inside a host framework that owns all
device buffers through its own pool, or a C caller without an allocator).

Called through the C ABI on several calls in a row with different sizes,
precisions, directions and kernels (the FP64 tile kernel, the generic FP32
kernel transposed, the register-tiled FP32 forward kernel), so that leftovers
of one call in the shared fixed scratch cannot leak into the next.  Each
result must equal stbem_apply's (caller workspace, same kernels) bit for bit
and meet the per-element bound of the product against the oracle's
toeplitz_apply.  The file sorts last so that a run stopping at the first
failure has already run every other test; it passes run alone
(pytest tests/test_zz_no_alloc.py) as well as after the others.
"""
import ctypes

import numpy as np
import pytest

from oracle import solve as OS

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


# (n_t, n_x, right-hand sides, precision, transpose); the third case has
# N_x % 4 == 0 and enough causal 128 x 128 tiles (18 x 19 / 2 = 171 >= one CTA
# per SM, two waves) for the register-tiled FP32 forward kernel, whose
# partial sums (2.4 MB) still fit the fixed scratch
CASES = [(256, 256, 1, "f64", 0), (37, 45, 3, "f32", 1), (2240, 4, 1, "f32", 0), (70, 64, 2, "f64", 1)]


def test_noalloc_apply_matches_workspace_apply_and_oracle(lib_ctx):
    lib, h, capi = lib_ctx
    rng = np.random.default_rng(11)
    for nt, nx, nb, pname, tr in CASES:
        prec = capi.F64 if pname == "f64" else capi.F32
        dt = torch.float64 if pname == "f64" else torch.float32
        A = torch.as_tensor(rng.standard_normal((nt, nx, nx))).to(dt).cuda()
        x = torch.as_tensor(rng.standard_normal((nb, nt, nx))).cuda()
        y = torch.full_like(x, float("nan"))
        code = lib.stbem_apply_noalloc(h, prec, tr, nt, nx, _p(A), nb, _p(x), _p(y))
        assert code == capi.STBEM_OK, lib.stbem_last_error(h)
        y_ref = _workspace_apply(lib, h, capi, prec, tr, A, x)
        torch.cuda.synchronize()
        assert torch.equal(y, y_ref), (nt, nx, nb, pname, tr)
        # per element against the oracle, with A as stored (FP32 rounded)
        Aeff = A.double().cpu().numpy()
        xh = x.cpu().numpy()
        yh = y.cpu().numpy()
        tol = 1e-13 if pname == "f64" else (nx + 2) * 2.0 ** -24
        for b in range(nb):
            ref = OS.toeplitz_apply(Aeff, xh[b], transpose=bool(tr))
            mag = OS.toeplitz_apply(np.abs(Aeff), np.abs(xh[b]), transpose=bool(tr))
            assert np.all(np.abs(yh[b] - ref) <= tol * mag + 1e-300), (nt, nx, pname, tr, b)


def test_noalloc_apply_allocates_no_device_memory(lib_ctx):
    """After a warm-up call, a synchronised call leaves the device's free
    memory unchanged: the scratch is the library's static array."""
    lib, h, capi = lib_ctx
    rng = np.random.default_rng(12)
    nt, nx = 128, 96
    A = torch.as_tensor(rng.standard_normal((nt, nx, nx))).cuda()
    x = torch.as_tensor(rng.standard_normal((2, nt, nx))).cuda()
    y = torch.empty_like(x)
    assert lib.stbem_apply_noalloc(h, capi.F64, 0, nt, nx, _p(A), 2, _p(x), _p(y)) == capi.STBEM_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.stbem_apply_noalloc(h, capi.F64, 0, nt, nx, _p(A), 2, _p(x), _p(y)) == capi.STBEM_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


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
    # 100000 right-hand sides of one step exceed the grid limit: an argument
    # error, also before any launch
    code = lib.stbem_apply_noalloc(h, capi.F64, 0, 1, 1, _p(A), 100000, _p(x), _p(y))
    assert code == capi.STBEM_ERR_ARG
    assert b"grid limit" in lib.stbem_last_error(h)
