"""Failure paths of the solvers and the tensor-core product, made on the host
(an iteration cap, a singular operator) or by a wait that nothing completes
(the tensor-core kernel's diagnostic stall): each returns its status code and
leaves the context usable for the next call."""
import numpy as np
import pytest

import workloads as W
from oracle import solve as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def _square(ctx):
    import paper_1811_05224_gb300 as P
    p = W.config("square32")
    m = P.Mesh(ctx, p.vertices, p.T, p.n_t, p.alpha)
    V, K, D = (P.assemble(ctx, m, o) for o in "VKD")
    L = P.lumped_mass(ctx, m)
    g, f = P.rhs(ctx, m, K, p.y_star)
    return V, D, L, f


def test_iteration_cap_returns_noconv(ctx):
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi
    V, D, L, f = _square(ctx)
    w, info = P.solve(ctx, V, f, D, L, tol=1e-12, max_iter=1, raise_on_fail=False)
    assert info["status"] == capi.STBEM_ERR_NOCONV and info["iterations"] == 1
    with pytest.raises(capi.StbemError) as e:
        P.solve(ctx, V, f, D, L, tol=1e-12, max_iter=1)
    assert e.value.code == capi.STBEM_ERR_NOCONV
    with pytest.raises(capi.StbemError) as e:
        P.solve_adjoint(ctx, V, f, D, L, tol=1e-12, max_iter=1)
    assert e.value.code == capi.STBEM_ERR_NOCONV
    # the context still solves
    w, info = P.solve(ctx, V, f, D, L, tol=1e-8)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-8


def test_singular_operator_returns_breakdown(ctx):
    """V = 0: the first Krylov column is zero, a zero Givens pivot."""
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi
    V, D, L, f = _square(ctx)
    Z = torch.zeros_like(V)
    for kw in ({}, {"D": D, "L": L}):
        w, info = P.solve(ctx, Z, f, tol=1e-8, raise_on_fail=False, **kw)
        assert info["status"] == capi.STBEM_ERR_BREAKDOWN, info
    with pytest.raises(capi.StbemError) as e:
        P.solve_mixed(ctx, V, Z.float(), f, D.float(), L, tol=1e-8)
    assert e.value.code == capi.STBEM_ERR_BREAKDOWN
    w, info = P.solve(ctx, V, f, D, L, tol=1e-8)
    assert info["status"] == 0


def test_tensor_core_wait_timeout_returns_timeout(ctx):
    """The diagnostic stall makes the kernel's MMA issuer wait on a barrier
    nothing arrives on, with pipeline waits of 2^20 cycles: the call returns
    STBEM_ERR_TIMEOUT; with the stall off the next product is correct, so the
    kernel released its tensor memory and the context is intact."""
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi
    lib = capi.load()
    rng = np.random.default_rng(5)
    nt, nx = 24, 64
    A = torch.as_tensor(rng.standard_normal((nt, nx, nx))).cuda()
    x = torch.as_tensor(rng.standard_normal((2, nt, nx))).cuda()
    Ab, xb = P.to_bf16(ctx, A), P.to_bf16(ctx, x)
    assert lib.stbem_debug_tc_stall(1, 100) == capi.STBEM_ERR_ARG
    assert lib.stbem_debug_tc_stall(1, 1 << 20) == capi.STBEM_OK
    try:
        with pytest.raises(capi.StbemError) as e:
            P.apply_tc(ctx, Ab, xb)
        assert e.value.code == capi.STBEM_ERR_TIMEOUT
    finally:
        assert lib.stbem_debug_tc_stall(0, 0) == capi.STBEM_OK
    torch.cuda.synchronize()
    for _ in range(2):
        y = P.apply_tc(ctx, Ab, xb).cpu().numpy()
        Ae, xe = Ab.double().cpu().numpy(), xb.double().cpu().numpy()
        for b in range(2):
            ref = OS.toeplitz_apply(Ae, xe[b])
            mag = OS.toeplitz_apply(np.abs(Ae), np.abs(xe[b]))
            # FP32 accumulation over nt * nx / 64 K steps of 4 MMAs
            assert np.all(np.abs(y[b] - ref) <= 4 * 4 * (nt * nx // 64) * 2.0 ** -24 * mag + 1e-300)
