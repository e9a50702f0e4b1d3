"""Tensor-core (tcgen05, BF16 x BF16 -> FP32) many-right-hand-side
block-Toeplitz product against the oracle's product of the same BF16-rounded
operands.

The BF16 rounding of the library's conversion kernel must equal torch's
round-to-nearest-even.  The product then differs from the exact product of the
rounded operands only by FP32 accumulation: at most (number of FP32
additions) x 2^-24 of |A| |x|, below 1e-4 of it for these sizes."""
import numpy as np
import pytest

from oracle import solve as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


@pytest.mark.parametrize("nt,nx,nb", [(37, 64, 2), (200, 72, 3), (130, 256, 1), (1, 8, 1), (129, 136, 2)])
def test_apply_tc_matches_oracle(ctx, nt, nx, nb):
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(nt * 1000 + nx)
    A = torch.as_tensor(rng.standard_normal((nt, nx, nx))).cuda()
    x = torch.as_tensor(rng.standard_normal((nb, nt, nx))).cuda()
    Ab = P.to_bf16(ctx, A)
    xb = P.to_bf16(ctx, x)
    # direct round-to-nearest from FP64: never farther than torch's conversion
    # (which rounds through FP32 and can miss on near-ties) and within half a
    # BF16 ulp (2^-8 relative)
    for src, r in ((A, Ab), (x, xb)):
        err = (r.double() - src).abs()
        assert bool((err <= (src.to(torch.bfloat16).double() - src).abs()).all())
        assert bool((err <= 2.0 ** -8 * src.abs()).all())
    y = P.apply_tc(ctx, Ab, xb).cpu().numpy()
    A64 = Ab.double().cpu().numpy()
    x64 = xb.double().cpu().numpy()
    for b in range(nb):
        ref = OS.toeplitz_apply(A64, x64[b])
        mag = OS.toeplitz_apply(np.abs(A64), np.abs(x64[b]))
        err = np.abs(y[b] - ref)
        assert np.all(err <= 1e-4 * mag + 1e-30), (b, float((err / (mag + 1e-300)).max()))


def test_apply_tc_rejects_bad_sizes(ctx):
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi
    A = torch.zeros((4, 12, 12), dtype=torch.bfloat16, device="cuda")
    x = torch.zeros((1, 4, 12), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(capi.StbemError) as e:
        P.apply_tc(ctx, A, x)
    assert e.value.code == capi.STBEM_ERR_ARG


def test_apply_tc3_accuracy(ctx):
    """Three-slice split product: ~1e-6 of |A||x| (FP32 accumulation), far
    below a single BF16 product."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(5)
    nt, nx, nb = 40, 48, 2
    A = torch.as_tensor(rng.standard_normal((nt, nx, nx))).cuda()
    x = torch.as_tensor(rng.standard_normal((nb, nt, nx))).cuda()
    y = P.apply_tc3(ctx, P.bf16_split3(ctx, A), x).cpu().numpy()
    An, xn = A.cpu().numpy(), x.cpu().numpy()
    for b in range(nb):
        ref = OS.toeplitz_apply(An, xn[b])
        mag = OS.toeplitz_apply(np.abs(An), np.abs(xn[b]))
        assert np.all(np.abs(y[b] - ref) <= 2e-5 * mag)
        assert float(np.abs(y[b] - ref).max() / mag.max()) < 2e-6


def test_batched_solve_matches_fp64_solves(ctx):
    """Batched tensor-core solve of several right-hand sides against the FP64
    single-right-hand-side solves (L-shape, seeded sources)."""
    import paper_1811_05224_gb300 as P
    import workloads as W
    X = W.l_shape(48, seed=3)
    nt = 40
    m = P.Mesh(ctx, X, 1.0, nt, 1.0)
    V = P.assemble(ctx, m, "V")
    K = P.assemble(ctx, m, "K")
    D = P.assemble(ctx, m, "D")
    L = P.lumped_mass(ctx, m)
    ys = W.annulus_sources(4, seed=4)
    G, F = P.rhs_batched(ctx, m, P.bf16_split3(ctx, K), ys)
    Wb, infos = P.solve_batched(ctx, P.bf16_split3(ctx, V), F, P.to_bf16(ctx, D), L, tol=2e-6)
    assert all(i["status"] == 0 for i in infos), infos
    for b in range(len(ys)):
        g1, f1 = P.rhs(ctx, m, K, ys[b])
        # the split product is ~1e-6 of |K||G|; K g cancels, so ~1e-5 of |f|
        assert float((F[b] - f1).norm() / f1.norm()) < 3e-5
        w1, info = P.solve(ctx, V, f1, D, L, tol=1e-10)
        r = F[b] - P.apply(ctx, V, Wb[b])           # FP64 residual of the batched system
        assert float(r.norm() / F[b].norm()) < 5e-6
        assert float((Wb[b] - w1).norm() / w1.norm()) < 3e-4
