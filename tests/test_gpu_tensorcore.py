"""Tensor-core (tcgen05, BF16 x BF16 -> FP32) many-right-hand-side
block-Toeplitz product against the oracle's product of the same BF16-rounded
operands.

The library's BF16 conversion rounds to nearest from FP64.  The product then
differs from the exact product of the rounded operands only by the FP32
accumulation: each 64-wide K step is four MMAs, each rounding its FP32
accumulator once (<= 2u, u = 2^-24, truncation allowed) after an internal
16-term sum (<= 2u), so one chain of S K steps errs by at most 16 S u of
|A| |x|."""
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
        steps = nt * ((nx + 63) // 64)          # K steps of the longest chain
        assert np.all(err <= 16 * steps * 2.0 ** -24 * mag + 1e-30), (b, float((err / (mag + 1e-300)).max()))


def test_apply_tc_rejects_bad_sizes(ctx):
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi
    A = torch.zeros((4, 12, 12), dtype=torch.bfloat16, device="cuda")
    x = torch.zeros((1, 4, 12), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(capi.StbemError) as e:
        P.apply_tc(ctx, A, x)
    assert e.value.code == capi.STBEM_ERR_ARG


U = 2.0 ** -24


@pytest.mark.parametrize("chunk", [1, 4, 7])
def test_apply_tc_comp_long_chain(ctx, chunk):
    """Compensated accumulation over a long lag chain (300 lags, ragged
    n_x = 136 so the last K step is partly zero-filled, chunk not dividing the
    chain).  Bound: each K step is four MMAs, each rounding its FP32 partial
    once (<= 2u, truncation allowed) after an internal 16-term sum (<= 2u), so
    a partial of `chunk` K steps errs by <= 16 chunk u of |A||x|, plus 2u for
    the Kahan sum.  The uncompensated product of the same operands must be
    worse by a clear factor (its error grows with the chain)."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(11)
    nt, nx, nb = 300, 136, 2
    # single-layer-like lag blocks: positive, decaying in the lag
    A = torch.as_tensor(rng.random((nt, nx, nx)) / (1.0 + np.arange(nt))[:, None, None]).cuda()
    x = torch.as_tensor(rng.standard_normal((nb, nt, nx)) + 0.3).cuda()
    Ab, xb = P.to_bf16(ctx, A), P.to_bf16(ctx, x)
    y = P.apply_tc(ctx, Ab, xb, chunk=chunk).cpu().numpy()
    y0 = P.apply_tc(ctx, Ab, xb).cpu().numpy()
    A64, x64 = Ab.double().cpu().numpy(), xb.double().cpu().numpy()
    for b in range(nb):
        ref = OS.toeplitz_apply(A64, x64[b])
        mag = OS.toeplitz_apply(np.abs(A64), np.abs(x64[b]))
        err = np.abs(y[b] - ref) / mag
        assert float(err.max()) <= (16 * chunk + 2) * U, float(err.max()) / U
        if chunk <= 4:
            assert float((np.abs(y0[b] - ref) / mag).max()) > 10 * float(err.max())


def test_apply_tc_comp_rejects_bad_chunk(ctx):
    from paper_1811_05224_gb300 import capi
    import paper_1811_05224_gb300 as P
    A = torch.zeros((4, 16, 16), dtype=torch.bfloat16, device="cuda")
    x = torch.zeros((1, 4, 16), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(capi.StbemError) as e:
        P.apply_tc(ctx, A, x, chunk=-1)
    assert e.value.code == capi.STBEM_ERR_ARG


def test_apply_tc3_accuracy(ctx):
    """Three-slice split product of FP64 operands.  The slices leave
    |x - (hi + mid + lo)| <= 2^-27 |x| and the dropped products (s + t >= 3)
    are <= 2^-26 |A||x|; the hi x hi product has partials of 4 K steps
    (<= 66 u, as above) and the other five are 2^-8 smaller or less with
    partials of 16 K steps.  Bound 70 u of |A||x|, far below one BF16
    product (2^-8)."""
    import paper_1811_05224_gb300 as P
    for (nt, nx, nb, seed) in [(40, 48, 2, 5), (260, 72, 2, 6)]:
        rng = np.random.default_rng(seed)
        A = torch.as_tensor(rng.standard_normal((nt, nx, nx))).cuda()
        x = torch.as_tensor(rng.standard_normal((nb, nt, nx))).cuda()
        y = P.apply_tc3(ctx, P.bf16_split3(ctx, A), x).cpu().numpy()
        An, xn = A.cpu().numpy(), x.cpu().numpy()
        for b in range(nb):
            ref = OS.toeplitz_apply(An, xn[b])
            mag = OS.toeplitz_apply(np.abs(An), np.abs(xn[b]))
            err = np.abs(y[b] - ref) / mag
            assert float(err.max()) <= 70 * U, float(err.max()) / U


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
        # the split product is <= 70 u of |K||G| (4e-6); K g cancels by up
        # to ~10 here, so 3e-5 of |f|
        assert float((F[b] - f1).norm() / f1.norm()) < 3e-5
        w1, info = P.solve(ctx, V, f1, D, L, tol=1e-10)
        # FP64 residual of the batched system: the refinement stops at 2e-6
        # measured with the split product, whose own error is <= 70 u of
        # |V||w| (V is positive, so ~|f|): 2e-6 + 4e-6
        r = F[b] - P.apply(ctx, V, Wb[b])
        assert float(r.norm() / F[b].norm()) < 6e-6
        assert float((Wb[b] - w1).norm() / w1.norm()) < 3e-4


def test_batched_solve_fp64_accuracy_against_oracle(ctx):
    """The batched solve with the FP64 residual phase (V64) and F from the FP64
    K product reaches what the FP64 path reaches: per right-hand side, F
    within 1e-12 of the oracle's (1/2 M_h + K_h) g, the FP64 residual with
    the oracle's V below 1e-8, and w within 1e-7 of the oracle's block forward
    substitution (kappa(V_h) ~ 100 times the residual)."""
    import paper_1811_05224_gb300 as P
    import workloads as W
    from oracle import assembly as OA
    from oracle import rhs as OR
    from oracle.geometry import BoundaryMesh
    X = W.l_shape(48, seed=3)
    nt = 40
    m = P.Mesh(ctx, X, 1.0, nt, 1.0)
    om = BoundaryMesh(X, 1.0, nt, 1.0)
    V = P.assemble(ctx, m, "V")
    K = P.assemble(ctx, m, "K")
    D = P.assemble(ctx, m, "D")
    L = P.lumped_mass(ctx, m)
    ys = W.annulus_sources(4, seed=4)
    G, F = P.rhs_batched(ctx, m, K, ys)
    Wb, infos = P.solve_batched(ctx, P.bf16_split3(ctx, V), F, P.to_bf16(ctx, D), L, tol=1e-8, V64=V)
    assert all(i["status"] == 0 and i["rel_residual"] <= 1e-8 for i in infos), infos
    Vo, Ko = OA.assemble("V", om), OA.assemble("K", om)
    for b in range(len(ys)):
        f_ref = OR.f_vec(om, Ko, OR.g_vec(om, ys[b]))
        Fb, Wn = F[b].cpu().numpy(), Wb[b].cpu().numpy()
        assert np.linalg.norm(Fb - f_ref) <= 1e-12 * np.linalg.norm(f_ref)
        r = Fb - OS.toeplitz_apply(Vo, Wn)
        assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(Fb)
        w_ref = OS.forward_substitution(Vo, Fb)
        assert np.linalg.norm(Wn - w_ref) <= 1e-7 * np.linalg.norm(w_ref)
