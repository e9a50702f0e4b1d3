"""The block-Toeplitz product through time FFTs (stbem_fft_operator,
stbem_apply_fft, stbem_solve_fft) against the oracle's direct product and
solves.

Bound (normwise per output row, derived from the error of radix-2 FFTs, the
frequency products and the inverse transform): for every right-hand side and
row i,
    ||y_i - (A x)_i||_2 <= c_L * sum_j ||a_ij||_1 ||x_j||_2,
    c_L = (sqrt(n_t) + 3) * eta_L + n_x u,  eta_L = 7 u (log2 L + 2),
with a_ij the lag sequence of entry (i, j), x_j the time sequence of column j
and u = 2^-53."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import assembly as OA
from oracle import solve as OS
from oracle.geometry import BoundaryMesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def fft_len(nt):
    L = 2
    while L < 2 * nt:
        L *= 2
    return L


def c_bound(nt, nx):
    L = fft_len(nt)
    eta = 7 * U * (math.log2(L) + 2)
    return (math.sqrt(nt) + 3) * eta + nx * U


def row_scale(A, x, transpose):
    """sum_j ||a_ij||_1 ||x_j||_2 per output row (A^T: the roles of i, j swap)."""
    a1 = np.abs(A).sum(axis=0)                 # ||a_ij||_1, n1 x n2
    x2 = np.sqrt((x * x).sum(axis=0))          # ||x_j||_2 over time
    return (a1.T @ x2) if transpose else (a1 @ x2)


def check_product(y, ref, A, x, transpose, nt, nx):
    err = np.sqrt(((y - ref) ** 2).sum(axis=0))          # per row, over time
    S = row_scale(A, x, transpose)
    c = c_bound(nt, nx)
    ratio = (err / np.maximum(S, 1e-300)).max()
    assert ratio <= c, (nt, nx, transpose, ratio, c)
    return ratio


@pytest.mark.parametrize("nt,nx,nb", [(1, 7, 1), (5, 3, 2), (37, 45, 3), (48, 33, 2), (130, 132, 2),
                                      (256, 256, 1), (1024, 16, 1), (3000, 4, 1)])
def test_fft_apply_matches_oracle(ctx, nt, nx, nb):
    """Both directions, several right-hand sides, odd n_x (a column pair with
    one member), n_t not a power of two, n_t = 1, and the transform lengths
    of every operator tile shape (L = 2 .. 8192)."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(nt * 1000 + nx)
    # lag blocks decaying in d like the heat kernel's, plus a random sign
    decay = np.exp(-0.05 * np.arange(nt))[:, None, None]
    A = rng.standard_normal((nt, nx, nx)) * decay
    x = rng.standard_normal((nb, nt, nx))
    Ah = P.fft_operator(ctx, torch.as_tensor(A).cuda())
    # the frequency blocks against their definition, sum_d A_d w^{dk}
    L = fft_len(nt)
    assert Ah.data.shape == (L // 2 + 1, nx, nx)
    k = np.arange(L // 2 + 1)
    sel = [0, L // 4, L // 2] if L >= 4 else [0, 1]
    w = np.exp(-2j * np.pi * np.outer(k[sel], np.arange(nt)) / L)
    Ahat_ref = np.einsum("kd,dij->kij", w, A)
    got = Ah.data.cpu().numpy()[sel]
    a2 = np.sqrt((A * A).sum(axis=0))
    assert np.all(np.abs(got - Ahat_ref) <= 7 * U * (math.log2(L) + 2) * math.sqrt(L) * a2 + 1e-300)
    xd = torch.as_tensor(x).cuda()
    for tr in (False, True):
        y = P.apply_fft(ctx, Ah, xd, transpose=tr).cpu().numpy()
        for b in range(nb):
            ref = OS.toeplitz_apply(A, x[b], transpose=tr)
            check_product(y[b], ref, A, x[b], tr, nt, nx)
    # in place: y may be x
    xi = xd[0].clone()
    P.apply_fft(ctx, Ah, xi, out=xi)
    check_product(xi.cpu().numpy(), OS.toeplitz_apply(A, x[0]), A, x[0], False, nt, nx)


def test_fft_operator_from_fp32(ctx):
    """An FP32 operator is widened exactly: its frequency blocks equal those
    of the same values stored in FP64."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(7)
    A32 = torch.as_tensor(rng.standard_normal((40, 24, 24)).astype(np.float32)).cuda()
    h32 = P.fft_operator(ctx, A32)
    h64 = P.fft_operator(ctx, A32.double())
    assert torch.equal(h32.data, h64.data)


def test_fft_apply_full_size_sampled(ctx):
    """n_t = N_x = 1024 (the transform length and operator size of the
    L-shape precision workload): every time step of 6 sampled rows against
    the oracle's direct sums (FP32-generated lag blocks, widened exactly)."""
    import paper_1811_05224_gb300 as P
    nt = nx = 1024
    rng = np.random.default_rng(11)
    A32 = rng.standard_normal((nt, nx, nx), dtype=np.float32)
    A32 *= np.exp(-0.01 * np.arange(nt, dtype=np.float32))[:, None, None]
    x = rng.standard_normal((nt, nx))
    Ad = torch.as_tensor(A32).cuda()
    Ah = P.fft_operator(ctx, Ad)
    del Ad
    torch.cuda.empty_cache()
    xd = torch.as_tensor(x).cuda()
    y = P.apply_fft(ctx, Ah, xd).cpu().numpy()
    yt = P.apply_fft(ctx, Ah, xd, transpose=True).cpu().numpy()
    c = c_bound(nt, nx)
    x2 = np.sqrt((x * x).sum(axis=0))
    for i in rng.choice(nx, 6, replace=False):
        Ai = A32[:, i, :].astype(np.float64)               # a_ij over (d, j)
        ref = np.array([(Ai[:n + 1] * x[n::-1]).sum() for n in range(nt)])
        err = np.sqrt(((y[:, i] - ref) ** 2).sum())
        assert err <= c * (np.abs(Ai).sum(axis=0) @ x2), (i, err)
        # transposed: y_n[j=i] = sum_d sum_r A_d[r][i] x_{n+d}[r]
        Ac = A32[:, :, i].astype(np.float64)               # a_ri over (d, r)
        reft = np.array([(Ac[:nt - n] * x[n:]).sum() for n in range(nt)])
        errt = np.sqrt(((yt[:, i] - reft) ** 2).sum())
        assert errt <= c * (np.abs(Ac).sum(axis=0) @ x2), (i, errt)


def test_solve_fft_matches_oracle(ctx):
    """square32: GMRES with the products through frequency blocks converges
    to the oracle's forward substitution (lumped and consistent mixed mass,
    and an FP32 D_h); the adjoint solve to the oracle's back substitution with
    V_h^T; iteration counts within 1 of the direct-product solve."""
    import paper_1811_05224_gb300 as P
    p = W.config("square32")
    m = P.Mesh(ctx, p.vertices, p.T, p.n_t, p.alpha)
    om = BoundaryMesh(p.vertices, p.T, p.n_t, p.alpha)
    V, K, D = (P.assemble(ctx, m, o) for o in "VKD")
    D32 = P.assemble(ctx, m, "D", "f32")
    L = P.lumped_mass(ctx, m)
    Mi = P.mixed_mass_inverse(ctx, m)
    g, f = P.rhs(ctx, m, K, p.y_star)
    Vo = OA.assemble("V", om)
    fo = f.cpu().numpy()
    w_ref = OS.forward_substitution(Vo, fo)
    Vh, Dh, Dh32 = P.fft_operator(ctx, V), P.fft_operator(ctx, D), P.fft_operator(ctx, D32)
    # the right-hand side with K g through the frequency blocks of K
    Gb, Fb = P.rhs_batched(ctx, m, P.fft_operator(ctx, K), [p.y_star])
    assert torch.equal(Gb[0], g)          # the same datum kernel
    Ko = OA.assemble("K", om)
    gn = g.cpu().numpy()
    Kg_ref = OS.toeplitz_apply(Ko, gn)
    Kg = Fb[0].cpu().numpy() - (f.cpu().numpy() - P.apply(ctx, K, g).cpu().numpy())
    check_product(Kg, Kg_ref, Ko, gn, False, p.n_t, p.n_x)
    for Dx, Lx in ((Dh, L), (Dh, Mi), (Dh32, L), (None, None)):
        w, info = P.solve_fft(ctx, Vh, f, Dx, Lx, tol=1e-10)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-10
        assert np.linalg.norm(w.cpu().numpy() - w_ref) <= 1e-8 * np.linalg.norm(w_ref)
        if Dx is not Dh32:
            _, info_d = P.solve(ctx, V, f, D if Dx is not None else None, Lx, tol=1e-10)
            assert abs(info["iterations"] - info_d["iterations"]) <= 1, (info, info_d)
    # adjoint: V^T lam = b, block upper triangular (back substitution)
    b = torch.as_tensor(np.random.default_rng(2).standard_normal(fo.shape)).cuda()
    lam, info = P.solve_fft(ctx, Vh, b, Dh, L, tol=1e-10, transpose=True)
    assert info["status"] == 0
    Vd = OS.dense(Vo)
    lam_ref = np.linalg.solve(Vd.T, b.cpu().numpy().reshape(-1)).reshape(fo.shape)
    assert np.linalg.norm(lam.cpu().numpy() - lam_ref) <= 1e-8 * np.linalg.norm(lam_ref)


def test_fft_errors(ctx):
    """Sizes beyond the limits, misaligned frequency blocks and a short
    workspace are rejected; the context stays usable afterwards."""
    import ctypes

    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi
    nb = ctypes.c_size_t()
    assert ctx.lib.stbem_fft_operator_bytes(4097, 8, None, ctypes.byref(nb)) == capi.STBEM_ERR_ARG
    assert ctx.lib.stbem_fft_operator_bytes(8, 8193, None, ctypes.byref(nb)) == capi.STBEM_ERR_ARG
    A = torch.randn(6, 5, 5, dtype=torch.float64, device="cuda")
    Ah = P.fft_operator(ctx, A)
    x = torch.randn(6, 5, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.StbemError) as e:
        P.apply_fft(ctx, Ah, x, work=torch.empty(16, dtype=torch.uint8, device="cuda"))
    assert e.value.code == capi.STBEM_ERR_NOMEM
    raw = torch.empty(Ah.data.numel() * 16 + 64, dtype=torch.uint8, device="cuda")
    work = P.api.apply_fft_workspace(ctx, 6, 5)
    code = ctx.lib.stbem_apply_fft(ctx.h, 0, 6, 5, 1, ctypes.c_void_p(raw.data_ptr() + 8),
                                   ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(work.data_ptr()), work.numel())
    assert code == capi.STBEM_ERR_ARG
    code = ctx.lib.stbem_apply_fft(ctx.h, 0, 6, 5, 0, ctypes.c_void_p(Ah.data.data_ptr()),
                                   ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(work.data_ptr()), work.numel())
    assert code == capi.STBEM_ERR_ARG
    y = P.apply_fft(ctx, Ah, x)
    ref = OS.toeplitz_apply(A.cpu().numpy(), x.cpu().numpy())
    check_product(y.cpu().numpy(), ref, A.cpu().numpy(), x.cpu().numpy(), False, 6, 5)


def test_batched_solve_fft_residual_against_oracle(ctx):
    """The batched solve whose refinement finishes on residuals through the
    frequency blocks of V (stbem_solve_batched_fft), with F from the
    frequency blocks of K: the FP64 residual with the oracle's V below 1e-8,
    w within 1e-7 of the oracle's forward substitution, F within 1e-12 of the
    oracle's (1/2 M_h + K_h) g."""
    import paper_1811_05224_gb300 as P
    from oracle import rhs as OR
    X = W.l_shape(48, seed=3)
    nt = 40
    m = P.Mesh(ctx, X, 1.0, nt, 1.0)
    om = BoundaryMesh(X, 1.0, nt, 1.0)
    V, K, D = (P.assemble(ctx, m, o) for o in "VKD")
    L = P.lumped_mass(ctx, m)
    ys = W.annulus_sources(4, seed=4)
    G, F = P.rhs_batched(ctx, m, P.fft_operator(ctx, K), ys)
    Wb, infos = P.solve_batched(ctx, P.bf16_split3(ctx, V), F, P.to_bf16(ctx, D), L, tol=1e-8,
                                V64=P.fft_operator(ctx, V))
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
