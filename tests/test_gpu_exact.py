"""Exact-slice tensor-core product (FP64-grade accuracy from BF16 MMAs)
against the oracle's FP64 block-Toeplitz product, and the batched solve that
finishes its refinement on it.

Error bound of the product (derived from the slicing, not measured): with
row scales 2^eA[d][i] > max_j |A[d][i][j]| and 2^eX[b][n] > max_j |x[b][n][j]|,
every term A x loses at most the two truncated tails (2^-(6S+1) each, relative
to 2^(eA + eX)) and the dropped slice pairs s + t >= S (at most
S 2^-(6S+2) (1 + 2^-6 + ...)), so
  |y - A x| <= 2^-6S (1 + 0.26 S) n_x sum_d 2^(eA[d][i] + eX[b][m-d])
             <= 2^-6S (1 + 0.26 S) 4 n_x sum_d max|A[d][i]| max|x[b][m-d]|,
plus rounding far below it (the double-float sum, 2^-48 of the output's
scale).  The oracle's own FP64 sum adds up to n u |A| |x| (n terms)."""
import numpy as np
import pytest

from oracle import solve as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def _ref(A, x):
    """oracle products: y, |A| |x|, and the row-maximum bound sum"""
    nt, nx = A.shape[0], A.shape[1]
    B = x.shape[0]
    y = np.stack([OS.toeplitz_apply(A, x[b]) for b in range(B)])
    mag = np.stack([OS.toeplitz_apply(np.abs(A), np.abs(x[b])) for b in range(B)])
    ra = np.abs(A).max(axis=2)            # (nt, nx): max_j |A[d][i][j]|
    rx = np.abs(x).max(axis=2)            # (B, nt)
    M = np.zeros((B, nt, nx))
    for d in range(nt):
        M[:, d:, :] += rx[:, :nt - d, None] * ra[d][None, None, :]
    return y, mag, M * nx


def _bound(S, M, mag, nt, nx):
    return 2.0 ** (-6 * S) * (1 + 0.26 * S) * 4 * M + 2 * nt * nx * U64 * mag + 1e-300


def test_slices_reconstruct_rows(ctx):
    """The slices are integers with |q_0| <= 64 and |q_s| <= 32 after, the
    scale is the smallest power of two above the row maximum, and the S
    slices reconstruct each row to within half a unit of the last one."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, 9, 40)) * np.exp(rng.uniform(-30, 30, (3, 9, 1)))
    X[1, 4] = 0.0
    X[2, 2, 7] = 2.0 ** 10                  # an exact power of two as the maximum
    Xd = torch.as_tensor(X).cuda()
    for S in (4, 7, 8):
        E = P.exact_slices(ctx, Xd, S)
        q = E.slices.double().cpu().numpy()
        e = E.row_exp.cpu().numpy().astype(np.int64)
        assert q.shape == (S,) + X.shape and e.shape == X.shape[:2]
        assert np.all(q == np.rint(q))
        assert np.abs(q[0]).max() <= 64 and np.abs(q[1:]).max() <= 32
        mx = np.abs(X).max(axis=2)
        nz = mx > 0
        assert np.all(e[~nz] == -16384)
        assert np.all(mx[nz] < np.ldexp(1.0, e[nz])) and np.all(mx[nz] >= np.ldexp(0.5, e[nz]))
        w = 2.0 ** (-6 * (np.arange(S) + 1))
        rec = np.ldexp(np.tensordot(w, q, axes=1), np.where(nz, e, 0)[..., None])
        err = np.abs(rec - X)
        assert np.all(err <= np.ldexp(1.0, np.where(nz, e, 0) - 6 * S - 1)[..., None]), S


@pytest.mark.parametrize("nt,nx,B,S", [(37, 64, 2, 7), (130, 200, 3, 7), (5, 1096, 1, 6), (1, 8, 1, 4),
                                       (20, 64, 2, 8), (129, 136, 1, 5)])
def test_apply_exact_matches_oracle(ctx, nt, nx, B, S):
    """Random lag blocks and right-hand sides: several row and step tiles with
    ragged tails, n_x > 1024 (two column groups), one step; the bound above."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(nt * 7919 + nx * 31 + S)
    A = rng.standard_normal((nt, nx, nx))
    x = rng.standard_normal((B, nt, nx))
    Ad, xd = torch.as_tensor(A).cuda(), torch.as_tensor(x).cuda()
    Ax = P.exact_slices(ctx, Ad, S)
    y = P.apply_exact(ctx, Ax, xd).cpu().numpy()
    # pre-sliced x: one launch over whole tiles (the FP64-x call may split the
    # lags of few tiles into chunks, summed afterwards); both within the bound
    y2 = P.apply_exact(ctx, Ax, P.exact_slices(ctx, xd, S)).cpu().numpy()
    ref, mag, M = _ref(A, x)
    err = np.abs(y - ref)
    assert np.all(err <= _bound(S, M, mag, nt, nx)), float((err / M).max())
    assert np.all(np.abs(y2 - ref) <= _bound(S, M, mag, nt, nx))
    # and elementwise against |A| |x| (4 2^-6S in a CPU emulation of the scheme)
    assert np.all(err <= 16 * 2.0 ** (-6 * S) * mag + 2 * nt * nx * U64 * mag + 1e-300), \
        float((err / (mag + 1e-300)).max())


def test_apply_exact_integer_data_is_exact(ctx):
    """Integer lag blocks and right-hand sides below 64 in magnitude slice
    into one nonzero slice each; the product of integers is then exact (and
    the oracle's FP64 sums of integers below 2^53 are exact too)."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(11)
    nt, nx, B = 70, 96, 2
    A = rng.integers(-63, 64, (nt, nx, nx)).astype(np.float64)
    x = rng.integers(-63, 64, (B, nt, nx)).astype(np.float64)
    x[1, 3] = 0.0
    Ax = P.exact_slices(ctx, torch.as_tensor(A).cuda(), 4)
    y = P.apply_exact(ctx, Ax, torch.as_tensor(x).cuda()).cpu().numpy()
    ref = np.stack([OS.toeplitz_apply(A, x[b]) for b in range(B)])
    assert np.array_equal(y, ref)


def test_apply_exact_wide_dynamic_range(ctx):
    """Lag blocks decaying by 2^-40 per lag, right-hand-side steps from 1e-80
    to 1 and a zero step, each row without internal range: each output keeps
    its accuracy relative to its own |A| |x| (per-row scales, and a
    per-output reference scale that follows the largest step so far)."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(13)
    nt, nx, B = 9, 48, 2
    A = rng.standard_normal((nt, nx, nx)) * np.ldexp(1.0, -40 * np.arange(nt))[:, None, None]
    x = rng.standard_normal((B, nt, nx)) * np.array([1e-80, 1e-40, 1e-10, 1, 3, 1e-5, 1, 0.5, 2])[None, :, None]
    x[1, 2] = 0.0
    Ax = P.exact_slices(ctx, torch.as_tensor(A).cuda(), 7)
    y = P.apply_exact(ctx, Ax, torch.as_tensor(x).cuda()).cpu().numpy()
    ref, mag, M = _ref(A, x)
    err = np.abs(y - ref)
    assert np.all(err <= _bound(7, M, mag, nt, nx))
    assert np.all(err <= 16 * 2.0 ** -42 * mag + 2 * nt * nx * U64 * mag + 1e-300), \
        float((err / (mag + 1e-300)).max())
    assert np.all(np.abs(y[:, 0]) > 0)           # the 1e-80 step is not flushed


def test_apply_exact_rows_with_internal_range(ctx):
    """Rows whose entries span hundreds of decades (like the early steps of
    a density whose source is far away: e^(-r^2 / 4t) along the boundary) and
    local lag blocks: the error stays within the row-scale bound, and
    normwise within 32 2^-42 (about 4 2^-42 in a CPU emulation); small
    entries of such rows are not resolved relative to themselves (the
    documented limit of per-row scales)."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(19)
    nt, nx, B = 12, 64, 2
    j = np.arange(nx)
    A = rng.standard_normal((nt, nx, nx)) * np.exp(-0.5 * (j[:, None] - j[None, :]) ** 2)[None]
    t = (np.arange(nt) + 1.0) / nt
    x = rng.standard_normal((B, nt, nx)) * np.exp(-(j[None, None, :] / 8.0) ** 2 / (4 * t[None, :, None]))
    Ax = P.exact_slices(ctx, torch.as_tensor(A).cuda(), 7)
    y = P.apply_exact(ctx, Ax, torch.as_tensor(x).cuda()).cpu().numpy()
    ref, mag, M = _ref(A, x)
    err = np.abs(y - ref)
    assert np.all(err <= _bound(7, M, mag, nt, nx))
    for b in range(B):
        assert np.linalg.norm(y[b] - ref[b]) <= 32 * 2.0 ** -42 * np.linalg.norm(ref[b])


def test_apply_exact_error_falls_with_slices(ctx):
    """Each added slice pair level gains about 2^6 in accuracy."""
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(17)
    nt, nx = 24, 64
    A = rng.standard_normal((nt, nx, nx))
    x = rng.standard_normal((1, nt, nx))
    ref, mag, _ = _ref(A, x)
    errs = []
    for S in (4, 5, 6):
        Ax = P.exact_slices(ctx, torch.as_tensor(A).cuda(), S)
        y = P.apply_exact(ctx, Ax, torch.as_tensor(x).cuda()).cpu().numpy()
        errs.append(float((np.abs(y - ref) / mag).max()))
    assert errs[0] > 16 * errs[1] > 256 * errs[2] > 0, errs


def test_apply_exact_rejects_bad_arguments(ctx):
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi
    A = torch.zeros((4, 12, 12), dtype=torch.float64, device="cuda")
    x = torch.zeros((1, 4, 12), dtype=torch.float64, device="cuda")
    Ax = P.exact_slices(ctx, A, 7)
    with pytest.raises(capi.StbemError) as e:
        P.apply_exact(ctx, Ax, x)                 # n_x % 8 != 0
    assert e.value.code == capi.STBEM_ERR_ARG
    with pytest.raises(capi.StbemError) as e:
        P.exact_slices(ctx, torch.zeros((2, 16), dtype=torch.float64, device="cuda"), 9)
    assert e.value.code == capi.STBEM_ERR_ARG
    A = torch.zeros((4, 16, 16), dtype=torch.float64, device="cuda")
    Ax = P.exact_slices(ctx, A, 7)
    xs = P.exact_slices(ctx, torch.zeros((1, 4, 16), dtype=torch.float64, device="cuda"), 6)
    with pytest.raises(capi.StbemError) as e:
        P.apply_exact(ctx, Ax, xs)                # different slice counts
    assert e.value.code == capi.STBEM_ERR_ARG


def test_batched_solve_exact_residual_against_oracle(ctx):
    """The batched solve whose refinement finishes on the exact-slice
    residual: the same bars as with the FP64 residual (FP64 residual with the
    oracle's V below 1e-8, w within 1e-7 of the oracle's forward
    substitution), and F from the exact-slice K product within 1e-11 of the
    oracle's (1/2 M_h + K_h) g."""
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
    G, F = P.rhs_batched(ctx, m, P.exact_slices(ctx, K, 7), ys)
    Wb, infos = P.solve_batched(ctx, P.bf16_split3(ctx, V), F, P.to_bf16(ctx, D), L, tol=1e-8,
                                V64=P.exact_slices(ctx, V, 7))
    assert all(i["status"] == 0 and i["rel_residual"] <= 1e-8 for i in infos), infos
    Vo, Ko = OA.assemble("V", om), OA.assemble("K", om)
    for b in range(len(ys)):
        f_ref = OR.f_vec(om, Ko, OR.g_vec(om, ys[b]))
        Fb, Wn = F[b].cpu().numpy(), Wb[b].cpu().numpy()
        assert np.linalg.norm(Fb - f_ref) <= 1e-11 * np.linalg.norm(f_ref)
        r = Fb - OS.toeplitz_apply(Vo, Wn)
        assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(Fb)
        w_ref = OS.forward_substitution(Vo, Fb)
        assert np.linalg.norm(Wn - w_ref) <= 1e-7 * np.linalg.norm(w_ref)


def test_mixed_solve_exact_residual_against_oracle(ctx):
    """The mixed solve whose outer residuals are exact-slice products
    (stbem_solve_mixed_exact; no FP64 V product): the FP64 residual with the
    oracle's V below 1e-8 and w within 1e-6 of the oracle's block forward
    substitution, as for the FP64-residual mixed solve."""
    import paper_1811_05224_gb300 as P
    import workloads as W
    from oracle import assembly as OA
    from oracle.geometry import BoundaryMesh
    p = W.config("square32")
    m = P.Mesh(ctx, p.vertices, p.T, p.n_t, p.alpha)
    om = BoundaryMesh(p.vertices, p.T, p.n_t, p.alpha)
    V = P.assemble(ctx, m, "V")
    K = P.assemble(ctx, m, "K")
    D32 = P.assemble(ctx, m, "D", "f32")
    V32 = P.round_f32(ctx, V)
    L = P.lumped_mass(ctx, m)
    g, f = P.rhs(ctx, m, K, p.y_star)
    wm, info = P.solve_mixed(ctx, P.exact_slices(ctx, V, 7), V32, f, D32, L, tol=1e-8, inner_tol=1e-4)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-8, info
    Vo = OA.assemble("V", om)
    fo = f.cpu().numpy()
    r = fo - OS.toeplitz_apply(Vo, wm.cpu().numpy())
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(fo)
    w_ref = OS.forward_substitution(Vo, fo)
    assert np.linalg.norm(wm.cpu().numpy() - w_ref) <= 1e-6 * np.linalg.norm(w_ref)


def test_mixed_solve_tensor_core_inner_against_oracle(ctx):
    """The mixed solve with the inner GMRES on the tensor cores (three-slice
    BF16 V and D, stbem_solve_mixed_tc) and exact-slice outer residuals: the
    FP64 residual with the oracle's V below 1e-8 and w within 1e-6 of the
    oracle's block forward substitution; lumped and consistent mass."""
    import paper_1811_05224_gb300 as P
    import workloads as W
    from oracle import assembly as OA
    from oracle.geometry import BoundaryMesh
    X, T, nt, al = W.l_shape(48, seed=3), 1.0, 24, 0.5
    m = P.Mesh(ctx, X, T, nt, al)
    om = BoundaryMesh(X, T, nt, al)
    V = P.assemble(ctx, m, "V")
    K = P.assemble(ctx, m, "K")
    D = P.assemble(ctx, m, "D")
    g, f = P.rhs(ctx, m, K, (1.5, 1.5))
    V3, D3, Vx = P.bf16_split3(ctx, V), P.bf16_split3(ctx, D), P.exact_slices(ctx, V, 7)
    Vo = OA.assemble("V", om)
    fo = f.cpu().numpy()
    w_ref = OS.forward_substitution(Vo, fo)
    for Lm in (P.lumped_mass(ctx, m), P.mixed_mass_inverse(ctx, m)):
        wm, info = P.solve_mixed(ctx, Vx, V3, f, D3, Lm, tol=1e-8, inner_tol=1e-4)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-8, info
        r = fo - OS.toeplitz_apply(Vo, wm.cpu().numpy())
        assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(fo)
        assert np.linalg.norm(wm.cpu().numpy() - w_ref) <= 1e-6 * np.linalg.norm(w_ref)
