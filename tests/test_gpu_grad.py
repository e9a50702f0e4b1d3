"""Differentiation on the GPU: the adjoint (backward-in-time) solve, the
assembly-derivative kernels (stbem_grad) against the oracle's gradient, and
the autograd loss gradient against central differences.

Tolerances.  stbem_grad is compared with the oracle for the same (lambda, w, g)
on the same rule: both sum the same FP64 terms in different orders, so they
agree to rounding of the contraction, 1e-11 of the largest component.  The
end-to-end gradients go through GMRES (tol 1e-13 here): 1e-8 against the
oracle's exact solves.  Central differences with h = 1e-6 carry
O(h^2) + O(eps_L / h) error: 1e-5 relative.
"""
import numpy as np
import pytest

import workloads as W
from oracle import assembly as OA
from oracle import gradient as OG
from oracle import solve as OS
from oracle.geometry import BoundaryMesh
from oracle.rhs import g_vec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def _oracle_contraction(m, ys, lam, w, g):
    CV = OG.correlation(lam, w, m.n_t)
    CK = OG.correlation(lam, g, m.n_t)
    gv, av = OG.dV_contract(m, CV)
    from oracle.assembly import assemble
    K = assemble('K', m)
    gk, ak = OG.dK_contract(m, CK)
    gbar = OG.half_mass_transpose(m, lam) + OS.toeplitz_apply(K, lam, transpose=True)
    gg, ag = OG.g_grad(m, ys, gbar)
    gm = OG.mass_grad(m, lam, g)
    return gk + gg + gm - gv, ak + ag - av


CASES = [
    ("star16", lambda: W.star(8, 2, seed=5), 6, 0.9, (1.5, 1.5)),
    ("lshape24_nt40", lambda: W.l_shape(24, seed=3), 40, 0.5, (1.3, 1.4)),
    ("square12_nt3", lambda: W.unit_square(3), 3, 1.0, (1.5, 1.5)),
    ("triangle_nt1", lambda: np.array([[0.0, 0.0], [1.0, 0.1], [0.3, 0.8]]), 1, 1.3, (1.6, 1.2)),
]


@pytest.mark.parametrize("name,mk,nt,alpha,ys", CASES)
def test_grad_kernel_matches_oracle(ctx, name, mk, nt, alpha, ys):
    """stbem_grad for seeded lambda, w against the oracle's contraction."""
    import paper_1811_05224_gb300 as P
    X = mk()
    m = BoundaryMesh(X, 1.0, nt, alpha)
    rng = np.random.default_rng(17)
    lam = rng.standard_normal((nt, m.N))
    w = rng.standard_normal((nt, m.N))
    g = g_vec(m, ys)
    ref_x, ref_a = _oracle_contraction(m, ys, lam, w, g)
    mesh = P.Mesh(ctx, X, 1.0, nt, alpha)
    K = P.assemble(ctx, mesh, "K")
    dev = lambda a: torch.as_tensor(a).cuda()    # noqa: E731
    dxy, dal = P.grad(ctx, mesh, K, ys, dev(g), dev(w), dev(lam))
    got = dxy.cpu().numpy()
    scale = max(np.abs(ref_x).max(), abs(ref_a))
    assert np.abs(got - ref_x).max() <= 1e-11 * scale, (name, np.abs(got - ref_x).max() / scale)
    assert abs(float(dal) - ref_a) <= 1e-11 * scale, (name, float(dal), ref_a)


def test_adjoint_solve_matches_backward_substitution(ctx):
    import paper_1811_05224_gb300 as P
    X = W.l_shape(24, seed=3)
    nt = 40
    m = BoundaryMesh(X, 1.0, nt, 0.5)
    mesh = P.Mesh(ctx, X, 1.0, nt, 0.5)
    V = P.assemble(ctx, mesh, "V")
    D = P.assemble(ctx, mesh, "D")
    L = P.lumped_mass(ctx, mesh)
    b = np.random.default_rng(2).standard_normal((nt, m.N))
    lam, info = P.solve_adjoint(ctx, V, torch.as_tensor(b).cuda(), D, L, tol=1e-13)
    ref = OG.backward_substitution(OA.assemble("V", m), b)     # the oracle's V
    assert info["status"] == 0
    assert float(np.abs(lam.cpu().numpy() - ref).max() / np.abs(ref).max()) < 1e-10
    # unpreconditioned, too
    lam2, _ = P.solve_adjoint(ctx, V, torch.as_tensor(b).cuda(), tol=1e-13)
    assert float(np.abs(lam2.cpu().numpy() - ref).max() / np.abs(ref).max()) < 1e-10


@pytest.mark.parametrize("products", ["direct", "fft"])
def test_autograd_loss_gradient_matches_oracle(ctx, products):
    """dL/d(vertices, alpha) of L = ||w_h - w_target||^2 through
    neumann_solve's backward against the oracle's adjoint gradient, with the
    GMRES products as block sums and through time FFTs."""
    import paper_1811_05224_gb300 as P
    X = W.star(8, 2, seed=5)
    T, nt, al, ys = 1.0, 6, 0.9, (1.5, 1.5)
    rng = np.random.default_rng(1)
    wt = OG.solve_w(BoundaryMesh(X + 0.01 * rng.standard_normal(X.shape), T, nt, al), ys)[0]
    Lref, gref, aref = OG.loss_grad(X, T, nt, al, ys, wt)
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    at = torch.tensor(al, dtype=torch.float64, requires_grad=True)
    w = P.neumann_solve(ctx, Xt, at, ys, T, nt, tol=1e-13, products=products)
    loss = ((w - torch.as_tensor(wt).cuda()) ** 2).sum()
    loss.backward()
    assert float(loss.detach()) == pytest.approx(Lref, rel=1e-9)
    scale = np.abs(gref).max()
    assert np.abs(Xt.grad.numpy() - gref).max() <= 1e-8 * scale
    assert abs(float(at.grad) - aref) <= 1e-8 * max(abs(aref), scale)


@pytest.mark.parametrize("products", ["direct", "fft"])
def test_star256_gradient_against_central_differences(ctx, products):
    """The differentiation workload: 16-vertex star (seeded radii), N_x = 256,
    N_t = 256, alpha = 1; w_target from seeded perturbed corners; gradient with
    respect to the 32 corner coordinates and alpha against FP64 central
    differences (h = 1e-6) in random directions of (corners, alpha)."""
    import paper_1811_05224_gb300 as P
    C0 = W.star_corners(16, seed=5)
    S = torch.as_tensor(W.subdivision_matrix(16, 16))
    T, nt, ys = 1.0, 256, (1.5, 1.5)
    rng = np.random.default_rng(23)
    Ct = torch.as_tensor(C0 + 0.01 * rng.standard_normal(C0.shape))
    with torch.no_grad():
        wt = P.neumann_solve(ctx, S @ Ct, torch.tensor(1.0, dtype=torch.float64), ys, T, nt, tol=1e-13)

    def loss_of(C, a):
        w = P.neumann_solve(ctx, S @ C, a, ys, T, nt, tol=1e-13, products=products)
        return ((w - wt) ** 2).sum()

    C = torch.tensor(C0, requires_grad=True)
    a = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    L = loss_of(C, a)
    L.backward()
    gC, ga = C.grad.numpy(), float(a.grad)
    h = 1e-6
    with torch.no_grad():
        for _ in range(3):
            v = rng.standard_normal(C0.shape)
            va = float(rng.standard_normal())
            vt = torch.as_tensor(v)
            Lp = float(loss_of(torch.as_tensor(C0) + h * vt, torch.tensor(1.0 + h * va, dtype=torch.float64)))
            Lm = float(loss_of(torch.as_tensor(C0) - h * vt, torch.tensor(1.0 - h * va, dtype=torch.float64)))
            fd = (Lp - Lm) / (2 * h)
            an = float((gC * v).sum() + ga * va)
            assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)
