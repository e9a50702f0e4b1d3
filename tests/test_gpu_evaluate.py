"""Evaluation of u in Q (representation formula, eq. (2)) on the GPU.

* stbem_evaluate against the oracle for seeded data (w, g, u0 standard
  normal) at interior points and times on, between and at the first time
  steps: both sides evaluate the same rule in FP64 in different orders, so
  they agree to 1e-12 of the sum of the terms' magnitudes, bounded here by
  1e-11 (the data are O(1) and the terms sum to O(1) values);
* exact reproduction of u = 1 and u = a + b . x (as the oracle's pin);
* the Section 4 example end to end (GPU assembly, right-hand side with
  M_h^0 u_0, GMRES, evaluation) at levels 2..6: u_h converges to
  exp(-t/alpha) sin(x . d) at interior points, and equals the oracle's
  evaluation of its exact solve at levels 2, 3 to the GMRES tolerance.
"""
import numpy as np
import pytest

import workloads as W
from oracle import evaluate as OE
from oracle import initial as OI
from oracle.geometry import BoundaryMesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def _points(rng, h, k, inside=None):
    pts = 0.5 * h + (1 - h) * rng.uniform(size=(8 * k, 2))
    if inside is not None:
        pts = pts[inside(pts)]
    return pts[:k]


def test_evaluate_matches_oracle(ctx):
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(7)
    in_l = lambda p: ~((p[:, 0] > 0.375) & (p[:, 1] > 0.375))      # noqa: E731
    for X, (nodes, tris), nt, al, inside in [
            (W.unit_square(4), W.square_triangulation(4, jitter=0.25, seed=2), 5, 3.0, None),
            (W.l_shape(16, jitter=(1.0, 1.0)), W.lshape_triangulation(4), 6, 10.0, in_l)]:
        bm = BoundaryMesh(X, 1.0, nt, al)
        od = OI.DomainMesh(nodes, tris, bm)
        mesh = P.Mesh(ctx, X, 1.0, nt, al)
        dom = P.Domain(ctx, mesh, nodes, tris)
        pts = _points(rng, bm.h.max(), 7, inside)
        ts = np.array([1.0, bm.ht, 2.5 * bm.ht, 0.5, 0.999, 3 * bm.ht, 0.77])[:len(pts)]
        w = rng.standard_normal((nt, bm.N))
        g = rng.standard_normal((nt, bm.N))
        u0 = rng.standard_normal(od.M)
        ref = OE.evaluate(bm, od, pts, ts, w, g, u0)
        dev = lambda a: torch.as_tensor(a).cuda()                   # noqa: E731
        got = P.evaluate(ctx, mesh, pts, ts, dev(w), dev(g), dom, dev(u0)).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), np.abs(got - ref).max()
        # without the initial datum
        ref0 = OE.evaluate(bm, None, pts, ts, w, g, None)
        got0 = P.evaluate(ctx, mesh, pts, ts, dev(w), dev(g)).cpu().numpy()
        assert np.abs(got0 - ref0).max() <= 1e-11 * max(1.0, np.abs(ref0).max())


def test_evaluate_reproduces_constant_and_linear(ctx):
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(9)
    X = W.l_shape(16, jitter=(1.0, 1.0))
    nodes, tris = W.lshape_triangulation(4)
    nt = 6
    bm = BoundaryMesh(X, 1.0, nt, 10.0)
    od = OI.DomainMesh(nodes, tris, bm)
    mesh = P.Mesh(ctx, X, 1.0, nt, 10.0)
    dom = P.Domain(ctx, mesh, nodes, tris)
    pts = _points(rng, bm.h.max(), 6, lambda p: ~((p[:, 0] > 0.375) & (p[:, 1] > 0.375)))
    ts = np.array([1.0, 0.5, bm.ht, 0.73, 1.0, 2.5 * bm.ht])[:len(pts)]
    a, b = 0.3, np.array([0.7, -0.4])
    dev = lambda v: torch.as_tensor(np.ascontiguousarray(v)).cuda()     # noqa: E731
    for u0, g, w, exact in [(np.ones(od.M), np.ones((nt, bm.N)), np.zeros((nt, bm.N)), np.ones(len(pts))),
                            (a + od.nodes @ b, np.tile(a + bm.X @ b, (nt, 1)), np.tile(bm.n @ b, (nt, 1)),
                             a + pts @ b)]:
        got = P.evaluate(ctx, mesh, pts, ts, dev(w), dev(g), dom, dev(u0)).cpu().numpy()
        assert np.abs(got - exact).max() <= 1e-11


def test_evaluate_rejects_bad_arguments(ctx):
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi
    mesh = P.Mesh(ctx, W.unit_square(2), 1.0, 2, 1.0)
    z = torch.zeros(16, dtype=torch.float64, device="cuda")
    code = ctx.lib.stbem_evaluate(ctx.h, mesh.h, None, 1, z.data_ptr(), z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                  z.data_ptr(), z.data_ptr())
    assert code == capi.STBEM_ERR_ARG                    # u0 without a domain
    other = P.Mesh(ctx, W.unit_square(2), 1.0, 2, 1.0)
    dom = P.Domain(ctx, other, *W.square_triangulation(2))
    code = ctx.lib.stbem_evaluate(ctx.h, mesh.h, dom.h, 1, z.data_ptr(), z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                  z.data_ptr(), z.data_ptr())
    assert code == capi.STBEM_ERR_ARG                    # domain of another mesh


def test_section4_solution_in_Q(ctx):
    import paper_1811_05224_gb300 as P
    th = np.pi / 8
    d = np.array([np.cos(th), np.sin(th)])
    pts = np.array([[0.5, 0.5], [0.3, 0.7], [0.62, 0.25], [0.8, 0.8]])
    ts = np.array([1.0, 0.5, 0.75, 1.0])
    exact = np.exp(-ts / 10.0) * np.sin(pts @ d)
    errs = []
    for L in range(2, 7):
        n = 2 ** L
        X = W.unit_square(n)
        nodes, tris = W.square_triangulation(n)
        mesh = P.Mesh(ctx, X, 1.0, n, 10.0)
        dom = P.Domain(ctx, mesh, nodes, tris)
        V = P.assemble(ctx, mesh, "V")
        K = P.assemble(ctx, mesh, "K")
        D = P.assemble(ctx, mesh, "D")
        g, u0 = P.planewave_data(ctx, dom)
        f = P.rhs_initial(ctx, dom, K, g, u0)
        w, info = P.solve(ctx, V, f, D, P.lumped_mass(ctx, mesh), tol=1e-10)
        u = P.evaluate(ctx, mesh, pts, ts, w, g, dom, u0).cpu().numpy()
        errs.append(np.abs(u - exact).max() / np.abs(exact).max())
        if L <= 3:
            from oracle import assembly as OA, rhs as OR, solve as OS
            bm = BoundaryMesh(X, 1.0, n, 10.0)
            od = OI.DomainMesh(nodes, tris, bm)
            go, uo = OI.planewave_g(bm), OI.planewave_u0(od)
            fo = OR.f_vec(bm, OA.assemble('K', bm), go) - OI.apply(OI.assemble(bm, od), uo)
            wo = OS.forward_substitution(OA.assemble('V', bm), fo)
            uref = OE.evaluate(bm, od, pts, ts, wo, go, uo)
            assert np.abs(u - uref).max() <= 1e-8 * np.abs(uref).max(), (L, np.abs(u - uref).max())
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1]), errs
    assert errs[-1] < 2e-4, errs
