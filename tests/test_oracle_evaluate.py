"""Pins of the oracle's evaluation of u in Q (representation formula, eq. (2)).

* u = 1 and u = a + b . x solve alpha u_t - Laplace u = 0 and lie in the
  discrete spaces exactly (u_0 and g nodal, w = d_n u = b . n piecewise
  constant), so u_h equals u up to the rule's quadrature error: at interior
  points, several times, on a jittered square and on the L-shape;
* the single- and double-layer terms of one segment against adaptive
  quadrature in (s, tau) of the unintegrated kernels U* and d_{n_y} U*;
* the Section 4 example: u_h(x, t) converges to exp(-t/alpha) sin(x . d)
  under refinement (levels 2, 3, w_h from the oracle's exact solve).
"""
import numpy as np
from scipy.integrate import dblquad

import workloads as W
from oracle import assembly, rhs, solve
from oracle import evaluate as OE
from oracle import initial as OI
from oracle.geometry import BoundaryMesh


def _exact_cases(bm, dom, pts):
    a, b = 0.3, np.array([0.7, -0.4])
    nt = bm.n_t
    yield "one", np.ones(dom.M), np.ones((nt, bm.N)), np.zeros((nt, bm.N)), np.ones(len(pts))
    yield ("linear", a + dom.nodes @ b, np.tile(a + bm.X @ b, (nt, 1)), np.tile(bm.n @ b, (nt, 1)),
           a + pts @ b)


def test_reproduces_constant_and_linear_solutions():
    rng = np.random.default_rng(3)
    for X, (nodes, tris), nt, al, inside in [
            (W.unit_square(4), W.square_triangulation(4, jitter=0.2, seed=1), 4, 10.0,
             lambda p: np.ones(len(p), bool)),
            (W.unit_square(8), W.square_triangulation(8), 16, 1.0, lambda p: np.ones(len(p), bool)),
            (W.l_shape(16, jitter=(1.0, 1.0)), W.lshape_triangulation(4), 6, 10.0,
             lambda p: ~((p[:, 0] > 0.5 - 0.125) & (p[:, 1] > 0.5 - 0.125)))]:
        bm = BoundaryMesh(X, 1.0, nt, al)
        dom = OI.DomainMesh(nodes, tris, bm)
        h = bm.h.max()
        pts = 0.5 * h + (1 - h) * rng.uniform(size=(40, 2))
        pts = pts[inside(pts)][:6]
        ts = np.array([1.0, 0.5, bm.ht, 0.73, 1.0, 2.5 * bm.ht])[:len(pts)]
        for name, u0, g, w, exact in _exact_cases(bm, dom, pts):
            u = OE.evaluate(bm, dom, pts, ts, w, g, u0)
            assert np.abs(u - exact).max() <= 1e-11, (name, np.abs(u - exact).max())


def test_layer_terms_against_bruteforce():
    """One segment, one time step: the oracle's closed-form time integrals
    with its Gauss rule against scipy's dblquad of U* and d_{n_y} U*."""
    bm = BoundaryMesh(W.unit_square(2), 1.0, 3, 2.0)
    N, ht, al = bm.N, bm.ht, bm.alpha
    x = np.array([0.35, 0.6])
    t = 0.9
    for i, n in [(0, 0), (2, 1), (5, 2)]:
        w = np.zeros((3, N))
        w[n, i] = 1.0
        g = np.zeros((3, N))
        g[n, i] = 1.0                          # hat at vertex i on tau_n
        got_w = OE.boundary_terms(bm, x, t, w, np.zeros((3, N)))
        got_g = OE.boundary_terms(bm, x, t, np.zeros((3, N)), g)
        a, b, h, nrm = bm.a[i], bm.b[i], bm.h[i], bm.n[i]

        def k_single(s, tau):
            y = a + s * (b - a)
            d = x - y
            r2 = d @ d
            sg = t - tau
            return al / (4 * np.pi * sg) * np.exp(-al * r2 / (4 * sg)) * h / al

        def k_double(s, tau):
            y = a + s * (b - a)
            d = x - y
            r2 = d @ d
            sg = t - tau
            return -al ** 2 * (d @ nrm) / (8 * np.pi * sg ** 2) * np.exp(-al * r2 / (4 * sg)) * (1 - s) * h / al

        lo, hi = n * ht, min((n + 1) * ht, t)
        ref_w = dblquad(k_single, lo, hi, 0.0, 1.0, epsabs=0.0, epsrel=1e-12)[0]
        ref_g = dblquad(k_double, lo, hi, 0.0, 1.0, epsabs=0.0, epsrel=1e-12)[0]
        # the hat at vertex i also lives on segment i-1 (its end, weight s)
        ip = (i - 1) % N
        a2, b2, h2, n2 = bm.a[ip], bm.b[ip], bm.h[ip], bm.n[ip]

        def k_double2(s, tau):
            y = a2 + s * (b2 - a2)
            d = x - y
            r2 = d @ d
            sg = t - tau
            return -al ** 2 * (d @ n2) / (8 * np.pi * sg ** 2) * np.exp(-al * r2 / (4 * sg)) * s * h2 / al
        ref_g += dblquad(k_double2, lo, hi, 0.0, 1.0, epsabs=0.0, epsrel=1e-12)[0]
        assert abs(got_w - ref_w) <= 1e-10 * abs(ref_w), (i, n, got_w, ref_w)
        assert abs(got_g - ref_g) <= 1e-10 * abs(ref_g), (i, n, got_g, ref_g)


def test_section4_interior_values_converge():
    th = np.pi / 8
    d = np.array([np.cos(th), np.sin(th)])
    pts = np.array([[0.5, 0.5], [0.3, 0.7], [0.62, 0.25]])
    ts = np.array([1.0, 0.5, 0.75])
    exact = np.exp(-ts / 10.0) * np.sin(pts @ d)
    errs = []
    for L in (2, 3):
        n = 2 ** L
        bm = BoundaryMesh(W.unit_square(n), 1.0, n, 10.0)
        dom = OI.DomainMesh(*W.square_triangulation(n), bm)
        V = assembly.assemble('V', bm)
        K = assembly.assemble('K', bm)
        g = OI.planewave_g(bm)
        u0 = OI.planewave_u0(dom)
        f = rhs.f_vec(bm, K, g) - OI.apply(OI.assemble(bm, dom), u0)
        w = solve.forward_substitution(V, f)
        u = OE.evaluate(bm, dom, pts, ts, w, g, u0)
        errs.append(np.abs(u - exact).max() / np.abs(exact).max())
    assert errs[1] < errs[0] / 2.5 and errs[1] < 5e-3, errs
