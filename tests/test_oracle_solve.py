"""Pins for oracle.solve and oracle.rhs: products against the dense block
matrix, forward substitution against a dense solve, GMRES against both,
convergence to the exact Neumann datum, and the iteration-count behaviour of
Section 4 (Table 1) for the operator preconditioner."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import assembly, rhs, solve
from oracle.geometry import BoundaryMesh

HERE = os.path.dirname(os.path.abspath(__file__))


def test_toeplitz_apply_matches_dense():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((5, 4, 3))
    x = rng.standard_normal((5, 3))
    y = solve.toeplitz_apply(A, x)
    assert np.allclose(y.ravel(), solve.dense(A) @ x.ravel(), rtol=0, atol=1e-13)
    xt = rng.standard_normal((5, 4))
    yt = solve.toeplitz_apply(A, xt, transpose=True)
    assert np.allclose(yt.ravel(), solve.dense(A).T @ xt.ravel(), rtol=0, atol=1e-13)


def _problem(nper, nt, alpha=1.0):
    m = BoundaryMesh(W.unit_square(nper), 1.0, nt, alpha)
    V = assembly.assemble('V', m)
    K = assembly.assemble('K', m)
    g = rhs.g_vec(m, [1.5, 1.5])
    return m, V, K, rhs.f_vec(m, K, g)


def test_forward_substitution_and_gmres():
    m, V, K, f = _problem(2, 8)
    w = solve.forward_substitution(V, f)
    wd = np.linalg.solve(solve.dense(V), f.ravel()).reshape(f.shape)
    assert np.abs(w - wd).max() <= 1e-12 * np.abs(wd).max()
    D = assembly.assemble('D', m)
    L = assembly.lumped_dual_mass(m)
    P = lambda v: solve.toeplitz_apply(D, v / L) / L            # noqa: E731
    for M in (None, P):
        wg, it, hist = solve.gmres(lambda v: solve.toeplitz_apply(V, v), f, M, tol=1e-10)
        r = f - solve.toeplitz_apply(V, wg)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(f) * 1.01
        assert np.abs(wg - w).max() <= 1e-7 * np.abs(w).max()


def test_rhs_data_against_quadrature():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 25
    m = BoundaryMesh(W.l_shape(8, seed=3), 1.0, 4, 0.6)
    ys = np.array([1.4, 1.7])
    g = rhs.g_vec(m, ys)
    al = m.alpha
    for n, p in [(0, 0), (1, 3), (3, 5)]:
        r2 = float(((m.X[p] - ys) ** 2).sum())
        U = lambda t: al / (4 * mp.pi * t) * mp.e ** (-al * r2 / (4 * t))   # noqa: E731
        ref = mp.quad(U, [n * m.ht, (n + 1) * m.ht]) / m.ht
        assert abs(g[n, p] - float(ref)) <= 1e-13 * abs(float(ref)) + 1e-300
    # exact Neumann datum: d_n U*(x - y*, t), checked by numerical differentiation
    wq = rhs.w_projection(m, ys, n_gauss=8)
    i, mstep = 2, 3
    xg, wg = np.polynomial.legendre.leggauss(8)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    tot = 0.0
    for s, ws in zip(xg, wg):
        x = m.a[i] + s * (m.b[i] - m.a[i])
        nvec = m.n[i]

        def u(eps, t):
            z0 = mp.mpf(x[0]) + eps * mp.mpf(nvec[0]) - mp.mpf(ys[0])
            z1 = mp.mpf(x[1]) + eps * mp.mpf(nvec[1]) - mp.mpf(ys[1])
            return al / (4 * mp.pi * t) * mp.e ** (-al * (z0 * z0 + z1 * z1) / (4 * t))
        dn = mp.quad(lambda t: mp.diff(lambda e: u(e, t), 0), [mstep * m.ht, (mstep + 1) * m.ht])
        tot += ws * float(dn)
    assert abs(wq[mstep, i] - tot / m.ht) <= 1e-10 * abs(tot / m.ht)


def test_half_mass_partition_of_unity():
    m = BoundaryMesh(W.l_shape(16, seed=3), 1.0, 3, 1.0)
    one = np.ones((3, m.N))
    assert np.allclose(assembly.half_mass_apply(m, one), 0.5 * m.ht * m.h[None, :], rtol=1e-15)
    L = assembly.lumped_dual_mass(m)
    assert abs(L.sum() - m.ht * m.h.sum()) <= 1e-14 * L.sum()


def test_convergence_to_exact_neumann_datum():
    errs = []
    for nper, nt in [(2, 8), (4, 16), (8, 32)]:
        m, V, K, f = _problem(nper, nt)
        w = solve.forward_substitution(V, f)
        errs.append(rhs.l2_rel_error(m, w, rhs.w_projection(m, [1.5, 1.5])))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.06
    assert np.log2(errs[1] / errs[2]) > 1.0


def test_iteration_counts_follow_table1_trend():
    """Section 4: preconditioned counts stay bounded while plain counts grow,
    here on the manufactured workload (u_0 = 0, alpha = 1), where the counts
    are not the paper's: the spread of the preconditioned counts must not
    exceed the paper's spread + 1, and the plain counts must grow by at least
    the paper's factor over the same two refinements.  Table 1's own workload
    is compared count by count in test_oracle_initial.py."""
    tab = np.loadtxt(os.path.join(HERE, 'golden', 'table1_gmres_iterations.txt'))
    paper_spread = tab[:, 3].max() - tab[:, 3].min()
    paper_growth = tab[2, 2] / tab[0, 2]
    plain, prec = [], []
    for nper, nt in [(2, 8), (4, 16), (8, 32)]:
        m, V, K, f = _problem(nper, nt)
        D = assembly.assemble('D', m)
        L = assembly.lumped_dual_mass(m)
        A = lambda v: solve.toeplitz_apply(V, v)                     # noqa: E731
        P = lambda v: solve.toeplitz_apply(D, v / L) / L            # noqa: E731
        plain.append(solve.gmres(A, f, None, tol=1e-8)[1])
        prec.append(solve.gmres(A, f, P, tol=1e-8)[1])
    assert max(prec) - min(prec) <= paper_spread + 1, prec
    assert plain[2] / plain[0] >= paper_growth, plain
    assert all(p < q for p, q in zip(prec[1:], plain[1:]))
