"""Pins of the oracle for non-uniform time grids (oracle.nonuniform).

* every branch of the time integral over two unequal steps (d = 0; d = 1
  with z < 1 and z >= 1; d >= 2 closed and Peano, with a plateau piece)
  against nested adaptive quadrature (mpmath) of the kernel G(t - tau);
* on a uniform grid every block equals the Toeplitz lag block of
  oracle.assembly (V, K, D);
* V and D blocks are symmetric, and on a graded grid the blocks are not
  Toeplitz;
* the manufactured solution u = U*(x - y*, t) converges on graded grids
  t_j = T (j / N_t)^{3/2}.
"""
import numpy as np
import pytest

import workloads as W
from oracle import assembly
from oracle import nonuniform as NU
from oracle.geometry import BoundaryMesh

mp = pytest.importorskip("mpmath")

ALPHA = 0.7
T_NODES = np.array([0.0, 0.02, 0.05, 0.07, 0.11, 0.16, 0.19, 0.26, 0.30])


def _G(kind, c):
    a = mp.mpf(ALPHA)

    def G(s):
        if s <= 0:
            return mp.mpf(0)
        e = mp.e ** (-c / s)
        if kind == 'V':
            return e / (4 * mp.pi * s)
        if kind == 'K':
            return a * e / (8 * mp.pi * s * s)
        return a / (4 * mp.pi) * e * (c / s ** 3 - 1 / s ** 2)
    return G


def nested(kind, c, m, n):
    mp.mp.dps = 20
    c = mp.mpf(c)
    G = _G(kind, c)
    tm0, tm1 = mp.mpf(T_NODES[m]), mp.mpf(T_NODES[m + 1])
    tn0, tn1 = mp.mpf(T_NODES[n]), mp.mpf(T_NODES[n + 1])

    def inner(tt):
        hi = min(tn1, tt)
        if hi <= tn0:
            return mp.mpf(0)
        pts = [tn0] + sorted(x for x in (tt - c, tt - c / 3, tt - 3 * c) if tn0 < x < hi) + [hi]
        return mp.quad(lambda tau: G(tt - tau), pts)
    outer = [tm0] + sorted(x for x in (tn0 + c / 10, tn0 + c, tn1, tn1 + c) if tm0 < x < tm1) + [tm1]
    return mp.quad(inner, outer)


# (m, n, c), one per branch: d = 0; d = 1 small z (unequal steps 0.02, 0.03)
# and large z; d = 2 Peano and closed; d = 4 Peano with a plateau (steps
# 0.07, 0.02); d = 6 closed
CASES = [(3, 3, 1e-4), (2, 1, 1e-4), (4, 3, 0.08), (4, 2, 2e-3), (4, 2, 0.3), (6, 2, 3e-3),
         (7, 1, 0.9)]


@pytest.mark.parametrize("kind", ["V", "K", "1"])
def test_time_integrals_against_nested_quadrature(kind, cpu_pool):
    refs = [cpu_pool.submit(nested, kind, c, m, n) for m, n, c in CASES]
    for (m, n, c), fut in zip(CASES, refs):
        got = float(NU.time_integral(kind, np.array([c]), T_NODES, m, n, ALPHA)[0])
        ref = float(fut.result())
        assert abs(got - ref) <= 1e-10 * abs(ref) + 1e-300, (kind, m, n, c, got, ref)


def test_geometric_grid_ratio_four():
    """Steps growing by a factor of 4 (the largest ratio the rule is stated
    for): d >= 2 blocks, Peano and closed, against nested quadrature."""
    global T_NODES
    saved = T_NODES
    h0 = 0.01
    T_NODES = np.array([0.0, h0, 5 * h0, 21 * h0, 85 * h0])
    try:
        for m, n, c in ((2, 0, 4e-5), (3, 1, 1e-5), (3, 0, 0.03)):
            for kind in ("V", "1"):
                got = float(NU.time_integral(kind, np.array([c]), T_NODES, m, n, ALPHA)[0])
                ref = float(nested(kind, c, m, n))
                assert abs(got - ref) <= 1e-12 * abs(ref), (kind, m, n, c, got, ref)
    finally:
        T_NODES = saved


def test_uniform_grid_equals_toeplitz_blocks():
    m = BoundaryMesh(W.l_shape(8, seed=3), 1.0, 6, 0.8)
    t = np.arange(7) * m.ht
    for op in "VKD":
        A = assembly.assemble(op, m)
        B = NU.assemble(op, m, t)
        for mm in range(6):
            for nn in range(6):
                if nn > mm:
                    assert not B[mm, nn].any()
                    continue
                d = mm - nn
                assert np.abs(B[mm, nn] - A[d]).max() <= 1e-13 * np.abs(A[d]).max(), (op, mm, nn)


def test_graded_blocks_symmetric_and_not_toeplitz():
    m = BoundaryMesh(W.unit_square(2), 1.0, 5, 1.0)
    t = (np.arange(6) / 5.0) ** 1.5
    V = NU.assemble('V', m, t)
    D = NU.assemble('D', m, t)
    for A in (V, D):
        for mm in range(5):
            for nn in range(mm + 1):
                assert np.array_equal(A[mm, nn], A[mm, nn].T)
    assert np.abs(V[2, 1] - V[3, 2]).max() > 1e-3 * np.abs(V[2, 1]).max()
    # the diagonal blocks grow with the step (h^{3/2}-like scaling of V's lag 0)
    assert V[4, 4, 0, 0] > V[1, 1, 0, 0]


def test_manufactured_solution_converges_on_graded_grids():
    ys = (1.5, 1.5)
    errs = []
    for nper, nt in [(1, 4), (2, 8), (4, 16)]:
        m = BoundaryMesh(W.unit_square(nper), 1.0, nt, 1.0)
        t = (np.arange(nt + 1) / nt) ** 1.5
        V = NU.assemble('V', m, t)
        K = NU.assemble('K', m, t)
        g = NU.g_vec(m, t, ys)
        f = NU.f_vec(m, t, K, g)
        w = NU.forward_substitution(V, f)
        errs.append(NU.l2_rel_error(m, t, w, NU.w_projection(m, t, ys)))
    assert errs[0] > errs[1] > errs[2], errs
    assert np.log2(errs[1] / errs[2]) > 1.0, errs
