"""Pins for oracle.gradient (shape / alpha derivatives and the adjoint loss
gradient) and for the c-derivatives of oracle.timeint.

The derivative of the discrete map is pinned against central differences of
the oracle's own values, which are pinned elsewhere against brute-force
quadrature and 40-digit closed forms.  A dropped term (a length derivative,
the rotation of the trial normal, the explicit alpha of K, a mass or datum
term), a wrong sign or a transposed contraction fails one of these.
"""
import numpy as np
import pytest

import workloads as W
from oracle import assembly as OA
from oracle import gradient as OG
from oracle import solve as OS
from oracle import timeint
from oracle.geometry import BoundaryMesh
from oracle.rules import DEFAULT_RULES as R

mp = pytest.importorskip("mpmath")

HT, ALPHA = 1.0 / 32.0, 0.7


def _closed(kind, c, d):
    ht, a = mp.mpf(HT), mp.mpf(ALPHA)

    def F(s):
        if s <= 0:
            return mp.mpf(0)
        z = c / s
        if kind == 'V':
            return s / (4 * mp.pi) * (mp.e1(z) - mp.expint(2, z))
        return a / (8 * mp.pi * c) * s * mp.expint(2, z)
    return F((d + 1) * ht) - 2 * F(d * ht) + F((d - 1) * ht)


# (lag, z_d): lag 0; lag 1 on both sides of the series switch (z = 1), tiny z;
# lags >= 2 on both sides of the closed / Peano switch (z_d = d / 2), large lags
CASES = [(0, 1e-9), (0, 0.3), (0, 2.0), (1, 1e-8), (1, 0.05), (1, 0.6), (1, 3.0),
         (2, 0.3), (2, 1.5), (3, 0.2), (6, 2.7), (6, 3.3), (20, 0.4), (20, 12.0),
         (40, 0.01), (40, 25.0), (200, 0.02), (200, 120.0)]


@pytest.mark.parametrize("kind", ['V', 'K'])
def test_c_derivative_against_40_digit_closed_form(kind):
    fn = timeint.dlag_V if kind == 'V' else timeint.dlag_Kq
    mp.mp.dps = 40
    try:
        for d, zd in CASES:
            c = zd * max(d, 1) * HT
            ref = float(mp.diff(lambda cc: _closed(kind, cc, d), mp.mpf(c)))
            got = fn(np.array([c]), d, HT, ALPHA, R)[0]
            assert abs(got - ref) <= 5e-13 * abs(ref), (kind, d, zd, got, ref)
    finally:
        mp.mp.dps = 15


def _mesh(X, alpha=0.9):
    return BoundaryMesh(X, 1.0, 6, alpha)


# pairs on a 16-node star: identical, adjacent both ways (incl. the ring wrap),
# near, regular, a collinear adjacent pair (K entry exactly 0, gradient not)
PAIRS = [(0, 0), (0, 1), (1, 0), (0, 15), (3, 5), (2, 9), (4, 4), (7, 8)]


@pytest.mark.parametrize("op", ['V', 'K'])
@pytest.mark.parametrize("d", [0, 1, 2, 5])
def test_entry_gradient_against_central_differences(op, d):
    X = W.star(8, 2, seed=5)
    m = _mesh(X)
    N, h = m.N, 1e-6
    for i, j in PAIRS:
        if op == 'V':
            gx, ga = OG.V_entry_grad(m, d, i, j)
            f = lambda M: OA.V_entries(M, d, np.array([i]), np.array([j]))[0]   # noqa: E731
        else:
            gx, ga = OG.K_entry_grad(m, d, i, j)
            f = lambda M: OA.K_entries(M, d, np.array([i]), np.array([j]))[0]   # noqa: E731
        fd = np.zeros_like(gx)
        for k in range(N):
            for c in range(2):
                Xp, Xm = X.copy(), X.copy()
                Xp[k, c] += h
                Xm[k, c] -= h
                fd[k, c] = (f(_mesh(Xp)) - f(_mesh(Xm))) / (2 * h)
        fa = (f(_mesh(X, 0.9 + h)) - f(_mesh(X, 0.9 - h))) / (2 * h)
        scale = np.abs(fd).max()
        assert np.abs(gx - fd).max() <= 1e-8 * scale, (op, d, i, j)
        assert abs(ga - fa) <= 1e-7 * abs(fa) + 1e-9 * scale, (op, d, i, j, ga, fa)


def test_backward_substitution_solves_the_transpose():
    m = _mesh(W.star(8, 1, seed=5))
    V = OA.assemble('V', m)
    b = np.random.default_rng(3).standard_normal((m.n_t, m.N))
    lam = OG.backward_substitution(V, b)
    ref = np.linalg.solve(OS.dense(V).T, b.ravel()).reshape(b.shape)
    assert np.abs(lam - ref).max() <= 1e-10 * np.abs(ref).max()
    # and the transposed Toeplitz product reproduces b
    assert np.abs(OS.toeplitz_apply(V, lam, transpose=True) - b).max() <= 1e-10 * np.abs(b).max()


def test_loss_gradient_against_central_differences():
    """dL/dtheta for L = ||w_h - w_target||^2 (w_target from perturbed
    vertices) in random directions of (vertices, alpha)."""
    X = W.star(8, 2, seed=5)
    T, nt, al, ys = 1.0, 6, 0.9, (1.5, 1.5)
    rng = np.random.default_rng(1)
    wt = OG.solve_w(BoundaryMesh(X + 0.01 * rng.standard_normal(X.shape), T, nt, al), ys)[0]
    L, gx, ga = OG.loss_grad(X, T, nt, al, ys, wt)
    assert L == pytest.approx(OG.loss(X, T, nt, al, ys, wt), rel=1e-14)
    h = 1e-6
    for _ in range(3):
        v, va = rng.standard_normal(X.shape), rng.standard_normal()
        fd = (OG.loss(X + h * v, T, nt, al + h * va, ys, wt)
              - OG.loss(X - h * v, T, nt, al - h * va, ys, wt)) / (2 * h)
        an = float((gx * v).sum() + ga * va)
        assert abs(fd - an) <= 1e-7 * abs(an), (fd, an)
