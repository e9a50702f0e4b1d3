"""Pins for oracle.assembly: entries against brute-force adaptive quadrature,
invariances, the integrated-by-parts D_h form and positive definiteness.

The brute force is written here from the definitions (Section 1 eq. (4),
Section 2 Theorem): QUADPACK (scipy.integrate) over the two space pieces, and
for the time part the closed-form double time integrals evaluated in 40-digit
mpmath (pinned against the nested time integral in test_oracle_timeint.py).  It
shares neither the quadrature rules nor the class switches of the oracle.
"""
import numpy as np
import pytest
from scipy import integrate

import workloads as W
from oracle import assembly
from oracle.geometry import BoundaryMesh

mp = pytest.importorskip("mpmath")


def d2(kind, r2, d, ht, al):
    """Exact double time integral of the V / K(/q) / D-time kernel at lag d.

    For z = alpha r^2 / (4 ht) >= 1e-3 (and the lags d <= 3 used here) the
    closed form in double precision loses at most ~1/z digits, so it is used
    directly; below that the same closed form runs in 25-digit mpmath."""
    if al * r2 / (4.0 * ht) >= 1e-3:
        from scipy.special import exp1, expn
        c = al * r2 / 4.0

        def Fd(s):
            if s <= 0:
                return 0.0
            z = c / s
            if kind == 'V':
                return s / (4 * np.pi) * (exp1(z) - expn(2, z))
            if kind == 'K':
                return al / (8 * np.pi * c) * s * expn(2, z)
            return al / (4 * np.pi) * exp1(z)
        return Fd((d + 1) * ht) - 2 * Fd(d * ht) + Fd((d - 1) * ht)
    mp.mp.dps = 25
    c = mp.mpf(al) * mp.mpf(r2) / 4
    ht = mp.mpf(ht)

    def F(s):
        if s <= 0:
            return mp.mpf(0)
        z = c / s
        if kind == 'V':
            return s / (4 * mp.pi) * (mp.e1(z) - mp.expint(2, z))
        if kind == 'K':
            return mp.mpf(al) / (8 * mp.pi * c) * s * mp.expint(2, z)
        return mp.mpf(al) / (4 * mp.pi) * mp.e1(z)
    return float(F((d + 1) * ht) - 2 * F(d * ht) + F((d - 1) * ht))


OPTS = dict(epsabs=0.0, epsrel=1e-12, limit=200)
DOPTS = dict(epsabs=0.0, epsrel=1e-12)


def piece_integral(kind, m, A0, A1, B0, B1, nb, d, wa=(1.0, 1.0), wb=(1.0, 1.0)):
    """int_a int_b k(x, y) wa(x) wb(y) ds_y ds_x by adaptive quadrature."""
    la = np.linalg.norm(A1 - A0)
    lb = np.linalg.norm(B1 - B0)
    ta, tb = (A1 - A0) / la, (B1 - B0) / lb

    def fa(s):
        return wa[0] + (wa[1] - wa[0]) * s / la

    def fb(g):
        return wb[0] + (wb[1] - wb[0]) * g / lb

    def k(dx):
        r2 = dx @ dx
        v = d2(kind, r2, d, m.ht, m.alpha)
        return v * (dx @ nb) if kind == 'K' else v

    if np.allclose(A0, B0) and np.allclose(A1, B1):
        # identical collinear piece: x - y = (s - g) ta; integrate in u = s - g
        def inner(u):       # polynomial part, exact with 3-point Gauss
            x, w = np.polynomial.legendre.leggauss(3)
            g = 0.5 * (la - u) * (x + 1.0)
            ww = 0.5 * (la - u) * w
            return (ww * (fa(g + u) * fb(g) + fa(g) * fb(g + u))).sum()
        return integrate.quad(lambda u: k(u * ta) * inner(u), 0.0, la, **OPTS)[0]
    if np.allclose(A1, B0) or np.allclose(A0, B1):
        # shared vertex: integrate from the shared point outward on both pieces
        if np.allclose(A1, B0):
            V, da, sa, db, sb = A1, -ta, la, tb, 0.0
        else:
            V, da, sa, db, sb = A0, ta, 0.0, -tb, lb

        def f(g, s):
            x = V + s * da
            y = V + g * db
            pa = s if sa == 0.0 else la - s
            pb = g if sb == 0.0 else lb - g
            return k(x - y) * fa(pa) * fb(pb)
        return integrate.dblquad(f, 0.0, la, 0.0, lb, **DOPTS)[0]

    def f(g, s):
        return k(A0 + s * ta - (B0 + g * tb)) * fa(s) * fb(g)
    return integrate.dblquad(f, 0.0, la, 0.0, lb, **DOPTS)[0]


def bf_V(m, i, j, d):
    return piece_integral('V', m, m.a[i], m.b[i], m.a[j], m.b[j], m.n[j], d)


def bf_K(m, i, p, d):
    N = m.N
    tot = 0.0
    for j, wb in ((p % N, (1.0, 0.0)), ((p - 1) % N, (0.0, 1.0))):
        if j == i:
            continue
        tot += piece_integral('K', m, m.a[i], m.b[i], m.a[j], m.b[j], m.n[j], d, wb=wb)
    return tot


def bf_D(m, l, k, d):
    tot = 0.0
    for pa, a0, a1, sa in m.dual_pieces(l):
        for pb, b0, b1, sb in m.dual_pieces(k):
            A0, A1, B0, B1 = m.hs0[pa], m.hs1[pa], m.hs0[pb], m.hs1[pb]
            tot += sa * sb * piece_integral('V', m, A0, A1, B0, B1, m.hs_n[pb], d)
            tot += (m.hs_n[pa] @ m.hs_n[pb]) * piece_integral(
                '1', m, A0, A1, B0, B1, m.hs_n[pb], d, wa=(a0, a1), wb=(b0, b1))
    return tot


def _meshes():
    pent = np.array([[0.0, 0.0], [1.1, 0.1], [1.3, 0.9], [0.5, 1.4], [-0.2, 0.8]])
    return {
        'square4': BoundaryMesh(W.unit_square(1), 1.0, 4, 1.0),
        'lshape8': BoundaryMesh(W.l_shape(8, seed=3), 0.75, 3, 0.5),
        'pentagon': BoundaryMesh(pent, 0.5, 2, 2.0),
    }


def _check(got, ref, scale, tol=2e-11):
    assert abs(got - ref) <= tol * max(abs(ref), 1e-6 * scale), (got, ref)


@pytest.mark.parametrize("name", ['square4', 'lshape8', 'pentagon'])
def test_V_K_entries_brute_force(name):
    m = _meshes()[name]
    N = m.N
    # one pair per class: identical, adjacent (both orders), near, regular
    pairs = [(0, 0), (0, 1), (N - 1, 0), (2, 0)]
    if N >= 6:
        pairs.append((0, 3))
    for d in range(min(m.n_t, 3)):
        I = np.array([p[0] for p in pairs])
        J = np.array([p[1] for p in pairs])
        V = assembly.V_entries(m, d, I, J)
        K = assembly.K_entries(m, d, I, J)
        sV = np.abs(V).max()
        sK = np.abs(K).max()
        for (i, j), v, kk in zip(pairs, V, K):
            _check(v, bf_V(m, i, j, d), sV)
            _check(kk, bf_K(m, i, j, d), sK)


def test_D_entries_brute_force():
    m = _meshes()['square4']
    cases = [(0, 0, 0), (0, 1, 1), (1, 3, 2)]
    for l, k, d in cases:
        got = assembly.D_entries(m, d, np.array([l]), np.array([k]))[0]
        _check(got, bf_D(m, l, k, d), abs(got))


def test_D_entries_brute_force_lshape():
    m = _meshes()['lshape8']
    for l, k, d in [(2, 3, 0), (1, 5, 1)]:
        got = assembly.D_entries(m, d, np.array([l]), np.array([k]))[0]
        _check(got, bf_D(m, l, k, d), abs(got))


def test_hypersingular_form_matches_normal_derivative_kernel():
    """On separated supports D_h[l,k] equals the integral of psi_l psi_k times
    -(1/alpha) d_{n_x} d_{n_y} U* (Section 2: D = -d_n W), no integration by
    parts needed; this pins the sign and scaling of both terms of the form."""
    m = BoundaryMesh(W.unit_square(4), 1.0, 8, 1.3)
    al, ht = m.alpha, m.ht
    xg, wg = np.polynomial.legendre.leggauss(12)
    xg, wg = 0.5 * (xg + 1.0), 0.5 * wg

    def kern(z, nx, ny, s):
        r2 = z @ z
        e = np.exp(-al * r2 / (4 * s))
        return -al / (8 * np.pi * s * s) * e * (nx @ ny - al * (z @ nx) * (z @ ny) / (2 * s))

    def tint(z, nx, ny, d):     # double time integral (box * box = hat)
        lo = max((d - 1) * ht, 0.0)
        return integrate.quad(lambda s: (ht - abs(s - d * ht)) * kern(z, nx, ny, s),
                              lo, (d + 1) * ht, epsabs=0, epsrel=1e-13, limit=200)[0]

    for l, k, d in [(0, 8, 0), (0, 8, 1), (0, 5, 2), (2, 12, 3), (1, 7, 0)]:
        ref = 0.0
        for pa, a0, a1, _ in m.dual_pieces(l):
            for pb, b0, b1, _ in m.dual_pieces(k):
                A0, A1, B0, B1 = m.hs0[pa], m.hs1[pa], m.hs0[pb], m.hs1[pb]
                la, lb = m.hs_len[pa], m.hs_len[pb]
                for xa, wa in zip(xg, wg):
                    x = A0 + xa * (A1 - A0)
                    for yb, wb in zip(xg, wg):
                        y = B0 + yb * (B1 - B0)
                        ref += wa * wb * la * lb * (a0 + (a1 - a0) * xa) * (b0 + (b1 - b0) * yb) * \
                            tint(x - y, m.hs_n[pa], m.hs_n[pb], d)
        got = assembly.D_entries(m, d, np.array([l]), np.array([k]))[0]
        assert abs(got - ref) <= 1e-10 * abs(ref), (l, k, d, got, ref)


def _rot_mesh(m, th, shift, scale=1.0, tscale=1.0, alpha=None):
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    X = scale * (m.X @ R.T) + shift
    return BoundaryMesh(X, m.T * tscale, m.n_t, m.alpha if alpha is None else alpha)


def test_invariances():
    m = BoundaryMesh(W.l_shape(16, seed=7), 1.0, 6, 0.8)
    ops = {o: assembly.assemble(o, m) for o in 'VKD'}
    # rigid motion
    mr = _rot_mesh(m, 0.37, np.array([2.0, -1.0]))
    for o, A in ops.items():
        B = assembly.assemble(o, mr)
        assert np.abs(A - B).max() <= 1e-12 * np.abs(A).max(), o
    # parabolic scaling x -> c x, t -> c^2 t: V ~ c^4, K ~ c^3, D ~ c^2
    c = 1.7
    ms = _rot_mesh(m, 0.0, 0.0, scale=c, tscale=c * c)
    for o, p in (('V', 4), ('K', 3), ('D', 2)):
        B = assembly.assemble(o, ms)
        assert np.abs(B - c ** p * ops[o]).max() <= 1e-12 * np.abs(B).max(), o
    # heat capacity: A(alpha, T) = alpha A(1, T / alpha)
    m1 = BoundaryMesh(m.X, m.T / m.alpha, m.n_t, 1.0)
    for o, A in ops.items():
        B = assembly.assemble(o, m1)
        assert np.abs(A - m.alpha * B).max() <= 1e-12 * np.abs(A).max(), o


def test_K_vanishes_on_collinear_pairs_and_V_D_symmetric():
    m = BoundaryMesh(W.unit_square(6), 1.0, 5, 1.0)
    K = assembly.assemble('K', m)
    # segments 1..4 lie on the bottom side with vertices 1..5: test i, trial p
    for i in range(1, 5):
        for p in range(2, 5):
            assert np.abs(K[:, i, p]).max() <= 1e-15 * np.abs(K).max()
    for o in 'VD':
        A = assembly.assemble(o, m)
        assert np.array_equal(A, np.transpose(A, (0, 2, 1)))


def test_positive_definite_square32():
    """V_h is positive definite (Section 1); D_h is elliptic (Section 2)."""
    from oracle.solve import dense
    p = W.config('square32')
    m = BoundaryMesh(p.vertices, p.T, p.n_t, p.alpha)
    for o in 'VD':
        M = dense(assembly.assemble(o, m))
        ev = np.linalg.eigvalsh(0.5 * (M + M.T))
        assert ev.min() > 0, (o, ev.min())


def test_mixed_mass_matrix_pins():
    """Consistent mixed mass M[l, k] = <phi0_k, psi_l>: row sums are the lumped
    masses ht (h_{l-1} + 2 h_l + h_{l+1}) / 4 (closed form), column sums are
    ht h_k (the dual hats sum to one on Gamma), and a uniform ring gives
    ht h tridiag(1/8, 3/4, 1/8)."""
    from oracle.assembly import lumped_dual_mass, mixed_mass_matrix
    m = BoundaryMesh(W.l_shape(24, seed=3), 1.0, 4, 0.5)
    M = mixed_mass_matrix(m)
    hm, h0, hp = np.roll(m.h, 1), m.h, np.roll(m.h, -1)
    assert np.allclose(M.sum(1), m.ht * (hm + 2 * h0 + hp) / 4, rtol=1e-14, atol=0)
    assert np.allclose(M.sum(0), m.ht * m.h, rtol=1e-14, atol=0)
    assert np.allclose(M.sum(1), lumped_dual_mass(m), rtol=1e-14, atol=0)
    u = BoundaryMesh(W.unit_square(3), 1.0, 5, 1.0)
    Mu = mixed_mass_matrix(u)
    h = u.h[0]
    ref = u.ht * h * (0.75 * np.eye(12) + 0.125 * (np.roll(np.eye(12), 1, 1) + np.roll(np.eye(12), -1, 1)))
    assert np.allclose(Mu, ref, rtol=1e-14, atol=1e-18)
