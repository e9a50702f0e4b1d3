"""Initial-data operator M_h^0 and the Section 4 example data (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 1, eq. (4): the initial datum u_0 is discretised in S_h^1(Omega_h), the
continuous piecewise linear functions phi_j^1 on a triangulation Omega_h of
the domain, and

    M_h^0[(m,i), j] = < M_0 phi_j^1, phi^0_(m,i) >_{L2(Sigma)}
                    = int_{tau_m} int_{gamma_i} int_Omega U*(x - y, t) phi_j^1(y) dy ds_x dt

with M_0 the initial potential of the representation formula, eq. (2)
(U* = alpha / (4 pi t) exp(-alpha |x - y|^2 / (4 t)), no 1/alpha factor in
front of M_0).  The right-hand side of eq. (4) is (1/2 M_h + K_h) g - M_h^0 u_0.
On a uniform time grid every entry depends on m itself (the initial time is
fixed), so M_h^0 is stored dense as M0[m][i][j], m = 0..N_t-1.

Time.  int_{tau_m} U*(r, t) dt = G(r, t_{m+1}) - G(r, t_m) exactly, with
G(r, s) = alpha / (4 pi) E1(alpha r^2 / (4 s)) and G(r, 0) = 0
(dG/ds = alpha e^{-z} / (4 pi s) = U*, z = alpha r^2 / (4 s)).

Space: per pair (segment gamma_i, triangle omega).  The paper prints no rule;
this one is fixed by ``M0Rules`` and is the rule the CUDA path implements.
Pair classes:
  T  omega has an endpoint of gamma_i as a vertex (touching);
  N  not T and dist(gamma_i, omega) < near_ratio * max(h_i, diam omega);
  R  otherwise.
Rules:
  * tensor rule of order n: n Gauss-Legendre points on gamma_i times the
    collapsed (conical product) rule on omega, y = v0 + u ((1-v)(v1-v0) +
    v (v2-v0)), dy = 2|omega| u du dv, u and v n-point Gauss-Legendre on
    [0,1]; barycentrics lambda = (1-u, u(1-v), uv);
  * m = 0: order 8 (R) or 12 (N);
  * m >= 1 (every class): the kernel G(., t_{m+1}) - G(., t_m) is an
    entire function of r^2 whose only length scale is the diffusion length
    sqrt(4 t_m / alpha), so the order follows rho^2 = 4 m ht / (alpha s^2),
    s = max(h_i, diam omega): rho^2 >= 1e4, 144, 5, 1.44, else -> order 3,
    4, 6, 8, 12 (thresholds measured for 1e-11 relative per pair).  rho^2 is
    a quotient of products (no sums), so every implementation switches at the
    same m;
  * T at m = 0 (G(., t_1) has a log r singularity where omega touches
    gamma_i): polar rule.  gamma_i is split at its midpoint; a half that ends
    at a shared vertex gets n_outer Gauss points graded toward that vertex
    (distance rho = (h_i/2) v^3), the other half plain Gauss.  For every
    outer point x, omega is the signed sum of the three triangles (x, v_a,
    v_{a+1}) (sign of the doubled area A2; |A2| <= 1e-12 L^2 skipped).  Each
    is swept by rays y = x + s (e(t) - x), s in [0,1], e(t) the edge point at
    arc position t from the foot of the perpendicular from x (distance p),
    dy = s p ds dt.  The far edge is parametrised by the sinh transformation
    t = p sinh(mu) (Johnston and Elliott, Int. J. Numer. Meth. Eng. 62, 2005),
    so |e - x| = p cosh(mu) and the log near-singularity of thin
    sub-triangles (x close to a vertex) becomes smooth in mu: n_angular Gauss
    points in mu, s = w^3 graded toward x with n_radial Gauss points in w.
    lambda is extended linearly outside omega.

Pins (tests/test_oracle_initial.py): on Omega = (0,1)^2 the sums
sum_j M0[m][i][j] p(y_j) for p in {1, y_1, y_2} equal the integrals of
int_Omega U*(x - y, t) p(y) dy, which are products of erf and exp in closed
form, integrated over gamma_i x tau_m by adaptive quadrature; single entries
of every class against adaptive quadrature of the triple integral; the Section
4 example: w_h converges to the exact Neumann datum.
"""
from dataclasses import dataclass

import numpy as np

from .geometry import BoundaryMesh
from .quadrature import gauss01
from .special import e1

T_CLS, N_CLS, R_CLS = 2, 1, 0


@dataclass(frozen=True)
class M0Rules:
    # m = 0: tensor order per class (touching pairs: polar rule)
    order0_R: int = 8
    order0_N: int = 12
    # m >= 1, every class: order by rho^2 = 4 m ht / (alpha s^2),
    # s = max(h_i, diam omega) (the diffusion length sqrt(4 t_m / alpha) over
    # the pair's size): the first (rho^2 threshold, order) step with
    # rho^2 >= threshold.  Thresholds measured for 1e-11 relative per pair.
    steps: tuple = ((1e4, 3), (144.0, 4), (5.0, 6), (1.44, 8), (0.0, 12))
    near_ratio: float = 1.0
    n_outer: int = 8        # polar rule: Gauss points per half of gamma_i
    n_radial: int = 12
    n_angular: int = 12
    grading: int = 3        # rho = v^grading
    degenerate: float = 1e-12   # |A2| <= degenerate L^2: sub-triangle skipped

    def order(self, cls: int, m: int, rho2: float) -> int:
        """Tensor order of a pair of class cls at step m (T at m = 0 uses the
        polar rule instead)."""
        if m == 0:
            return self.order0_R if cls == R_CLS else self.order0_N
        for thr, o in self.steps:
            if rho2 >= thr:
                return o
        raise AssertionError("unreachable")


DEFAULT_M0_RULES = M0Rules()


class DomainMesh:
    """Triangulation Omega_h of the domain, conforming with Gamma_h.

    ``nodes`` (M, 2), ``tris`` (K, 3) indices, counter-clockwise.  Every
    boundary vertex x_p of ``bmesh`` must coincide with a node (within
    1e-12 of the domain's diameter); that node is moved onto x_p exactly, and
    ``bnode[p]`` is its index.
    """

    def __init__(self, nodes, tris, bmesh: BoundaryMesh):
        Y = np.array(nodes, dtype=np.float64)
        tr = np.asarray(tris, dtype=np.int64)
        if Y.ndim != 2 or Y.shape[1] != 2 or tr.ndim != 2 or tr.shape[1] != 3:
            raise ValueError("need nodes (M, 2) and triangles (K, 3)")
        if tr.min() < 0 or tr.max() >= Y.shape[0]:
            raise ValueError("triangle index out of range")
        diam = float(np.ptp(Y, axis=0).max())
        bnode = np.empty(bmesh.N, dtype=np.int64)
        for p in range(bmesh.N):
            d = np.sqrt(((Y - bmesh.X[p]) ** 2).sum(1))
            k = int(np.argmin(d))
            if d[k] > 1e-12 * diam:
                raise ValueError("boundary vertex %d is not a node of the triangulation" % p)
            bnode[p] = k
        Y[bnode] = bmesh.X
        v0, v1, v2 = Y[tr[:, 0]], Y[tr[:, 1]], Y[tr[:, 2]]
        a2 = (v1[:, 0] - v0[:, 0]) * (v2[:, 1] - v0[:, 1]) - (v1[:, 1] - v0[:, 1]) * (v2[:, 0] - v0[:, 0])
        if np.any(a2 <= 0):
            raise ValueError("triangles must be counter-clockwise with positive area")
        self.nodes, self.tris, self.bnode = Y, tr, bnode
        self.M, self.K = Y.shape[0], tr.shape[0]
        self.area = 0.5 * a2
        e = [np.sqrt(((Y[tr[:, a]] - Y[tr[:, (a + 1) % 3]]) ** 2).sum(1)) for a in range(3)]
        self.diam = np.maximum.reduce(e)


def _pt_seg(p, s0, s1):
    e = s1 - s0
    L2 = (e * e).sum(-1)
    tt = np.clip(((p - s0) * e).sum(-1) / L2, 0.0, 1.0)
    q = s0 + tt[..., None] * e
    return np.sqrt(((p - q) ** 2).sum(-1))


def classify(bmesh: BoundaryMesh, dom: DomainMesh, rules=DEFAULT_M0_RULES):
    """Class of every (segment i, triangle k) pair, shape (N_x, K)."""
    N = bmesh.N
    ia = dom.bnode
    ib = dom.bnode[(np.arange(N) + 1) % N]
    tr = dom.tris
    touch = np.zeros((N, dom.K), dtype=bool)
    for c in range(3):
        touch |= (tr[None, :, c] == ia[:, None]) | (tr[None, :, c] == ib[:, None])
    Y = dom.nodes
    a = bmesh.a[:, None, :]
    b = bmesh.b[:, None, :]
    gaps = []
    for c in range(3):
        v = Y[tr[:, c]][None, :, :]
        w = Y[tr[:, (c + 1) % 3]][None, :, :]
        gaps += [_pt_seg(v, a, b), _pt_seg(a, v, w), _pt_seg(b, v, w)]
    gap = np.minimum.reduce(gaps)
    lmax = np.maximum(bmesh.h[:, None], dom.diam[None, :])
    cls = np.full((N, dom.K), R_CLS, dtype=np.int64)
    cls[gap < rules.near_ratio * lmax] = N_CLS
    cls[touch] = T_CLS
    return cls


def G(r2, s, alpha):
    """G(r, s) = alpha/(4 pi) E1(alpha r^2 / (4 s)) for s > 0, 0 for s = 0."""
    if s <= 0.0:
        return np.zeros_like(r2)
    return alpha / (4.0 * np.pi) * e1(alpha * r2 / (4.0 * s))


def tensor_points(bmesh, dom, I, Kt, n):
    """Tensor rule of order n for pairs (I[p], Kt[p]): squared distances
    (P, Q) and weights times barycentrics (P, Q, 3)."""
    g, gw = gauss01(n)
    a, b = bmesh.a[I], bmesh.b[I]                         # (P, 2)
    h = bmesh.h[I]
    x = a[:, None, :] + g[None, :, None] * (b - a)[:, None, :]     # (P, n, 2)
    wx = h[:, None] * gw[None, :]                                   # (P, n)
    U = np.repeat(g, n)
    Vv = np.tile(g, n)
    wuv = np.repeat(gw, n) * np.tile(gw, n) * U
    lam = np.stack([1.0 - U, U * (1.0 - Vv), U * Vv], axis=1)      # (n^2, 3)
    tr = dom.tris[Kt]
    v0, v1, v2 = dom.nodes[tr[:, 0]], dom.nodes[tr[:, 1]], dom.nodes[tr[:, 2]]
    y = (v0[:, None, :] + U[None, :, None] * ((1.0 - Vv)[None, :, None] * (v1 - v0)[:, None, :]
                                               + Vv[None, :, None] * (v2 - v0)[:, None, :]))  # (P, n^2, 2)
    wy = 2.0 * dom.area[Kt][:, None] * wuv[None, :]                 # (P, n^2)
    d = x[:, :, None, :] - y[:, None, :, :]                         # (P, n, n^2, 2)
    r2 = (d * d).sum(-1).reshape(len(I), -1)
    w = (wx[:, :, None] * wy[:, None, :]).reshape(len(I), -1)
    return r2, w[:, :, None] * np.tile(lam, (n, 1))[None, :, :]


def polar_points(bmesh, dom, i, k, rules=DEFAULT_M0_RULES):
    """Polar rule for a touching pair (i, k): r^2 (Q,) and weight x
    barycentrics (Q, 3)."""
    N = bmesh.N
    tri = dom.tris[k]
    V = dom.nodes[tri]                              # (3, 2)
    pa, pb = bmesh.a[i], bmesh.b[i]
    h = bmesh.h[i]
    shared = [dom.bnode[i] in tri, dom.bnode[(i + 1) % N] in tri]
    g, gw = gauss01(rules.n_outer)
    q = rules.grading
    xs, wxs = [], []
    # half at the start vertex: x = pa + rho (pb - pa)/h, rho in (0, h/2)
    for end, p_end, p_other in ((0, pa, pb), (1, pb, pa)):
        if shared[end]:
            rho = 0.5 * h * g ** q
            wr = 0.5 * h * q * g ** (q - 1) * gw
        else:
            rho = 0.5 * h * g
            wr = 0.5 * h * gw
        xs.append(p_end[None, :] + (rho / h)[:, None] * (p_other - p_end)[None, :])
        wxs.append(wr)
    x = np.concatenate(xs)                          # (n_o', 2)
    wx = np.concatenate(wxs)
    # barycentrics of x (linear extension): lambda_c(x)
    def bary(p):
        d0 = p - V[0]
        e1v, e2v = V[1] - V[0], V[2] - V[0]
        det = e1v[0] * e2v[1] - e1v[1] * e2v[0]
        u1 = (d0[..., 0] * e2v[1] - d0[..., 1] * e2v[0]) / det
        u2 = (e1v[0] * d0[..., 1] - e1v[1] * d0[..., 0]) / det
        return np.stack([1.0 - u1 - u2, u1, u2], axis=-1)
    lx = bary(x)                                    # (n_o', 3)
    ws, wsw = gauss01(rules.n_radial)
    s = ws ** q
    sw = q * ws ** (q - 1) * wsw
    mu01, muw = gauss01(rules.n_angular)
    r2s, wls = [], []
    for a in range(3):
        bb = (a + 1) % 3
        e = V[bb] - V[a]
        L = np.sqrt(e @ e)
        u = e / L
        A2 = (V[a, 0] - x[:, 0]) * (V[bb, 1] - x[:, 1]) - (V[a, 1] - x[:, 1]) * (V[bb, 0] - x[:, 0])
        keep = np.abs(A2) > rules.degenerate * L * L
        xs_, A2_, lx_, wx_ = x[keep], A2[keep], lx[keep], wx[keep]
        p = np.abs(A2_) / L                          # distance from x to the edge's line
        t0 = (xs_ - V[a]) @ u                        # arc position of the foot from v_a
        m0 = np.arcsinh(-t0 / p)
        m1 = np.arcsinh((L - t0) / p)
        mu = m0[:, None] + (m1 - m0)[:, None] * mu01[None, :]          # (P', n_a)
        wmu = (m1 - m0)[:, None] * muw[None, :]
        rho = p[:, None] * np.cosh(mu)                                   # |edge point - x|
        sig = (t0[:, None] + p[:, None] * np.sinh(mu)) / L              # edge parameter
        r2 = (s[None, None, :] * rho[:, :, None]) ** 2                  # (P', n_a, n_r)
        w = (np.sign(A2_)[:, None, None] * wx_[:, None, None] * wmu[:, :, None]
             * (p[:, None] * rho)[:, :, None] * (sw * s)[None, None, :])
        le = np.zeros(sig.shape + (3,))
        le[..., a] = 1.0 - sig
        le[..., bb] = sig
        lam = lx_[:, None, None, :] + s[None, None, :, None] * (le - lx_[:, None, :])[:, :, None, :]
        r2s.append(r2.ravel())
        wls.append((w[..., None] * lam).reshape(-1, 3))
    return np.concatenate(r2s), np.concatenate(wls)


def rho2(bmesh, dom, I, Kt, m):
    """rho^2 = 4 m ht / (alpha s^2), s = max(h_i, diam_k), for pairs (I, Kt)."""
    s = np.maximum(bmesh.h[I], dom.diam[Kt])
    return 4.0 * m * bmesh.ht / (bmesh.alpha * s * s)


def assemble(bmesh: BoundaryMesh, dom: DomainMesh, rules=DEFAULT_M0_RULES, magnitude=False, chunk=4096):
    """M0[m][i][j], shape (N_t, N_x, M).  With ``magnitude`` also returns S,
    the same sums with |G(t_{m+1})| + |G(t_m)| in place of the difference
    (bounds the rounding of the time difference)."""
    nt, N, M = bmesh.n_t, bmesh.N, dom.M
    al, ht = bmesh.alpha, bmesh.ht
    out = np.zeros((nt, N, M))
    mag = np.zeros((nt, N, M)) if magnitude else None
    cls = classify(bmesh, dom, rules)
    I_all, K_all = np.nonzero(np.ones((N, dom.K), dtype=bool))
    C_all = cls[I_all, K_all]
    for m in range(nt):
        live = C_all != T_CLS if m == 0 else np.ones(C_all.shape, dtype=bool)
        r2m = rho2(bmesh, dom, I_all, K_all, m)
        orders = np.array([rules.order(c, m, r) for c, r in zip(C_all, r2m)], dtype=np.int64)
        for order in np.unique(orders[live]):
            sel = np.nonzero(live & (orders == order))[0]
            for p0 in range(0, sel.size, chunk):
                Ii, Kk = I_all[sel[p0:p0 + chunk]], K_all[sel[p0:p0 + chunk]]
                r2, wl = tensor_points(bmesh, dom, Ii, Kk, int(order))
                Gb, Ga = G(r2, (m + 1) * ht, al), G(r2, m * ht, al)
                val = np.einsum('pq,pqc->pc', Gb - Ga, wl)
                J = dom.tris[Kk]
                for cc in range(3):
                    np.add.at(out[m], (Ii, J[:, cc]), val[:, cc])
                if magnitude:
                    mv = np.einsum('pq,pqc->pc', np.abs(Gb) + np.abs(Ga), np.abs(wl))
                    for cc in range(3):
                        np.add.at(mag[m], (Ii, J[:, cc]), mv[:, cc])
    # touching pairs, m = 0: polar rule
    for i, k in zip(*np.nonzero(cls == T_CLS)):
        r2, wl = polar_points(bmesh, dom, i, k, rules)
        Gv = G(r2, ht, al)
        val = Gv @ wl
        for cc in range(3):
            out[0, i, dom.tris[k, cc]] += val[cc]
            if magnitude:
                mag[0, i, dom.tris[k, cc]] += np.abs(Gv) @ np.abs(wl[:, cc])
    return (out, mag) if magnitude else out


def apply(M0, u0):
    """(M_h^0 u_0)[m][i] for u0 of shape (M,) or (B, M)."""
    return np.einsum('mij,...j->...mi', M0, u0)


# ---- Section 4 example: u(x, t) = exp(-t/alpha) sin(x . d), d = (cos th, sin th)

def planewave_g(bmesh: BoundaryMesh, theta=np.pi / 8):
    """g[n][p]: time average over tau_n of u(x_p, .) (the discrete Dirichlet
    datum of the repository's reading: time averages at the vertices)."""
    d = np.array([np.cos(theta), np.sin(theta)])
    al, ht = bmesh.alpha, bmesh.ht
    t = np.arange(bmesh.n_t + 1) * ht
    tavg = al / ht * (np.exp(-t[:-1] / al) - np.exp(-t[1:] / al))
    return tavg[:, None] * np.sin(bmesh.X @ d)[None, :]


def planewave_u0(dom: DomainMesh, theta=np.pi / 8):
    """Nodal interpolant of u_0 = u(., 0) in S_h^1(Omega_h)."""
    d = np.array([np.cos(theta), np.sin(theta)])
    return np.sin(dom.nodes @ d)


def planewave_w_projection(bmesh: BoundaryMesh, theta=np.pi / 8):
    """(Q_h w)[m][i], the element average of w = d_n u = exp(-t/alpha)
    cos(x . d) (d . n): time average exact, the segment average of cos(x . d)
    exact (a sinc form)."""
    d = np.array([np.cos(theta), np.sin(theta)])
    al, ht = bmesh.alpha, bmesh.ht
    t = np.arange(bmesh.n_t + 1) * ht
    tavg = al / ht * (np.exp(-t[:-1] / al) - np.exp(-t[1:] / al))
    c = bmesh.mid @ d
    half = 0.5 * bmesh.h * (bmesh.t @ d)
    savg = np.cos(c) * np.sinc(half / np.pi)          # np.sinc(x) = sin(pi x)/(pi x)
    return tavg[:, None] * (savg * (bmesh.n @ d))[None, :]
