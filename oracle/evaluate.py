"""Evaluation of u in Q by the representation formula, eq. (2) (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 1, eq. (2): for (x, t) in Q

    u(x, t) = int_Omega U*(x - y, t) u_0(y) dy
              + 1/alpha int_Sigma U*(x - y, t - tau) w(y, tau) ds_y dtau
              - 1/alpha int_Sigma d_{n_y} U*(x - y, t - tau) g(y, tau) ds_y dtau,

evaluated with the discrete data: u_0 in S_h^1(Omega_h) (nodal values u0[j]),
w piecewise constant (w[n][i] on gamma_i x tau_n), g piecewise linear in
space and constant in time (g[n][p] at vertex p on tau_n).

Time, exactly: with s = t - tau, int_{tau_n, tau < t} U*(r, t - tau) dtau =
G(r, t - t_n) - G(r, t - min(t_{n+1}, t)), G(r, s) = alpha/(4 pi)
E1(alpha r^2 / (4 s)); and d_{n_y} U*(x - y, s) = alpha^2 q e^{-z} / (8 pi s^2)
(q = (x - y) . n_y, z = alpha r^2 / (4 s)) has the s-antiderivative
H(r, s) = alpha q / (2 pi r^2) e^{-alpha r^2 / (4 s)}; G(., 0) = H(., 0) = 0.

Space: the paper prints no rule; this one is fixed here and is the rule the
CUDA path implements.  Boundary: per segment gamma_i, n_b Gauss-Legendre
points, n_b = 16 if dist(x, gamma_i) < 2 h_i, 12 if < 4 h_i, else 8.
Volume: per triangle, the collapsed tensor rule (initial.tensor rule on the
triangle only) of the order of the M_h^0 rule's step table with
rho^2 = 4 t / (alpha diam^2) (diffusion length over the triangle size).  The
rule is meant for points inside Omega at a distance of at least half a
segment from Gamma and times t >= ht; closer points need near-singular rules
that are not built.

Pins (tests/test_oracle_evaluate.py): u = 1 and u = a + b . x solve the heat
equation and are reproduced exactly by the discrete spaces (u_0 and g nodal,
w = b . n piecewise constant), so u_h equals them up to the rule's error;
the Section 4 example converges to its exact solution under refinement.
"""
import numpy as np

from .geometry import BoundaryMesh
from .initial import DEFAULT_M0_RULES, DomainMesh
from .quadrature import gauss01
from .special import e1


def boundary_order(dist, h):
    """Gauss points on a segment of length h at distance dist from x."""
    return 16 if dist < 2.0 * h else (12 if dist < 4.0 * h else 8)


def volume_order(t, alpha, diam, rules=DEFAULT_M0_RULES):
    """Order of the triangle rule for U*(., t) on a triangle of size diam."""
    r2 = (4.0 * t) / (alpha * diam * diam)
    for thr, o in rules.steps:
        if r2 >= thr:
            return o
    raise AssertionError("unreachable")


def _G(r2, s, alpha):
    if s <= 0.0:
        return np.zeros_like(r2)
    return alpha / (4.0 * np.pi) * e1(alpha * r2 / (4.0 * s))


def _H(r2, q, s, alpha):
    if s <= 0.0:
        return np.zeros_like(r2)
    return alpha * q / (2.0 * np.pi * r2) * np.exp(-alpha * r2 / (4.0 * s))


def _pt_seg(p, a, b):
    e = b - a
    tt = np.clip(((p - a) * e).sum(-1) / (e * e).sum(-1), 0.0, 1.0)
    d = p - (a + tt[..., None] * e)
    return np.sqrt((d * d).sum(-1))


def boundary_terms(bmesh: BoundaryMesh, x, t, w, g):
    """Single- minus double-layer part of u_h(x, t) (the two Sigma integrals)."""
    N, al, ht = bmesh.N, bmesh.alpha, bmesh.ht
    n_last = min(int(np.ceil(t / ht)), bmesh.n_t)        # steps with t_n < t
    tot = 0.0
    for i in range(N):
        a, b, h = bmesh.a[i], bmesh.b[i], bmesh.h[i]
        nb = boundary_order(_pt_seg(x, a, b), h)
        xi, wq = gauss01(nb)
        y = a[None, :] + xi[:, None] * (b - a)[None, :]
        d = x[None, :] - y
        r2 = (d * d).sum(1)
        q = d @ bmesh.n[i]
        wq = wq * h
        for n in range(n_last):
            s0 = t - n * ht
            s1 = t - min((n + 1) * ht, t)
            dG = _G(r2, s0, al) - _G(r2, s1, al)
            dH = _H(r2, q, s0, al) - _H(r2, q, s1, al)
            tot += w[n, i] * (wq @ dG) / al
            gv = g[n, i] * (1.0 - xi) + g[n, (i + 1) % N] * xi
            tot -= (wq * gv) @ dH / al
    return tot


def volume_term(dom: DomainMesh, x, t, alpha, u0, rules=DEFAULT_M0_RULES):
    """int_Omega U*(x - y, t) u0_h(y) dy."""
    tot = 0.0
    for k in range(dom.K):
        n = volume_order(t, alpha, dom.diam[k], rules)
        g, gw = gauss01(n)
        U = np.repeat(g, n)
        V = np.tile(g, n)
        wuv = np.repeat(gw, n) * np.tile(gw, n) * U
        tri = dom.tris[k]
        v0, v1, v2 = dom.nodes[tri[0]], dom.nodes[tri[1]], dom.nodes[tri[2]]
        y = v0[None, :] + U[:, None] * ((1.0 - V)[:, None] * (v1 - v0)[None, :] + V[:, None] * (v2 - v0)[None, :])
        lam = np.stack([1.0 - U, U * (1.0 - V), U * V], axis=1)
        uh = lam @ u0[tri]
        d = x[None, :] - y
        r2 = (d * d).sum(1)
        Us = alpha / (4.0 * np.pi * t) * np.exp(-alpha * r2 / (4.0 * t))
        tot += 2.0 * dom.area[k] * (wuv * Us) @ uh
    return tot


def evaluate(bmesh: BoundaryMesh, dom, points, times, w, g, u0=None):
    """u_h at the points (P, 2) and times (P,); dom and u0 may be None
    (u_0 = 0)."""
    out = np.zeros(len(times))
    for p, (x, t) in enumerate(zip(np.asarray(points, dtype=np.float64), times)):
        v = boundary_terms(bmesh, x, float(t), w, g)
        if u0 is not None:
            v += volume_term(dom, x, float(t), bmesh.alpha, u0)
        out[p] = v
    return out
