"""Manufactured data for the oracle: g, f = (1/2 M_h + K_h) g, exact w.

The workload replaces the paper's example (Section 4, which needs u_0 != 0) by
u(x, t) = U*(x - y*, t) with the source y* outside the closure of Omega: it
solves the heat equation of eq. (1) in Q with u_0 = 0, so eq. (4) reduces to
V_h w = (1/2 M_h + K_h) g and the Neumann datum w = d_n u is known exactly.

* g: the coefficient of the P1-in-space / P0-in-time function at vertex p and
  step n is the time average of g(x_p, .) over tau_n,
      g[n][p] = (1/ht) int_{tau_n} U*(x_p - y*, t) dt
              = (1/ht) alpha/(4 pi) [E1(a_p / t_{n+1}) - E1(a_p / t_n)],
  a_p = alpha |x_p - y*|^2 / 4, E1(inf) = 0  (the time antiderivative of U* is
  alpha/(4 pi) E1(a / t)).
* w = d_n U*(x - y*, t) = -alpha^2 / (8 pi t^2) ((x - y*) . n) e^{-a/t}, whose
  integral over tau_m is -alpha / (2 pi |x - y*|^2) ((x - y*) . n)
  [e^{-a/t_{m+1}} - e^{-a/t_m}].
* Q_h w: the piecewise-constant L2 projection (element averages), space by
  8-point Gauss-Legendre per segment, time exact.

Pins: tests/test_oracle_rhs.py (g against mpmath quadrature of U* in time, the
time integral of w against mpmath, convergence of w_h to Q_h w).
"""
import numpy as np

from .quadrature import gauss01
from .solve import toeplitz_apply
from .special import e1
from .assembly import half_mass_apply


def g_vec(mesh, y_star):
    """g[n][p], n = 0..N_t-1, p = 0..N_x-1 (time averages at the vertices)."""
    ys = np.asarray(y_star, dtype=np.float64)
    a = mesh.alpha * ((mesh.X - ys) ** 2).sum(1) / 4.0
    t = np.arange(mesh.n_t + 1) * mesh.ht
    with np.errstate(divide='ignore'):
        E = np.where(t[:, None] > 0, e1(a[None, :] / np.where(t[:, None] > 0, t[:, None], 1.0)), 0.0)
    return (E[1:] - E[:-1]) * mesh.alpha / (4.0 * np.pi) / mesh.ht


def f_vec(mesh, K_blocks, g):
    """f = 1/2 M_h g + K_h g (eq. (4) with u_0 = 0); g, f shaped (N_t, N_x)."""
    return half_mass_apply(mesh, g) + toeplitz_apply(K_blocks, g)


def w_projection(mesh, y_star, n_gauss: int = 8):
    """(Q_h w)[m][i]: average of the exact Neumann datum over gamma_i x tau_m."""
    ys = np.asarray(y_star, dtype=np.float64)
    xg, wg = gauss01(n_gauss)
    x = mesh.a[:, None, :] + xg[None, :, None] * (mesh.b - mesh.a)[:, None, :]
    dx = x - ys
    r2 = (dx * dx).sum(-1)
    qn = (dx * mesh.n[:, None, :]).sum(-1)
    a = mesh.alpha * r2 / 4.0
    t = np.arange(mesh.n_t + 1) * mesh.ht
    with np.errstate(divide='ignore', over='ignore'):
        ex = np.where(t[:, None, None] > 0, np.exp(-a[None] / np.where(t[:, None, None] > 0, t[:, None, None], 1.0)), 0.0)
    tint = -(mesh.alpha / (2.0 * np.pi * r2))[None] * qn[None] * (ex[1:] - ex[:-1])
    return (tint * wg[None, None, :]).sum(-1) / mesh.ht


def l2_rel_error(mesh, w_h, w_ref):
    """||w_h - w_ref||_{L2(Sigma)} / ||w_ref|| for piecewise constants."""
    wt = mesh.h[None, :] * mesh.ht
    return np.sqrt((wt * (w_h - w_ref) ** 2).sum() / (wt * w_ref ** 2).sum())
