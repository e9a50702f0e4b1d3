"""Quadrature rules on [0,1] and [0,1]^2 for the oracle (test infrastructure).

Gauss-Legendre nodes come from the library routine
``numpy.polynomial.legendre.leggauss``.  The singular rules are the textbook
constructions:

* geometrically graded composite Gauss on [0,1] toward 0 (breakpoints
  sigma^L < ... < sigma < 1, ``p`` points per sub-interval), which integrates
  u^a log u type singularities at 0 with exponential convergence
  (Schwab, p- and hp-FEM, 1998, Sec. 4.4);
* for identical pieces, the split of [0,1]^2 along the diagonal and the change
  of variables u = |xi - eta| (the inner variable along the diagonal);
* for pieces sharing a vertex, the Duffy transformation of each of the two
  triangles of [0,1]^2 about the shared corner (Duffy, SIAM J. Numer. Anal. 19,
  1982).

Pins (tests/test_oracle_quadrature.py): polynomial exactness, integrals of
log|xi - eta| and log(xi^2 + eta^2) against closed forms.
"""
import numpy as np


def gauss01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def graded01(sigma: float, levels: int, p: int):
    """Composite Gauss on [0,1] graded geometrically toward 0."""
    bps = [0.0] + [sigma ** k for k in range(levels, 0, -1)] + [1.0]
    g, gw = gauss01(p)
    xs, ws = [], []
    for a, b in zip(bps[:-1], bps[1:]):
        xs.append(a + (b - a) * g)
        ws.append((b - a) * gw)
    return np.concatenate(xs), np.concatenate(ws)


# Every rule returns (xi, eta, w, mode, p, q).  (xi, eta) are the local
# parameters on the two pieces (for the basis functions); (p, q) are the same
# points written as offsets from the singular point, so that x - y can be formed
# without cancellation (points come within 1e-10 of the shared vertex):
#   mode 'T': x - y = (A0 - B0) + xi ea - eta eb           (p = xi, q = eta)
#   mode 'S': x - y = p ea, p = xi - eta                   (identical pieces)
#   mode 'N': x - y = -p ea - q eb, p = 1 - xi, q = eta    (end of a = start of b)
#   mode 'P': x - y = p ea + q eb, p = xi, q = 1 - eta     (start of a = end of b)
# with ea = A1 - A0, eb = B1 - B0.


def tensor_rule(n: int):
    """n x n tensor Gauss on [0,1]^2."""
    g, gw = gauss01(n)
    xi = np.repeat(g, n)
    eta = np.tile(g, n)
    w = np.repeat(gw, n) * np.tile(gw, n)
    return xi, eta, w, 'T', xi, eta


def identical_rule(rules):
    """Rule on [0,1]^2 for a piece paired with itself (singular diagonal).

    Triangle xi > eta: u = xi - eta graded toward 0, eta = (1 - u) tau with tau
    Gauss; triangle xi < eta mirrored.  Jacobian (1 - u).
    """
    u, wu = graded01(rules.graded_sigma, rules.graded_levels, rules.graded_points)
    tau, wt = gauss01(rules.singular_inner)
    U = np.repeat(u, tau.size)
    WU = np.repeat(wu, tau.size)
    TA = np.tile(tau, u.size)
    WT = np.tile(wt, u.size)
    lo = (1.0 - U) * TA
    w = WU * WT * (1.0 - U)
    xi = np.concatenate([lo + U, lo])
    eta = np.concatenate([lo, lo + U])
    u = np.concatenate([U, -U])
    return xi, eta, np.concatenate([w, w]), 'S', u, None


def adjacent_rule(rules, xi_c: float, eta_c: float):
    """Rule on [0,1]^2 for two pieces sharing the vertex at (xi_c, eta_c).

    In reflected coordinates (xi', eta') with the corner at the origin, the two
    triangles eta' <= xi' and xi' <= eta' are mapped by Duffy's
    (rho, t) -> (rho, rho t) with Jacobian rho; rho is graded toward 0.
    """
    rho, wr = graded01(rules.graded_sigma, rules.graded_levels, rules.graded_points)
    t, wt = gauss01(rules.duffy_angular)
    R = np.repeat(rho, t.size)
    WR = np.repeat(wr, t.size)
    Tt = np.tile(t, rho.size)
    WT = np.tile(wt, rho.size)
    w = WR * WT * R
    a1, b1 = R, R * Tt            # eta' <= xi'
    a2, b2 = R * Tt, R            # xi' <= eta'
    xp = np.concatenate([a1, a2])
    ep = np.concatenate([b1, b2])
    W = np.concatenate([w, w])
    if (xi_c, eta_c) == (1.0, 0.0):
        return 1.0 - xp, ep, W, 'N', xp, ep
    if (xi_c, eta_c) == (0.0, 1.0):
        return xp, 1.0 - ep, W, 'P', xp, ep
    raise ValueError("shared corner must be (1,0) or (0,1)")
