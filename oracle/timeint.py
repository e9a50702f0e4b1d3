"""Exact double time integrals of the heat kernels over uniform time steps.

Section 1 defines the fundamental solution
    U*(x - y, s) = alpha / (4 pi s) exp(-alpha |x-y|^2 / (4 s)),  s > 0,
and 0 for s <= 0; the single layer operator carries (1/alpha) U* and the double
layer (1/alpha) d_{n_y} U* (eq. (2), (3)).  With r = |x - y|,
c = alpha r^2 / 4, z(s) = c / s and q = (x - y) . n_y, a kernel G(s) and its
second antiderivative F (F'' = G, F(0) = F'(0) = 0) give the exact integral
over two time steps of length ht at lag d = m - n:

    int_{tau_m} int_{tau_n} G(t - tau) dtau dt = F((d+1) ht) - 2 F(d ht) + F((d-1) ht)

(the "second difference" D2_d F, F = 0 for s <= 0).  The antiderivatives are

    V : G_V = (1/alpha) U*          F_V = s/(4 pi) [E1(z) - E2(z)]
    K : G_K = (1/alpha) d_{n_y} U*  F_K = q s E2(z) alpha / (8 pi c)
    D : G_1 = d_s U*                F_1 = alpha/(4 pi) E1(z)

(G_1 is the kernel of the time term of the hypersingular form, Section 2).
Each function below returns D2_d F (for K divided by q) for an array of c.

Evaluation (the reference discretisation, identical on the CUDA side):
* d = 0: F(ht) in closed form;
* d = 1, z = c/ht < 1: a series rearrangement in which the log c terms cancel
  analytically (E1(z) = -gamma - ln z + Ein(z)); z >= 1: closed form;
* d >= 2: closed form when z_d = c/(d ht) > d/2, otherwise the Peano form
  D2_d F = int_{-ht}^{ht} (ht - |u|) G(d ht + u) du with Gauss nodes on the two
  time intervals, which avoids the cancellation of the second difference.

Pins: tests/test_oracle_timeint.py compares every branch with nested
adaptive mpmath quadrature of the kernel G over the two time steps.
"""
import numpy as np

from .quadrature import gauss01
from .special import EULER_GAMMA, e1, e2, ein, phi

FOUR_PI = 4.0 * np.pi


# --- closed-form antiderivatives (c > 0, s > 0) ---------------------------------

def F_V(c, s):
    return s / FOUR_PI * phi(c / s)


def F_Kq(c, s, alpha):
    return alpha / (2.0 * FOUR_PI * c) * s * e2(c / s)


def F_1(c, s, alpha):
    return alpha / FOUR_PI * e1(c / s)


# --- kernels G (second derivative of F in s) -------------------------------------

def G_V(c, s):
    return np.exp(-c / s) / (FOUR_PI * s)


def G_Kq(c, s, alpha):
    return alpha * np.exp(-c / s) / (2.0 * FOUR_PI * s * s)


def G_1(c, s, alpha):
    return alpha / FOUR_PI * np.exp(-c / s) * (c / s ** 3 - 1.0 / (s * s))


def _closed(Ffun, c, d, ht):
    out = Ffun(c, (d + 1) * ht) - 2.0 * Ffun(c, d * ht)
    if d >= 2:
        out = out + Ffun(c, (d - 1) * ht)
    return out


def _peano(Gfun, c, d, ht, rules):
    """int_{(d-1)ht}^{(d+1)ht} (ht - |s - d ht|) G(s) ds, Gauss per interval."""
    tl, wl = gauss01(rules.peano_order(d - 1))
    tr, wr = gauss01(rules.peano_order(d))
    c_ = np.asarray(c)[..., None]
    left = (wl * tl * Gfun(c_, (d - 1 + tl) * ht)).sum(-1)
    right = (wr * (1.0 - tr) * Gfun(c_, (d + tr) * ht)).sum(-1)
    return ht * ht * (left + right)


def _split(c, d, ht, closed_fn, peano_fn):
    c = np.asarray(c, dtype=np.float64)
    out = np.empty_like(c)
    zd = c / (d * ht)
    use_closed = zd > 0.5 * d
    if np.any(use_closed):
        out[use_closed] = closed_fn(c[use_closed])
    if np.any(~use_closed):
        out[~use_closed] = peano_fn(c[~use_closed])
    return out


# --- V ------------------------------------------------------------------------

def lag_V(c, d, ht, alpha, rules):
    """D2_d F_V for an array of c = alpha r^2 / 4."""
    c = np.asarray(c, dtype=np.float64)
    if d == 0:
        return F_V(c, ht)
    if d == 1:
        z = c / ht
        out = np.empty_like(c)
        sm = z < 1.0
        zs = z[sm]
        e_half, e_full = ein(0.5 * zs), ein(zs)
        out[sm] = ht / (2.0 * np.pi) * (
            np.log(2.0) + e_half - e_full
            + 0.5 * zs * (EULER_GAMMA + np.log(2.0 * zs) + e_half - 2.0 * e_full)
            + np.exp(-0.5 * zs) * np.expm1(-0.5 * zs))
        out[~sm] = _closed(F_V, c[~sm], 1, ht)
        return out
    return _split(c, d, ht, lambda cc: _closed(F_V, cc, d, ht),
                  lambda cc: _peano(G_V, cc, d, ht, rules))


# --- K (divided by q) -------------------------------------------------------------

def lag_Kq(c, d, ht, alpha, rules):
    """D2_d F_K / q for an array of c = alpha r^2 / 4."""
    c = np.asarray(c, dtype=np.float64)
    F = lambda cc, s: F_Kq(cc, s, alpha)       # noqa: E731
    G = lambda cc, s: G_Kq(cc, s, alpha)       # noqa: E731
    if d == 0:
        return F(c, ht)
    if d == 1:
        z = c / ht
        out = np.empty_like(c)
        sm = z < 1.0
        zs = z[sm]
        out[sm] = alpha / FOUR_PI * (
            -np.exp(-0.5 * zs) * np.expm1(-0.5 * zs) / zs
            - 0.5 * (EULER_GAMMA + np.log(2.0 * zs))
            - 0.5 * ein(0.5 * zs) + ein(zs))
        out[~sm] = _closed(F, c[~sm], 1, ht)
        return out
    return _split(c, d, ht, lambda cc: _closed(F, cc, d, ht),
                  lambda cc: _peano(G, cc, d, ht, rules))


# --- D time term ------------------------------------------------------------------

def lag_1(c, d, ht, alpha, rules):
    """D2_d F_1 (time term of the hypersingular form) for c = alpha r^2 / 4."""
    c = np.asarray(c, dtype=np.float64)
    F = lambda cc, s: F_1(cc, s, alpha)        # noqa: E731
    G = lambda cc, s: G_1(cc, s, alpha)        # noqa: E731
    if d == 0:
        return F(c, ht)
    if d == 1:
        z = c / ht
        out = np.empty_like(c)
        sm = z < 1.0
        zs = z[sm]
        out[sm] = alpha / FOUR_PI * (
            EULER_GAMMA + np.log(2.0 * zs) + ein(0.5 * zs) - 2.0 * ein(zs))
        out[~sm] = _closed(F, c[~sm], 1, ht)
        return out
    return _split(c, d, ht, lambda cc: _closed(F, cc, d, ht),
                  lambda cc: _peano(G, cc, d, ht, rules))


# --- derivatives in c (shape and alpha gradients) ----------------------------------
#
# Each entry depends on the geometry and on alpha only through c = alpha r^2 / 4
# (and, for K, the explicit factor alpha and q), so the gradients need
# d/dc of every branch above.  With E1' = -e^{-z}/z and E2' = -E1:
#   d/dc F_V(c, s)  = (1/(4 pi)) (E1 - E2)'(c/s) = -E2(z) / (4 pi z)
#   d/dc F_Kq(c, s) = -alpha / (8 pi c) (E2(z)/z + E1(z))
#   d/dc G(c, s)    = -G(c, s) / s            (G = e^{-c/s} x factors of s)
# The lag-1 forms, written with z = c/ht (d/dc = (1/ht) d/dz):
#   V: the derivative of the series form,
#      (1/(4 pi)) [gamma + ln(2 z) + Ein(z/2) - 2 Ein(z) + (2/z) e^{-z/2} expm1(-z/2)],
#      in which the log terms of E1(z/2) - 2 E1(z) are again combined analytically;
#   K: D2_1 F_Kq = alpha (E2(z/2) - E2(z)) / (4 pi z) =: alpha B(z) / (4 pi), and
#      B'(z) = (E1(z) - E1(z/2)/2) / z - B(z) / z = -(e^{-z/2} - e^{-z}) / z^2,
#      valid for every z (e^{-z/2} - e^{-z} = -e^{-z/2} expm1(-z/2), no cancellation).

def dF_V(c, s):
    z = c / s
    return -e2(z) / (FOUR_PI * z)


def dF_Kq(c, s, alpha):
    z = c / s
    return -alpha / (2.0 * FOUR_PI * c) * (e2(z) / z + e1(z))


def dG_V(c, s):
    return -G_V(c, s) / s


def dG_Kq(c, s, alpha):
    return -G_Kq(c, s, alpha) / s


def dlag_V(c, d, ht, alpha, rules):
    """d/dc of lag_V (same branches)."""
    c = np.asarray(c, dtype=np.float64)
    if d == 0:
        return dF_V(c, ht)
    if d == 1:
        z = c / ht
        out = np.empty_like(c)
        sm = z < 1.0
        zs = z[sm]
        out[sm] = (EULER_GAMMA + np.log(2.0 * zs) + ein(0.5 * zs) - 2.0 * ein(zs)
                   + 2.0 / zs * np.exp(-0.5 * zs) * np.expm1(-0.5 * zs)) / FOUR_PI
        out[~sm] = _closed(dF_V, c[~sm], 1, ht)
        return out
    return _split(c, d, ht, lambda cc: _closed(dF_V, cc, d, ht),
                  lambda cc: _peano(dG_V, cc, d, ht, rules))


def dlag_Kq(c, d, ht, alpha, rules):
    """d/dc of lag_Kq (same branches; lag 1 in the closed form above)."""
    c = np.asarray(c, dtype=np.float64)
    F = lambda cc, s: dF_Kq(cc, s, alpha)      # noqa: E731
    G = lambda cc, s: dG_Kq(cc, s, alpha)      # noqa: E731
    if d == 0:
        return F(c, ht)
    if d == 1:
        z = c / ht
        return alpha / (FOUR_PI * ht) * np.exp(-0.5 * z) * np.expm1(-0.5 * z) / (z * z)
    return _split(c, d, ht, lambda cc: _closed(F, cc, d, ht),
                  lambda cc: _peano(G, cc, d, ht, rules))
