"""Pins for oracle.timeint: every evaluation branch of the double time integral.

The definition is the double integral over tau_m x tau_n of the kernel G(t - tau)
(heat kernels of Section 1).  Moderate cases are compared with that nested
integral done by mpmath; extreme cases (tiny z, large lags, huge z), where
nested adaptive quadrature is itself unreliable, are compared with the closed
forms evaluated in 40-digit arithmetic, which the moderate cases pin.
"""
import numpy as np
import pytest

from oracle import timeint
from oracle.rules import DEFAULT_RULES as R

mp = pytest.importorskip("mpmath")

HT, ALPHA = 1.0 / 32.0, 0.7


def _G(kind, c):
    a = mp.mpf(ALPHA)

    def G(s):
        if s <= 0:
            return mp.mpf(0)
        e = mp.e ** (-c / s)
        if kind == 'V':       # (1/alpha) U*
            return e / (4 * mp.pi * s)
        if kind == 'K':       # (1/alpha) d_{n_y} U* / q
            return a * e / (8 * mp.pi * s * s)
        return a / (4 * mp.pi) * e * (c / s ** 3 - 1 / s ** 2)   # d_s U*
    return G


def nested(kind, c, d):
    mp.mp.dps = 20
    c = mp.mpf(c)
    ht = mp.mpf(HT)
    G = _G(kind, c)

    def inner(t):
        pts = [mp.mpf(0)] + sorted(x for x in (t - c, t - c / 3, t - 3 * c) if 0 < x < ht) + [ht]
        return mp.quad(lambda tau: G(t - tau), pts)
    outer = [d * ht] + sorted(x for x in (c / 10, c, 10 * c) if d * ht < x < (d + 1) * ht) + [(d + 1) * ht]
    return mp.quad(inner, outer)


def closed40(kind, c, d):
    mp.mp.dps = 40
    c = mp.mpf(c)
    ht = mp.mpf(HT)
    a = mp.mpf(ALPHA)

    def F(s):
        if s <= 0:
            return mp.mpf(0)
        z = c / s
        if kind == 'V':
            return s / (4 * mp.pi) * (mp.e1(z) - mp.expint(2, z))
        if kind == 'K':
            return a / (8 * mp.pi * c) * s * mp.expint(2, z)
        return a / (4 * mp.pi) * mp.e1(z)
    return F((d + 1) * ht) - 2 * F(d * ht) + F((d - 1) * ht)


FN = {'V': timeint.lag_V, 'K': timeint.lag_Kq, '1': timeint.lag_1}


def oracle(kind, c, d):
    return FN[kind](np.array([float(c)]), d, HT, ALPHA, R)[0]


MODERATE = [(0, 0.3), (0, 2.0), (1, 0.05), (1, 0.6), (1, 3.0), (2, 0.3), (2, 1.5), (3, 0.2),
            (6, 0.5 * 6 * 0.9), (6, 0.5 * 6 * 1.1), (20, 0.4), (20, 12.0)]


@pytest.mark.parametrize("kind", ['V', 'K', '1'])
def test_against_nested_double_integral(kind, cpu_pool):
    refs = [cpu_pool.submit(nested, kind, zd * max(d, 1) * HT, d) for d, zd in MODERATE]
    for (d, zd), fut in zip(MODERATE, refs):
        c = zd * max(d, 1) * HT
        ref = float(fut.result())
        got = oracle(kind, c, d)
        assert abs(got - ref) <= 5e-13 * abs(ref), (kind, d, zd, got, ref)


EXTREME = [(0, 1e-9), (0, 1e-4), (1, 1e-9), (1, 1e-4), (1, 0.999), (1, 1.001), (2, 1e-8), (2, 0.99),
           (2, 1.01), (5, 1e-6), (5, 2.49), (5, 2.51), (33, 1e-3), (33, 16.4), (33, 16.6),
           (200, 0.05), (200, 99.0), (200, 101.0), (900, 3.0), (40, 120.0)]


@pytest.mark.parametrize("kind", ['V', 'K', '1'])
def test_extreme_branches_against_closed_form_40_digits(kind):
    for d, zd in EXTREME:
        c = zd * max(d, 1) * HT
        ref = float(closed40(kind, c, d))
        got = oracle(kind, c, d)
        # closed form at large z: E1 - E2 loses ~z eps, the second difference up
        # to 4x more at the switch z_d = d/2
        tol = 2e-13 * max(1.0, zd / 50.0)
        assert abs(got - ref) <= tol * abs(ref), (kind, d, zd, got, ref)


def test_kernel_mass_is_one():
    """int_{R^2} U*(x, t) dx = 1 for every t > 0 (Section 1, U*)."""
    mp.mp.dps = 25
    for t in (1e-3, 0.1, 2.0):
        a = ALPHA
        val = mp.quad(lambda r: 2 * mp.pi * r * a / (4 * mp.pi * t) * mp.e ** (-a * r * r / (4 * t)), [0, mp.inf])
        assert abs(val - 1) < 1e-18
