"""Exponential integrals for the oracle (test infrastructure only).

E1 and E2 are the library routines ``scipy.special.exp1`` and
``scipy.special.expn(2, .)``.  ``ein`` is the entire function
Ein(z) = sum_{k>=1} (-1)^{k+1} z^k / (k k!)  (Abramowitz & Stegun 5.1.11,
E1(z) = -gamma - ln z + Ein(z)), summed term by term; it is only used for
z <= 1 where the series converges fast.

Pins (tests/test_oracle_special.py): E1, E2 against mpmath over z in
[1e-12, 700]; Ein against mpmath's ``ein``-free identity E1 + gamma + ln z at
40 digits.
"""
import numpy as np
from scipy.special import exp1, expn

EULER_GAMMA = 0.577215664901532860606512090082402431


def e1(z):
    """E1(z) = int_1^inf e^{-z t} / t dt, z > 0 (scipy.special.exp1)."""
    return exp1(z)


def e2(z):
    """E2(z) = int_1^inf e^{-z t} / t^2 dt, z >= 0 (scipy.special.expn)."""
    return expn(2, z)


def phi(z):
    """E1(z) - E2(z) = int_1^inf e^{-z t} (t - 1) / t^2 dt  (> 0)."""
    return exp1(z) - expn(2, z)


def ein(z, terms: int = 30):
    """Ein(z) = sum_{k=1}^{terms} (-1)^{k+1} z^k / (k k!) for |z| <= 1."""
    z = np.asarray(z, dtype=np.float64)
    acc = np.zeros_like(z)
    term = np.ones_like(z)          # z^k / k!
    for k in range(1, terms + 1):
        term = term * z / k
        acc = acc + ((-1.0) ** (k + 1)) * term / k
    return acc
