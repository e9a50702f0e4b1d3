"""Pins for oracle.special: E1, E2 and Ein against mpmath (independent code)."""
import numpy as np
import pytest

from oracle import special

mp = pytest.importorskip("mpmath")


def test_e1_e2_against_mpmath():
    mp.mp.dps = 40
    zs = np.concatenate([np.logspace(-12, 0, 25), np.linspace(1.0, 60.0, 40), [100.0, 300.0, 699.0]])
    for z in zs:
        e1 = float(mp.e1(z))
        e2 = float(mp.expint(2, z))
        assert abs(special.e1(z) / e1 - 1) < 2e-15
        assert abs(special.e2(z) / e2 - 1) < 2e-15
        ph = float(mp.e1(z) - mp.expint(2, z))
        assert abs(special.phi(z) / ph - 1) < max(1e-14, 1e-15 * z)   # E1 - E2 cancels about 3x near z = 1


def test_ein_series():
    mp.mp.dps = 40
    for z in np.concatenate([np.logspace(-10, 0, 21)]):
        ref = mp.e1(z) + mp.euler + mp.log(z)           # Ein = E1 + gamma + ln z
        assert abs(special.ein(z) - float(ref)) <= 4e-16 * max(1.0, abs(float(ref)))
