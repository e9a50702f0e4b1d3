"""Pins for oracle.quadrature: exactness and singular integrals in closed form."""
import numpy as np

from oracle import quadrature as Q
from oracle.rules import DEFAULT_RULES as R


def test_gauss_polynomial_exactness():
    for n in (2, 4, 8, 16):
        x, w = Q.gauss01(n)
        for k in range(2 * n):
            assert abs((w * x ** k).sum() - 1.0 / (k + 1)) < 1e-14


def test_graded_log():
    x, w = Q.graded01(R.graded_sigma, R.graded_levels, R.graded_points)
    assert abs((w * np.log(x)).sum() + 1.0) < 1e-13                  # int ln u = -1
    assert abs((w * x * x * np.log(x)).sum() + 1.0 / 9.0) < 1e-14     # int u^2 ln u = -1/9


def test_identical_rule_log_diagonal():
    xi, eta, w, mode, p, _ = Q.identical_rule(R)
    assert mode == 'S'
    assert np.allclose(p, xi - eta, atol=1e-15)
    # int_0^1 int_0^1 ln|xi - eta| = -3/2 ; int xi*eta ln|xi-eta| = -7/16 (by 2 int_0^1 (1-u) .. )
    assert abs((w * np.log(np.abs(p))).sum() + 1.5) < 1e-13
    assert abs(w.sum() - 1.0) < 1e-14
    # polynomial weights: int xi eta = 1/4
    assert abs((w * xi * eta).sum() - 0.25) < 1e-14


def test_adjacent_rule_log_corner():
    # int_0^1 int_0^1 ln(x^2 + y^2) dx dy = ln 2 - 3 + pi/2
    ref = np.log(2.0) - 3.0 + np.pi / 2.0
    for corner, mode in (((1.0, 0.0), 'N'), ((0.0, 1.0), 'P')):
        xi, eta, w, m, p, q = Q.adjacent_rule(R, *corner)
        assert m == mode
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs((w * np.log(p * p + q * q)).sum() - ref) < 1e-13
        # offsets measure the distance to the shared corner
        assert np.allclose(np.abs(xi - corner[0]), p, atol=1e-15)
        assert np.allclose(np.abs(eta - corner[1]), q, atol=1e-15)
        assert abs((w * xi * eta).sum() - 0.25) < 1e-14
