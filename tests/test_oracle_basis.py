"""Pins of the oracle's 1D bases against textbook closed forms (Sec. 2.2)."""
import math

import numpy as np
import pytest

from oracle.basis import gauss_legendre, gll_points, lagrange
from oracle.discretization import ricker

# Textbook GLL nodes/weights (e.g. Canuto et al., Spectral Methods, Table 2.2 values)
GLL = {
    1: ([-1, 1], [1, 1]),
    2: ([-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1],
        [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_textbook(p):
    x, w = gll_points(p)
    np.testing.assert_allclose(x, GLL[p][0], atol=1e-15)
    np.testing.assert_allclose(w, GLL[p][1], rtol=1e-14)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 8])
def test_gll_exactness_degree(p):
    x, w = gll_points(p)
    for k in range(0, 2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    # degree 2p is NOT integrated exactly by GLL (distinguishes it from Gauss)
    assert abs(np.sum(w * x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("n", [2, 3, 5])
def test_gauss_exactness(n):
    x, w = gauss_legendre(n)
    for k in range(0, 2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_cardinal_and_derivative(p):
    nodes, _ = gll_points(p)
    L, D = lagrange(nodes, nodes)
    np.testing.assert_allclose(L, np.eye(p + 1), atol=1e-14)
    xs = np.linspace(-1, 1, 13)
    L, D = lagrange(nodes, xs)
    np.testing.assert_allclose(L.sum(axis=0), 1.0, atol=1e-13)
    np.testing.assert_allclose(D.sum(axis=0), 0.0, atol=1e-12)
    # derivative against the exact derivative of the interpolating polynomial
    for a in range(p + 1):
        coef = np.polyfit(nodes, np.eye(p + 1)[a], p)
        np.testing.assert_allclose(D[a], np.polyval(np.polyder(coef), xs), atol=1e-10)


def test_ricker_closed_form():
    f_e = 10.0
    t_s = 2 * math.sqrt(6) / (math.pi * f_e)
    assert ricker(t_s, f_e) == pytest.approx(1.0)
    # zero crossings at q = +-1/sqrt(2)
    tz = t_s + 1 / (math.sqrt(2) * math.pi * f_e)
    assert abs(ricker(tz, f_e)) < 1e-14
    # value at q = 1: (1 - 2) e^-1
    assert ricker(t_s + 1 / (math.pi * f_e), f_e) == pytest.approx(-math.exp(-1))
