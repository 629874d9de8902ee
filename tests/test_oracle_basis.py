"""Pins of the oracle's 1D building blocks against numpy's Legendre module and
closed forms (textbook quadrature exactness, Legendre derivatives)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle import oracle as O


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_rule_matches_library_and_is_exact(n):
    x, w = O.gauss_rule(n)
    xr, wr = L.leggauss(n)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w, wr, rtol=0, atol=1e-14)
    # exact for monomials of degree <= 2n-1: int_{-1}^{1} x^k = 2/(k+1) for even k, 0 for odd k
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


@pytest.mark.parametrize("m", range(0, 6))
@pytest.mark.parametrize("k", range(0, 6))
def test_legendre_derivatives_match_library(m, k):
    c = np.zeros(m + 1)
    c[m] = 1.0
    dc = L.legder(c, k) if k else c
    for x in (-1.0, -0.7, -0.13, 0.0, 0.42, 1.0):
        ref = L.legval(x, dc) if dc.size else 0.0
        assert abs(O.legendre_dk(m, k, x) - ref) < 1e-11 * max(1.0, abs(ref))


def test_legendre_closed_forms():
    # P_2 = (3x^2-1)/2, P_3 = (5x^3 - 3x)/2 ; P_m(1) = 1, P_m(-1) = (-1)^m, P_m'(1) = m(m+1)/2
    for x in np.linspace(-1, 1, 7):
        assert abs(O.legendre_dk(2, 0, x) - 0.5 * (3 * x * x - 1)) < 1e-15
        assert abs(O.legendre_dk(3, 0, x) - 0.5 * (5 * x ** 3 - 3 * x)) < 1e-15
    for m in range(8):
        assert abs(O.legendre_dk(m, 0, 1.0) - 1.0) < 1e-13
        assert abs(O.legendre_dk(m, 0, -1.0) - (-1.0) ** m) < 1e-13
        assert abs(O.legendre_dk(m, 1, 1.0) - m * (m + 1) / 2.0) < 1e-12
