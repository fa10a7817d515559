"""Pins of the oracle's 1D basis: Gauss-Legendre nodes/weights and Lagrange polynomials
(nodal tensor-product basis of Eq. 4, collocated quadrature)."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_matches_library_rule(n):
    x, w = O.gauss(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, wr, rtol=0, atol=2e-15)


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_exact_on_monomials(n):
    # an n-point Gauss rule integrates x^k exactly for k <= 2n-1: int_{-1}^{1} x^k = 2/(k+1), k even
    x, w = O.gauss(n)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    # and not for k = 2n (x^{2n} has a nonzero error)
    k = 2 * n
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("n", range(2, 9))
def test_lagrange_cardinal_and_partition_of_unity(n):
    x, _ = O.gauss(n)
    for a in range(n):
        for b in range(n):
            assert O.lagrange(x, a, x[b]) == (1.0 if a == b else 0.0)
    for xi in (-1.0, -0.3, 0.77, 1.0):
        assert abs(sum(O.lagrange(x, a, xi) for a in range(n)) - 1.0) < 1e-13
        assert abs(sum(O.lagrange_deriv(x, a, xi) for a in range(n))) < 1e-11


@pytest.mark.parametrize("n", range(2, 9))
def test_lagrange_derivative_exact_for_polynomials(n):
    # interpolating f(x) = sum_j c_j x^j (degree n-1) reproduces f and f' exactly
    rng = np.random.default_rng(n)
    coef = rng.standard_normal(n)
    x, _ = O.gauss(n)
    f = np.polyval(coef[::-1], x)
    dcoef = np.polyder(np.poly1d(coef[::-1]))
    for xi in (-1.0, -0.41, 0.0, 0.63, 1.0):
        val = sum(f[a] * O.lagrange(x, a, xi) for a in range(n))
        der = sum(f[a] * O.lagrange_deriv(x, a, xi) for a in range(n))
        assert abs(val - np.polyval(coef[::-1], xi)) < 1e-12
        assert abs(der - dcoef(xi)) < 1e-10
