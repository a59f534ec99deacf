"""Pins of the oracle's 1D tables (Gauss-Legendre rule, Lagrange basis)
against mathematics that does not go through the oracle: monomial moments,
numpy's independent Golub-Welsch routine, and polynomial identities."""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

from oracle.dg import gauss_legendre, lagrange


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_legendre_matches_numpy(n):
    x, w = gauss_legendre(n)
    z, ww = npleg.leggauss(n)
    np.testing.assert_allclose(x, (z + 1) / 2, rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, ww / 2, rtol=0, atol=2e-15)


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_legendre_exactness(n):
    """n points integrate x^m exactly on [0,1] for m <= 2n-1, not for 2n."""
    x, w = gauss_legendre(n)
    for m in range(2 * n):
        assert abs((w * x ** m).sum() - 1.0 / (m + 1)) < 1e-14
    assert abs((w * x ** (2 * n)).sum() - 1.0 / (2 * n + 1)) > 1e-12


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_lagrange_identities(n):
    nodes, _ = gauss_legendre(n)
    for i, xi in enumerate(nodes):
        v, _ = lagrange(nodes, xi)
        np.testing.assert_allclose(v, np.eye(n)[i], atol=1e-14)
    rng = np.random.default_rng(0)
    coef = rng.standard_normal(n)       # polynomial of degree n-1
    poly = np.polynomial.Polynomial(coef)
    for x in rng.uniform(0, 1, 7):
        v, d = lagrange(nodes, x)
        assert abs(v.sum() - 1.0) < 1e-13          # partition of unity
        assert abs(d.sum()) < 1e-12                # derivative of the constant
        assert abs(v @ poly(nodes) - poly(x)) < 1e-12
        assert abs(d @ poly(nodes) - poly.deriv()(x)) < 1e-11
