"""Pins for oracle.spectral: textbook identities, independent of the oracle's
own formulas (Section 3.1, Appendix A.1)."""

import numpy as np
import pytest

from oracle import spectral as sp


@pytest.mark.parametrize("p", [4, 8, 12, 16])
def test_cheb_points_are_extrema_of_T(p):
    # Chebyshev--Lobatto points are the extrema of T_{p-1}: |T_{p-1}(x_j)| = 1
    x = sp.cheb_points(p)
    T = np.polynomial.chebyshev.Chebyshev.basis(p - 1)
    assert np.allclose(np.abs(T(x)), 1.0, atol=1e-13)
    assert np.all(np.diff(x) > 0) and x[0] == -1.0 and x[-1] == 1.0


@pytest.mark.parametrize("p", [4, 8, 12, 16])
def test_diff_matrix_exact_on_polynomials(p):
    x = sp.cheb_points(p, -0.3, 0.7)
    D = sp.diff_matrix(x)
    rng = np.random.default_rng(p)
    for deg in range(p):
        c = rng.standard_normal(deg + 1)
        P = np.polynomial.Polynomial(c)
        assert np.allclose(D @ P(x), P.deriv()(x), atol=1e-9 * max(1, np.abs(c).sum()) * p ** 2)
    # negative control: degree p is not differentiated exactly
    t = lambda y: (2 * y - 0.4) / 1.0  # noqa: E731  (maps [-0.3, 0.7] onto [-1, 1])
    err = np.abs(D @ t(x) ** p - 2 * p * t(x) ** (p - 1)).max()
    assert err > 1e-6 * 2 * p


@pytest.mark.parametrize("q", [1, 2, 6, 10, 14, 20])
def test_gauss_legendre_matches_leggauss(q):
    x, w = sp.gauss_legendre(q)
    xr, wr = np.polynomial.legendre.leggauss(q)
    assert np.allclose(x, xr, atol=1e-14)
    assert np.allclose(w, wr, atol=1e-14)
    a, b = 0.25, 2.0
    x2, w2 = sp.gauss_legendre(q, a, b)
    # exact for degree 2q-1 on [a, b]
    P = np.polynomial.Polynomial(np.arange(1, 2 * q + 1, dtype=float))
    I = P.integ()
    assert np.isclose(w2 @ P(x2), I(b) - I(a), rtol=1e-13)


@pytest.mark.parametrize("p", [6, 8, 12, 16])
def test_interp_exactness(p):
    q = p - 2
    xc = sp.cheb_points(p)
    xg, _ = sp.gauss_legendre(q)
    G2C = sp.interp_matrix(xg, xc)
    C2G = sp.interp_matrix(xc, xg)
    rng = np.random.default_rng(0)
    for deg in range(q):
        P = np.polynomial.Polynomial(rng.standard_normal(deg + 1))
        assert np.allclose(G2C @ P(xg), P(xc), atol=1e-11)
    for deg in range(p):
        P = np.polynomial.Polynomial(rng.standard_normal(deg + 1))
        assert np.allclose(C2G @ P(xc), P(xg), atol=1e-11)
    # rows sum to one (constants are reproduced) and degree q is not exact
    assert np.allclose(G2C.sum(axis=1), 1.0)
    P = np.polynomial.Polynomial(np.r_[np.zeros(q), 1.0])
    assert np.abs(G2C @ P(xg) - P(xc)).max() > 1e-6


def test_interp_coincident_node():
    x = np.array([-1.0, 0.0, 1.0])
    M = sp.interp_matrix(x, np.array([0.0, 0.5]))
    assert np.array_equal(M[0], [0.0, 1.0, 0.0])
    assert np.allclose(M[1], [-0.125, 0.75, 0.375])
