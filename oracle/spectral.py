"""One-dimensional spectral building blocks (Section 3.1, Appendix A.1).

* Chebyshev--Lobatto points, p per dimension, endpoints included, ascending.
* Chebyshev spectral differentiation matrix (Trefethen, Spectral Methods in
  MATLAB, ch. 6), written here through barycentric weights:
  D_ij = (w_j / w_i) / (x_i - x_j) for i != j, D_ii = -sum_{j != i} D_ij.
* Gauss--Legendre nodes and weights by the Golub--Welsch eigenvalue method.
* Barycentric Lagrange interpolation matrices (Berrut & Trefethen 2004),
  the "barycentric Lagrange interpolation matrix" of Appendix A.1.

Pins: tests/test_oracle_spectral.py (exactness on polynomials, agreement of
Gauss rules with numpy.polynomial.legendre.leggauss).
"""

from __future__ import annotations

import numpy as np


def cheb_points(p: int, a: float = -1.0, b: float = 1.0) -> np.ndarray:
    """p Chebyshev--Lobatto points on [a, b], ascending (Section 3.1)."""
    if p < 2:
        raise ValueError("p >= 2")
    t = -np.cos(np.pi * np.arange(p) / (p - 1))
    return 0.5 * (a + b) + 0.5 * (b - a) * t


def bary_weights(x: np.ndarray) -> np.ndarray:
    """Barycentric weights w_j = 1 / prod_{k != j} (x_j - x_k), rescaled."""
    x = np.asarray(x, float)
    n = len(x)
    w = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                w[j] *= (x[j] - x[k])
    w = 1.0 / w
    return w / np.max(np.abs(w))


def diff_matrix(x: np.ndarray) -> np.ndarray:
    """Spectral differentiation matrix on the nodes x (exact on polynomials of
    degree <= len(x) - 1)."""
    x = np.asarray(x, float)
    n = len(x)
    w = bary_weights(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def gauss_legendre(q: int, a: float = -1.0, b: float = 1.0):
    """q-point Gauss--Legendre rule on [a, b] (Golub--Welsch): the nodes are
    the eigenvalues of the symmetric Jacobi matrix of the Legendre recurrence
    and the weights are 2 * (first eigenvector component)^2."""
    if q < 1:
        raise ValueError("q >= 1")
    k = np.arange(1, q)
    beta = k / np.sqrt(4.0 * k * k - 1.0)
    J = np.diag(beta, 1) + np.diag(beta, -1)
    lam, V = np.linalg.eigh(J)
    order = np.argsort(lam)
    t = lam[order]
    w = 2.0 * V[0, order] ** 2
    return 0.5 * (a + b) + 0.5 * (b - a) * t, 0.5 * (b - a) * w


def interp_matrix(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Barycentric Lagrange interpolation from values on ``src`` to ``dst``:
    M_ij = (w_j / (t_i - s_j)) / sum_k (w_k / (t_i - s_k)), with an exact unit
    row when t_i coincides with a node."""
    src = np.asarray(src, float)
    dst = np.asarray(dst, float)
    w = bary_weights(src)
    M = np.zeros((len(dst), len(src)))
    for i, t in enumerate(dst):
        diff = t - src
        hit = np.nonzero(diff == 0.0)[0]
        if len(hit):
            M[i, hit[0]] = 1.0
            continue
        r = w / diff
        M[i, :] = r / r.sum()
    return M
