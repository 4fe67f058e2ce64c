"""Leaf stage of the oracle (Section 3.2, Algorithm "local solve").

* 2D DtN: Algorithm "2D DtN local solve" (Appendix A.1).
* 3D DtN: the same algorithm with the 3D P and Q (Appendix C.1).
* 2D ItI: Algorithm "2D ItI local solve" (Appendix B.1).

Readings of points the paper leaves open:

* v = [0; +L_ii^{-1} f_i].  The printed algorithm has a minus sign, which
  contradicts L v = f, v = 0 on the boundary (Section 2) and the ItI line
  v = B^{-1}(:, I_i) f without one; the closed-form tests fail with it.
* DtN Q = (per-side Chebyshev->Gauss interpolation) o (outward normal
  derivative at the p Chebyshev points of each side, corners included once
  per side); 3D per face with p^2 points.
* DtN P: a boundary Chebyshev node on k sides (faces) gets the mean of the k
  one-panel Gauss->Chebyshev interpolants (k = 2 at 2D corners, 2 on 3D edges,
  3 at 3D corners).
* ItI: side S owns its first p-1 Chebyshev points counterclockwise (x
  ascending, SW corner included), E owns y ascending from SE, N owns x
  descending from NE, W owns y descending from NW.  G and P rows follow the
  owning side; N and H double-count corners.
* "Invert" is LU with partial pivoting (LAPACK getrf through scipy).
"""

from __future__ import annotations

from functools import lru_cache

import numpy as np
import scipy.linalg as sla

from .spectral import cheb_points, diff_matrix, gauss_legendre, interp_matrix


@lru_cache(maxsize=None)
def reference_ops(dim: int, p: int, q: int):
    """Leaf operators for a leaf of side length 2 (rescaled per leaf).

    Returns a dict with the 1D differentiation matrix, the index sets and the
    P / Q (DtN) or P / G / H / Q (ItI) pieces that do not depend on eta."""
    xc = cheb_points(p)
    D = diff_matrix(xc)
    xg, _ = gauss_legendre(q)
    Pi_GC = interp_matrix(xg, xc)   # p x q
    Pi_CG = interp_matrix(xc, xg)   # q x p
    ops = {"xc": xc, "D": D, "Pi_GC": Pi_GC, "Pi_CG": Pi_CG}
    if dim == 2:
        def idx(ix, iy):
            return ix + p * iy
        inner = [idx(ix, iy) for iy in range(1, p - 1) for ix in range(1, p - 1)]
        all_idx = np.arange(p * p)
        Ie = np.array(sorted(set(all_idx) - set(inner)))
        Ii = np.array(inner)
        # nodes of each side, increasing coordinate, with the outward normal
        sides = [
            ([idx(i, 0) for i in range(p)], 1, -1.0),      # S: -d/dy
            ([idx(p - 1, i) for i in range(p)], 0, +1.0),  # E: +d/dx
            ([idx(i, p - 1) for i in range(p)], 1, +1.0),  # N: +d/dy
            ([idx(0, i) for i in range(p)], 0, -1.0),      # W: -d/dx
        ]
        ops.update(Ie=Ie, Ii=Ii, sides=sides)
    else:
        def idx(ix, iy, iz):
            return ix + p * iy + p * p * iz
        inner = set(idx(ix, iy, iz) for iz in range(1, p - 1)
                    for iy in range(1, p - 1) for ix in range(1, p - 1))
        Ie = np.array(sorted(set(range(p ** 3)) - inner))
        Ii = np.array(sorted(inner))
        faces = []
        for axis in range(3):
            for side in (0, 1):
                t1, t2 = [k for k in range(3) if k != axis]
                nodes = []
                for i2 in range(p):
                    for i1 in range(p):
                        ii = [0, 0, 0]
                        ii[axis] = (p - 1) if side else 0
                        ii[t1] = i1
                        ii[t2] = i2
                        nodes.append(idx(*ii))
                faces.append((nodes, axis, +1.0 if side else -1.0))
        ops.update(Ie=Ie, Ii=Ii, sides=faces)
    return ops


@lru_cache(maxsize=None)
def _cheb_D(p: int):
    return diff_matrix(cheb_points(p))


def derivative_matrices(dim: int, p: int, hlen: float):
    """Dx, Dy(, Dz) on the p^dim tensor grid of a leaf of side ``hlen``."""
    D = _cheb_D(p) * (2.0 / hlen)
    I = np.eye(p)
    if dim == 2:
        return [np.kron(I, D), np.kron(D, I)]
    return [np.kron(I, np.kron(I, D)), np.kron(I, np.kron(D, I)), np.kron(D, np.kron(I, I))]


def assemble_L(dim, p, hlen, a, b, c):
    """L = diag(a) Lap + sum_k diag(b_k) d/dx_k + diag(c) on one leaf
    (Section 3.2: spectral differentiation matrices and coefficient samples)."""
    Ds = derivative_matrices(dim, p, hlen)
    lap = sum(Dk @ Dk for Dk in Ds)
    L = a[:, None] * lap + c[:, None] * np.eye(p ** dim)
    for k in range(dim):
        L = L + b[k][:, None] * Ds[k]
    return L


def dtn_P_Q(dim: int, p: int, q: int, hlen: float):
    """P (|I_e| x n_b) and Q (n_b x p^dim) of Appendices A.1 / C.1."""
    ops = reference_ops(dim, p, q)
    Ds = derivative_matrices(dim, p, hlen)
    Pi_GC, Pi_CG = ops["Pi_GC"], ops["Pi_CG"]
    sides = ops["sides"]
    Ie = ops["Ie"]
    npts = p ** dim
    if dim == 2:
        nb = 4 * q
        Q = np.zeros((nb, npts))
        for s, (nodes, axis, sgn) in enumerate(sides):
            Nrows = sgn * Ds[axis][nodes, :]           # p x p^2
            Q[s * q:(s + 1) * q, :] = Pi_CG @ Nrows
        P = np.zeros((len(Ie), nb))
        for r, e in enumerate(Ie):
            hits = [(s, nodes.index(e)) for s, (nodes, _, _) in enumerate(sides) if e in nodes]
            for s, pos in hits:
                P[r, s * q:(s + 1) * q] += Pi_GC[pos, :] / len(hits)
        return P, Q
    nb = 6 * q * q
    Pi2_CG = np.kron(Pi_CG, Pi_CG)                     # q^2 x p^2 (t1 fastest)
    Q = np.zeros((nb, npts))
    for s, (nodes, axis, sgn) in enumerate(sides):
        Nrows = sgn * Ds[axis][nodes, :]
        Q[s * q * q:(s + 1) * q * q, :] = Pi2_CG @ Nrows
    P = np.zeros((len(Ie), nb))
    for r, e in enumerate(Ie):
        hits = [(s, nodes.index(e)) for s, (nodes, _, _) in enumerate(sides) if e in nodes]
        for s, pos in hits:
            i1, i2 = pos % p, pos // p
            P[r, s * q * q:(s + 1) * q * q] += np.kron(Pi_GC[i2, :], Pi_GC[i1, :]) / len(hits)
    return P, Q


def dtn_leaf(dim, p, q, hlen, a, b, c, f):
    """Algorithm "2D DtN local solve" (3D: Appendix C.1) for one leaf.

    Returns T (n_b x n_b), h (n_b), Y (p^d x n_b, natural node order) and
    v (p^d)."""
    ops = reference_ops(dim, p, q)
    Ie, Ii = ops["Ie"], ops["Ii"]
    P, Q = dtn_P_Q(dim, p, q, hlen)
    L = assemble_L(dim, p, hlen, a, b, c)
    Lii = L[np.ix_(Ii, Ii)]
    Lie = L[np.ix_(Ii, Ie)]
    lu = sla.lu_factor(Lii)
    X = sla.lu_solve(lu, Lie @ P)
    Y = np.zeros((p ** dim, P.shape[1]))
    Y[Ie, :] = P
    Y[Ii, :] = -X
    v = np.zeros(p ** dim, dtype=np.result_type(f, float))
    v[Ii] = sla.lu_solve(lu, f[Ii])
    T = Q @ Y
    h = Q @ v
    return T, h, Y, v


def iti_ops(p: int, q: int, hlen: float, eta: float):
    """P, G, H and Q of Appendix B.1 for one 2D leaf of side ``hlen``."""
    ops = reference_ops(2, p, q)
    Dx, Dy = derivative_matrices(2, p, hlen)
    Pi_GC, Pi_CG = ops["Pi_GC"], ops["Pi_CG"]
    sides = ops["sides"]
    npts = p * p
    Ds = [Dx, Dy]
    # owned points per side, as positions along the side (increasing coordinate)
    owned_pos = [list(range(0, p - 1)),      # S: x ascending from SW
                 list(range(0, p - 1)),      # E: y ascending from SE
                 list(range(1, p)),          # N: from NE going west -> x = 1..p-1
                 list(range(1, p))]          # W: from NW going south -> y = 1..p-1
    nown = 4 * (p - 1)
    G = np.zeros((nown, npts), complex)
    P = np.zeros((nown, 4 * q))
    r = 0
    for s, (nodes, axis, sgn) in enumerate(sides):
        for pos in owned_pos[s]:
            node = nodes[pos]
            G[r, :] = sgn * Ds[axis][node, :]
            G[r, node] += 1j * eta
            P[r, s * q:(s + 1) * q] = Pi_GC[pos, :]
            r += 1
    H = np.zeros((4 * p, npts), complex)
    for s, (nodes, axis, sgn) in enumerate(sides):
        H[s * p:(s + 1) * p, :] = sgn * Ds[axis][nodes, :]
        H[s * p + np.arange(p), nodes] -= 1j * eta
    Qb = sla.block_diag(*([Pi_CG] * 4))           # 4q x 4p
    return P, G, H, Qb


def iti_leaf(p, q, hlen, a, b, c, f, eta):
    """Algorithm "2D ItI local solve" for one leaf."""
    ops = reference_ops(2, p, q)
    Ii = ops["Ii"]
    P, G, H, Qb = iti_ops(p, q, hlen, eta)
    L = assemble_L(2, p, hlen, a, b, c)
    B = np.vstack([G, L[Ii, :]])
    lu = sla.lu_factor(B)
    nown = G.shape[0]
    rhs_Y = np.zeros((p * p, 4 * q), complex)
    rhs_Y[:nown, :] = P
    Y = sla.lu_solve(lu, rhs_Y)
    rhs_v = np.zeros(p * p, complex)
    rhs_v[nown:] = f[Ii]
    v = sla.lu_solve(lu, rhs_v)
    QH = Qb @ H
    T = QH @ Y
    h = QH @ v
    return T, h, Y, v
