"""Size-independent checks of a computed leaf solution: the composite
collocation equations that the HPS solution satisfies exactly (see
oracle/composite.py), evaluated leaf by leaf on a sample of leaves with the
oracle's leaf operators.  Used where the full oracle is too slow to run.

DtN (2D and 3D): per leaf, the interior collocation rows
    L(I_i, :) u - f_i = 0;
per shared side (face), the Gauss data recovered from either leaf agree and
the outward normal derivatives (Q u) cancel; on the root boundary the
recovered Gauss data equal g.
ItI (2D): per leaf L(I_i, :) u - f_i = 0 and G u - P g_in = 0, with g_in =
root data or -(Q H u_neighbour) on a shared side.
"""

from __future__ import annotations

import numpy as np

from oracle import geometry as geo
from oracle import leaf as lf
from oracle.spectral import cheb_points, gauss_legendre, interp_matrix


def _leaf_index_coords(dim, L):
    n1 = 2 ** L
    nl = n1 ** dim
    coords = np.zeros((nl, dim), int)
    for m in range(nl):
        idx = [0] * dim
        for lev in range(L):
            c = (m >> (dim * (L - 1 - lev))) & ((1 << dim) - 1)
            for k in range(dim):
                idx[k] = idx[k] * 2 + ((c >> k) & 1)
        coords[m] = idx
    lookup = {tuple(c): m for m, c in enumerate(coords)}
    return coords, lookup


def _root_panel_slice(dim, L, q, axis, side, tang):
    """Slice of the canonical root boundary vector for one leaf panel."""
    slots = geo.SIDES_2D if dim == 2 else geo.FACES_3D
    s = slots.index((axis, side))
    if dim == 2:
        npan = 2 ** L
        k = s * npan + tang[0]
        return slice(k * q, (k + 1) * q)
    order = geo._face_panel_order(L)
    k = s * len(order) + order.index(tuple(tang))
    return slice(k * q * q, (k + 1) * q * q)


def _gauss_from_side(dim, p, q, u_leaf, nodes):
    """Gauss data of one side (face) recovered from the p-2 (squared)
    non-corner Chebyshev values (exact for data of degree <= q-1)."""
    xc = cheb_points(p)[1:-1]
    xg, _ = gauss_legendre(q)
    M = interp_matrix(xc, xg)
    vals = u_leaf[nodes]
    if dim == 2:
        return M @ vals[1:-1]
    V = vals.reshape(p, p)[1:-1, 1:-1]          # [t2][t1]
    return (M @ V @ M.T).reshape(-1)


def check_dtn(dim, p, L, lo, hi, a, b, c, f, g, u, sample):
    """Returns the largest normalised residual over the sampled leaves."""
    q = p - 2
    corners, hvec = geo.uniform_leaf_boxes(dim, lo, hi, L)
    hlen = float(hvec[0])
    ops = lf.reference_ops(dim, p, q)
    Ii = ops["Ii"]
    P_, Q = lf.dtn_P_Q(dim, p, q, hlen)
    sides = ops["sides"]
    coords, lookup = _leaf_index_coords(dim, L)
    slots = geo.SIDES_2D if dim == 2 else geo.FACES_3D
    n1 = 2 ** L
    uscale = np.abs(u).max()
    worst = 0.0
    for m in sample:
        Lm = lf.assemble_L(dim, p, hlen, a[m], [bk[m] for bk in b], c[m])
        res = Lm[Ii, :] @ u[m] - f[m][Ii]
        scale = np.abs(Lm[Ii, :]).sum(axis=1).max() * uscale + np.abs(f[m]).max()
        worst = max(worst, np.abs(res).max() / scale)
        nrm = Q @ u[m]
        nsc = np.abs(Q).sum(axis=1).max() * uscale
        npan = q ** (dim - 1)
        for s, (axis, side) in enumerate(slots):
            nodes = sides[s][0]
            gs = _gauss_from_side(dim, p, q, u[m], nodes)
            idx = coords[m].copy()
            idx[axis] += 1 if side else -1
            tang = [coords[m][k] for k in range(dim) if k != axis]
            if idx[axis] < 0 or idx[axis] >= n1:
                sl = _root_panel_slice(dim, L, q, axis, side, tang)
                worst = max(worst, np.abs(gs - g[sl]).max() / max(uscale, 1e-300))
                continue
            nb_leaf = lookup[tuple(idx)]
            s2 = slots.index((axis, 1 - side))
            gs2 = _gauss_from_side(dim, p, q, u[nb_leaf], sides[s2][0])
            worst = max(worst, np.abs(gs - gs2).max() / max(uscale, 1e-300))
            nrm2 = Q @ u[nb_leaf]
            flux = nrm[s * npan:(s + 1) * npan] + nrm2[s2 * npan:(s2 + 1) * npan]
            worst = max(worst, np.abs(flux).max() / nsc)
    return worst


def check_iti(p, L, lo, hi, a, b, c, f, g, u, eta, sample):
    dim, q = 2, p - 2
    corners, hvec = geo.uniform_leaf_boxes(dim, lo, hi, L)
    hlen = float(hvec[0])
    ops = lf.reference_ops(dim, p, q)
    Ii = ops["Ii"]
    P_, G, H, Qb = lf.iti_ops(p, q, hlen, eta)
    QH = Qb @ H
    coords, lookup = _leaf_index_coords(dim, L)
    n1 = 2 ** L
    uscale = np.abs(u).max()
    worst = 0.0
    for m in sample:
        Lm = lf.assemble_L(dim, p, hlen, a[m], [bk[m] for bk in b], c[m])
        res = Lm[Ii, :] @ u[m] - f[m][Ii]
        scale = np.abs(Lm[Ii, :]).sum(axis=1).max() * uscale + np.abs(f[m]).max()
        worst = max(worst, np.abs(res).max() / scale)
        gin = np.zeros(4 * q, complex)
        for s, (axis, side) in enumerate(geo.SIDES_2D):
            idx = coords[m].copy()
            idx[axis] += 1 if side else -1
            if idx[axis] < 0 or idx[axis] >= n1:
                tang = [coords[m][1 - axis]]
                gin[s * q:(s + 1) * q] = g[_root_panel_slice(2, L, q, axis, side, tang)]
            else:
                nb_leaf = lookup[tuple(idx)]
                s2 = geo.SIDES_2D.index((axis, 1 - side))
                gin[s * q:(s + 1) * q] = -(QH @ u[nb_leaf])[s2 * q:(s2 + 1) * q]
        res2 = G @ u[m] - P_ @ gin
        sc2 = np.abs(G).sum(axis=1).max() * uscale + np.abs(gin).max()
        worst = max(worst, np.abs(res2).max() / sc2)
    return worst
