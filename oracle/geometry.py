"""Tree geometry and point orderings used by the oracle (Section 3.1).

Conventions (the interface of the solver, fixed here and in include/hps.h):

* Leaves of a uniform tree of depth L are numbered depth first, children in
  Morton order c = cx + 2 cy (+ 4 cz), so leaf numbers are Morton codes with
  the coarsest level in the most significant bits.
* Inside a leaf, the p^d Chebyshev--Lobatto nodes are in tensor order, x
  fastest: node (ix, iy, iz) has index ix + p iy + p^2 iz.
* A node's boundary (leaf or merged) is ordered by sides S, E, N, W in 2D
  (y = min, x = max, y = max, x = min) and by faces -x, +x, -y, +y, -z, +z in
  3D.  A 2D side lists its Gauss points by increasing coordinate.  A 3D face
  is the quadtree of its leaf panels in Morton order over its two tangential
  axes (lower axis index = first Morton bit); inside one panel the q^2 Gauss
  points are in tensor order with the lower tangential axis fastest.
* Paper child labels: 2D a, b, c, d = SW, SE, NE, NW = Morton 0, 1, 3, 2
  (Fig. "2D merges"); 3D a-d = the lower layer counterclockwise from the
  origin corner and e-h the layer above them = Morton 0, 1, 3, 2, 4, 5, 7, 6
  (from the interface pairs of the 3D h_int vector, Appendix C.2).
"""

from __future__ import annotations

import numpy as np

from .spectral import cheb_points, gauss_legendre

LABELS_2D = "abcd"
MORTON_2D = {"a": 0, "b": 1, "c": 3, "d": 2}
LABELS_3D = "abcdefgh"
MORTON_3D = {"a": 0, "b": 1, "c": 3, "d": 2, "e": 4, "f": 5, "g": 7, "h": 6}

# 2D sides: (axis, 0 = min / 1 = max); 3D faces likewise.
SIDES_2D = [(1, 0), (0, 1), (1, 1), (0, 0)]            # S, E, N, W
FACES_3D = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]


def uniform_leaf_boxes(dim: int, lo, hi, L: int):
    """Lower corners and side lengths of the 2^(dL) leaves in Morton order."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    n1 = 2 ** L
    h = (hi - lo) / n1
    nl = n1 ** dim
    corners = np.zeros((nl, dim))
    for m in range(nl):
        idx = np.zeros(dim, int)
        for lev in range(L):
            c = (m >> (dim * (L - 1 - lev))) & ((1 << dim) - 1)
            for k in range(dim):
                idx[k] = idx[k] * 2 + ((c >> k) & 1)
        corners[m] = lo + idx * h
    return corners, h


def leaf_nodes(dim: int, lo, hi, L: int, p: int) -> np.ndarray:
    """Coordinates of all leaf Chebyshev nodes, shape (n_leaves * p^dim, dim)."""
    corners, h = uniform_leaf_boxes(dim, lo, hi, L)
    t = cheb_points(p, 0.0, 1.0)
    grids = np.meshgrid(*([t] * dim), indexing="ij")
    # tensor order x fastest: reverse the meshgrid axes
    loc = np.stack([grids[k].transpose(*range(dim)[::-1]).ravel() for k in range(dim)], axis=1)
    out = corners[:, None, :] + loc[None, :, :] * h[None, None, :]
    return out.reshape(-1, dim)


def _face_panel_order(level: int):
    """Morton order of the 4^level panels of a face: list of (i1, i2)."""
    out = []
    for m in range(4 ** level):
        i1 = i2 = 0
        for lev in range(level):
            c = (m >> (2 * (level - 1 - lev))) & 3
            i1 = i1 * 2 + (c & 1)
            i2 = i2 * 2 + (c >> 1)
        out.append((i1, i2))
    return out


def root_boundary_points(dim: int, lo, hi, L: int, q: int) -> np.ndarray:
    """Root boundary Gauss points of a uniform depth-L tree, canonical order."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    n1 = 2 ** L
    h = (hi - lo) / n1
    tg, _ = gauss_legendre(q, 0.0, 1.0)
    pts = []
    if dim == 2:
        for axis, side in SIDES_2D:
            tang = 1 - axis
            for i in range(n1):
                for t in tg:
                    x = np.zeros(2)
                    x[axis] = hi[axis] if side else lo[axis]
                    x[tang] = lo[tang] + (i + t) * h[tang]
                    pts.append(x)
    else:
        for axis, side in FACES_3D:
            t1, t2 = [k for k in range(3) if k != axis]
            for (i1, i2) in _face_panel_order(L):
                for b in tg:          # slow axis t2
                    for a in tg:      # fast axis t1
                        x = np.zeros(3)
                        x[axis] = hi[axis] if side else lo[axis]
                        x[t1] = lo[t1] + (i1 + a) * h[t1]
                        x[t2] = lo[t2] + (i2 + b) * h[t2]
                        pts.append(x)
    return np.array(pts)
