"""Adaptive 3D DtN HPS (Section 4.2): refinement criterion (Eq. refinement
check), level restriction, nonuniform merges and the downward pass.

Readings of points the paper leaves open:

* Refinement (Eq. refinement check): a leaf is sufficiently refined for f when
  max |f(x_1) - L_8f1 f(x_0)| / ||f||_inf < eps, with x_0 its p^3 Chebyshev
  nodes and x_1 the Chebyshev nodes of its 8 children.  ||f||_inf is the
  largest |f| over every point sampled so far: the tree is refined level by
  level, and before the leaves of level l are tested the norm is updated with
  all x_0 and x_1 samples of levels <= l.  Depths are clamped to
  [min_depth, max_depth]; the final tree is the union of the trees of all
  functions (a leaf is split when any function asks for it).
* Level restriction: face neighbours differ by at most one level; leaves
  with a face neighbour two or more levels finer are split until none is left.
* Nonuniform merge: every interface between two siblings is discretised on
  the coarser of the two panel sets at each place.  Where one side has four
  panels under one panel of the other side, its rows of T are projected onto
  the coarse panel (L2 projection onto Q_{q-1} by the fine panels' Gauss
  quadrature) and its columns take coarse data through interpolation (the
  coarse tensor Legendre interpolant evaluated at the fine Gauss nodes).
  Exterior panels are inherited unchanged.  The downward pass interpolates
  the coarse interface data back onto the fine panels.
* Node boundary order: faces -x, +x, -y, +y, -z, +z; each face lists its
  panels as the quadtree of the node's children in Morton order over the two
  tangential axes (a leaf face is one panel of q^2 points in tensor order,
  lower tangential axis fastest).  For a uniform tree this is the order of
  oracle.geometry.

Pins: tests/test_oracle_adaptive.py (projection exactness on Q_{q-1},
projection o interpolation = identity, polynomial exactness on 2:1 trees,
agreement with the brute-force composite solve on a two-level 2:1 tree,
agreement with the uniform oracle when the tree is uniform).
"""

from __future__ import annotations

from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import leaf as lf
from .spectral import cheb_points, gauss_legendre, interp_matrix

FACES = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]


def tangential(axis):
    return [k for k in range(3) if k != axis]


# ---------------------------------------------------------------------------
# trees
# ---------------------------------------------------------------------------

def morton_key(level, idx, max_level=30):
    """Sort key that orders leaves depth first with children in Morton order."""
    key = 0
    for lev in range(level):
        sh = level - 1 - lev
        c = ((idx[0] >> sh) & 1) | (((idx[1] >> sh) & 1) << 1) | (((idx[2] >> sh) & 1) << 2)
        key |= c << (3 * (max_level - 1 - lev))
    return key


def sort_leaves(leaves):
    return sorted(leaves, key=lambda lv: morton_key(lv[0], lv[1]))


def children_of(level, idx):
    return [(level + 1, (2 * idx[0] + (c & 1), 2 * idx[1] + ((c >> 1) & 1), 2 * idx[2] + (c >> 2)))
            for c in range(8)]


@lru_cache(maxsize=None)
def child_interp_1d(p):
    """p Chebyshev values on [-1, 1] -> values at the two children's Chebyshev
    nodes ([-1, 0] then [0, 1]): 2p x p."""
    x = cheb_points(p)
    xs = np.concatenate([0.5 * (x - 1.0), 0.5 * (x + 1.0)])
    return interp_matrix(x, xs)


def leaf_nodes(lo, hi, level, idx, p):
    lo = np.asarray(lo, float)
    h = (np.asarray(hi, float) - lo) / 2 ** level
    t = cheb_points(p, 0.0, 1.0)
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    loc = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    return lo + (np.asarray(idx) + loc) * h


def eight_child_nodes(lo, hi, level, idx, p):
    return np.concatenate([leaf_nodes(lo, hi, lv, ix, p) for lv, ix in children_of(level, idx)])


def L8f1_apply(p, f0):
    """Interpolate p^3 Chebyshev values (x fastest) of a leaf to the Chebyshev
    nodes of its 8 children (children in Morton order, x fastest inside)."""
    I = child_interp_1d(p)                      # 2p x p
    F = f0.reshape(p, p, p)                     # [z][y][x]
    G = np.einsum("ai,bj,ck,kji->abc", I, I, I, F)   # [x2][y2][z2]
    out = []
    for c in range(8):
        cx, cy, cz = c & 1, (c >> 1) & 1, c >> 2
        blk = G[cx * p:(cx + 1) * p, cy * p:(cy + 1) * p, cz * p:(cz + 1) * p]  # [x][y][z]
        out.append(np.transpose(blk, (2, 1, 0)).ravel())
    return np.concatenate(out)


def refine(funcs, lo, hi, p, eps, min_depth, max_depth):
    """Eq. "refinement check" applied level by level, union over funcs."""
    norms = np.zeros(len(funcs))
    final = []
    cand = [(min_depth, (i, j, k)) for i in range(2 ** min_depth)
            for j in range(2 ** min_depth) for k in range(2 ** min_depth)]
    while cand:
        lev = cand[0][0]
        if lev >= max_depth:
            final.extend(cand)
            break
        samples = []
        for (lv, idx) in cand:
            x0 = leaf_nodes(lo, hi, lv, idx, p)
            x1 = eight_child_nodes(lo, hi, lv, idx, p)
            vals = [(fn(x0), fn(x1)) for fn in funcs]
            samples.append(vals)
            for k, (v0, v1) in enumerate(vals):
                norms[k] = max(norms[k], np.abs(v0).max(), np.abs(v1).max())
        nxt = []
        for (lv, idx), vals in zip(cand, samples):
            split = False
            for k, (v0, v1) in enumerate(vals):
                if norms[k] == 0.0:
                    continue
                err = np.abs(v1 - L8f1_apply(p, v0)).max() / norms[k]
                if err >= eps:
                    split = True
            if split:
                nxt.extend(children_of(lv, idx))
            else:
                final.append((lv, idx))
        cand = nxt
    return sort_leaves(balance(final))


def _ancestors(level, idx):
    out = []
    for l2 in range(level - 1, -1, -1):
        sh = level - l2
        out.append((l2, tuple(i >> sh for i in idx)))
    return out


def balance(leaves):
    """Level restriction: split leaves that have a face neighbour two or more
    levels finer, until none is left."""
    leaves = set((lv, tuple(ix)) for lv, ix in leaves)
    while True:
        internal = set()
        for lv, ix in leaves:
            internal.update(_ancestors(lv, ix))
        to_split = set()
        for lv, ix in leaves:
            n1 = 2 ** lv
            for axis, side in FACES:
                nb = list(ix)
                nb[axis] += 1 if side else -1
                if nb[axis] < 0 or nb[axis] >= n1:
                    continue
                nb = tuple(nb)
                if (lv, nb) not in internal:
                    continue
                # neighbour cell is subdivided: any of its children touching the
                # shared face subdivided again means a leaf two levels finer
                for cl, cix in children_of(lv, nb):
                    touching = (cix[axis] & 1) == (0 if side else 1)
                    if touching and (cl, cix) in internal:
                        to_split.add((lv, ix))
        if not to_split:
            return sorted(leaves)
        for lv, ix in to_split:
            leaves.remove((lv, ix))
            leaves.update(children_of(lv, ix))


# ---------------------------------------------------------------------------
# 4 -> 1 panel projections
# ---------------------------------------------------------------------------

@lru_cache(maxsize=None)
def panel_projections(q):
    """(C2F, F2C): coarse q^2 Gauss data -> the 4 fine panels (Morton order
    over the tangential axes, tensor order inside) and back.  1D pieces on
    the coarse panel [0, 1] with fine halves [0, 1/2], [1/2, 1]."""
    xc, wc = gauss_legendre(q, 0.0, 1.0)
    xf = np.concatenate([gauss_legendre(q, 0.0, 0.5)[0], gauss_legendre(q, 0.5, 1.0)[0]])
    wf = np.concatenate([gauss_legendre(q, 0.0, 0.5)[1], gauss_legendre(q, 0.5, 1.0)[1]])
    c2f1 = interp_matrix(xc, xf)                     # 2q x q: coarse interpolant at fine nodes
    # L2 projection onto polynomials of degree < q, nodal at the coarse
    # Gauss points: value_i = (1 / wc_i) * sum_k wf_k l_i(xf_k) v_k
    f2c1 = (c2f1 * wf[:, None]).T / wc[:, None]       # q x 2q
    C2F = np.zeros((4 * q * q, q * q))
    F2C = np.zeros((q * q, 4 * q * q))
    for quad in range(4):
        a, b = quad & 1, quad >> 1
        A1 = c2f1[a * q:(a + 1) * q]                  # t1 half
        B1 = c2f1[b * q:(b + 1) * q]                  # t2 half
        C2F[quad * q * q:(quad + 1) * q * q] = np.kron(B1, A1)
        F2C[:, quad * q * q:(quad + 1) * q * q] = np.kron(f2c1[:, b * q:(b + 1) * q],
                                                         f2c1[:, a * q:(a + 1) * q])
    return C2F, F2C


# ---------------------------------------------------------------------------
# node boundaries: per face a list of panels (level, (t1, t2)) in order
# ---------------------------------------------------------------------------

@dataclass
class Node:
    level: int
    idx: tuple
    leaf_id: int = -1
    children: list = field(default_factory=list)
    faces: list = field(default_factory=list)    # 6 lists of panels (level, (i1, i2))


def build_tree(leaves):
    """Internal nodes over a sorted leaf list (complete octree)."""
    nodes = {}
    for n, (lv, ix) in enumerate(leaves):
        nodes[(lv, ix)] = Node(lv, ix, leaf_id=n)
    maxl = max(lv for lv, _ in leaves)
    for lev in range(maxl - 1, -1, -1):
        for key in list(nodes):
            lv, ix = key
            if lv != lev + 1:
                continue
            par = (lev, tuple(i >> 1 for i in ix))
            if par not in nodes:
                nodes[par] = Node(lev, par[1])
    for (lv, ix), nd in nodes.items():
        if nd.leaf_id < 0:
            nd.children = [nodes[c] for c in children_of(lv, ix)]
    root = nodes[(0, (0, 0, 0))]
    _set_faces(root)
    return root, nodes


def _set_faces(nd):
    if nd.leaf_id >= 0:
        nd.faces = []
        for axis, side in FACES:
            t1, t2 = tangential(axis)
            nd.faces.append([(nd.level, (nd.idx[t1], nd.idx[t2]))])
        return
    for ch in nd.children:
        _set_faces(ch)
    nd.faces = []
    for f, (axis, side) in enumerate(FACES):
        t1, t2 = tangential(axis)
        lst = []
        for quad in range(4):
            bits = [0, 0, 0]
            bits[axis] = side
            bits[t1] = quad & 1
            bits[t2] = quad >> 1
            c = bits[0] | (bits[1] << 1) | (bits[2] << 2)
            lst.extend(nd.children[c].faces[f])
        nd.faces.append(lst)


def coarse_interface(pa, pb, level, pos):
    """Coarse panel list of the interface square (level, pos) between two
    siblings, from the two sides' panel lists (each (level, (i1, i2)) in
    quadtree order).  Returns [(level, pos, kind_a, kind_b)] in quadtree
    order, kind 'same' (the side has exactly this panel) or 'fine' (the side
    has the four panels one level below)."""
    sa, sb = set(pa), set(pb)
    out = []

    def rec(lev, ps):
        ina, inb = (lev, ps) in sa, (lev, ps) in sb
        if ina or inb:
            ka = "same" if ina else "fine"
            kb = "same" if inb else "fine"
            for side_set, kind in ((sa, ka), (sb, kb)):
                if kind == "fine":
                    for quad in range(4):
                        sub = (lev + 1, (2 * ps[0] + (quad & 1), 2 * ps[1] + (quad >> 1)))
                        if sub not in side_set:
                            raise ValueError("interface is not 2:1 balanced")
            out.append((lev, ps, ka, kb))
            return
        for quad in range(4):
            rec(lev + 1, (2 * ps[0] + (quad & 1), 2 * ps[1] + (quad >> 1)))

    rec(level, pos)
    return out


def panel_points(lo, hi, q, axis, side, level, pos):
    """q^2 Gauss points of the face panel (tensor order, t1 fastest)."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    h = (hi - lo) / 2 ** level
    t1, t2 = tangential(axis)
    tg, _ = gauss_legendre(q, 0.0, 1.0)
    pts = np.zeros((q * q, 3))
    B, A = np.meshgrid(tg, tg, indexing="ij")
    pts[:, axis] = hi[axis] if side else lo[axis]
    pts[:, t1] = lo[t1] + (pos[0] + A.ravel()) * h[t1]
    pts[:, t2] = lo[t2] + (pos[1] + B.ravel()) * h[t2]
    return pts


def root_boundary_points(leaves, lo, hi, q):
    root, _ = build_tree(leaves)
    out = []
    for f, (axis, side) in enumerate(FACES):
        for lev, pos in root.faces[f]:
            out.append(panel_points(lo, hi, q, axis, side, lev, pos))
    return np.concatenate(out)


def all_leaf_nodes(leaves, lo, hi, p):
    return np.concatenate([leaf_nodes(lo, hi, lv, ix, p) for lv, ix in leaves])


# ---------------------------------------------------------------------------
# nonuniform merge (Section 4.2) and the adaptive solver
# ---------------------------------------------------------------------------

def _face_offsets(faces, q2):
    """Start of each panel of each face in the node's boundary vector."""
    offs, o = [], 0
    for f in range(6):
        d = {}
        for pn in faces[f]:
            d[pn] = o
            o += q2
        offs.append(d)
    return offs, o


def _merge_plan(nd, q):
    """Projection operators and scatter maps of one merge."""
    q2 = q * q
    C2F, F2C = panel_projections(q)
    kids = nd.children
    # interfaces: id = axis * 4 + (t1 bit + 2 t2 bit) of the low child
    iface = {}
    for axis in range(3):
        t1, t2 = tangential(axis)
        for c in range(8):
            if (c >> axis) & 1:
                continue
            ch = c | (1 << axis)
            lo_k, hi_k = kids[c], kids[ch]
            fa = 2 * axis + 1          # face (axis, +) of the low child
            fb = 2 * axis              # face (axis, -) of the high child
            lst = coarse_interface(lo_k.faces[fa], hi_k.faces[fb], lo_k.level,
                                   (lo_k.idx[t1], lo_k.idx[t2]))
            sid = axis * 4 + ((c >> t1) & 1) + 2 * ((c >> t2) & 1)
            iface[sid] = (c, ch, fa, fb, lst)
    var_off, nv = {}, 0
    for sid in sorted(iface):
        var_off[sid] = nv
        nv += len(iface[sid][4]) * q2
    poffs, n_ext = _face_offsets(nd.faces, q2)
    plans = []
    for c, kd in enumerate(kids):
        koffs, nk = _face_offsets(kd.faces, q2)
        rows_R, cols_R, vals_R = [], [], []
        rows_P, cols_P, vals_P = [], [], []
        ext_of, var_of = [], []
        npr = 0
        for f, (axis, side) in enumerate(FACES):
            if side == ((c >> axis) & 1):          # exterior face
                for pn in kd.faces[f]:
                    o = koffs[f][pn]
                    for t in range(q2):
                        rows_R.append(npr + t); cols_R.append(o + t); vals_R.append(1.0)
                        rows_P.append(o + t); cols_P.append(npr + t); vals_P.append(1.0)
                        ext_of.append(poffs[f][pn] + t)
                        var_of.append(-1)
                    npr += q2
                continue
            low = side == 1
            cc = c if low else c ^ (1 << axis)
            t1b = (cc >> tangential(axis)[0]) & 1
            t2b = (cc >> tangential(axis)[1]) & 1
            sid = axis * 4 + t1b + 2 * t2b
            _, _, _, _, lst = iface[sid]
            for k, (lev, pos, ka, kb) in enumerate(lst):
                kind = ka if low else kb
                vb = var_off[sid] + k * q2
                if kind == "same":
                    o = koffs[f][(lev, pos)]
                    for t in range(q2):
                        rows_R.append(npr + t); cols_R.append(o + t); vals_R.append(1.0)
                        rows_P.append(o + t); cols_P.append(npr + t); vals_P.append(1.0)
                else:
                    subs = [(lev + 1, (2 * pos[0] + (qd & 1), 2 * pos[1] + (qd >> 1))) for qd in range(4)]
                    for qd, sub in enumerate(subs):
                        o = koffs[f][sub]
                        for t in range(q2):
                            for u in range(q2):
                                rows_R.append(npr + u); cols_R.append(o + t)
                                vals_R.append(F2C[u, qd * q2 + t])
                                rows_P.append(o + t); cols_P.append(npr + u)
                                vals_P.append(C2F[qd * q2 + t, u])
                for t in range(q2):
                    ext_of.append(-1)
                    var_of.append(vb + t)
                npr += q2
        R = sp.csr_matrix((vals_R, (rows_R, cols_R)), shape=(npr, nk))
        Pc = sp.csr_matrix((vals_P, (rows_P, cols_P)), shape=(nk, npr))
        plans.append({"R": R, "Pc": Pc, "ext": np.array(ext_of), "var": np.array(var_of)})
    return plans, n_ext, nv


def merge_nonuniform(Ts, hs, plans, n_ext, n_int, want_T=True):
    """Eqs. "merge linear system" / "merge outputs 1-2" with the blocks of
    Appendix C.2 on the coarsened interfaces: D sums both sides of every
    interface, C / B / A are the children's interface-exterior, exterior-
    interface and exterior-exterior blocks."""
    dt = Ts[0].dtype
    A = np.zeros((n_ext, n_ext), dt)
    B = np.zeros((n_ext, n_int), dt)
    C = np.zeros((n_int, n_ext), dt)
    D = np.zeros((n_int, n_int), dt)
    h_ext = np.zeros(n_ext, dt)
    h_int = np.zeros(n_int, dt)
    for T, h, pl in zip(Ts, hs, plans):
        Tp = pl["R"] @ (pl["Pc"].T @ T.T).T          # R T Pc
        hp = pl["R"] @ h
        e = pl["ext"] >= 0
        i = ~e
        ee, vi = pl["ext"][e], pl["var"][i]
        A[np.ix_(ee, ee)] += Tp[np.ix_(e, e)]
        B[np.ix_(ee, vi)] += Tp[np.ix_(e, i)]
        C[np.ix_(vi, ee)] += Tp[np.ix_(i, e)]
        D[np.ix_(vi, vi)] += Tp[np.ix_(i, i)]
        h_ext[ee] += hp[e]
        h_int[vi] += hp[i]
    lu = sla.lu_factor(D)
    DinvC = sla.lu_solve(lu, C)
    Dinvh = sla.lu_solve(lu, h_int)
    S, gt = -DinvC, -Dinvh
    if not want_T:
        return None, None, S, gt
    return A - B @ DinvC, h_ext - B @ Dinvh, S, gt


@dataclass
class AdaptiveSolver:
    p: int
    leaves: list
    root: Node
    leaf_T: list
    leaf_h: list
    leaf_Y: list
    leaf_v: list
    merges: dict


def build_adaptive(leaves, p, lo, hi, a, b, c, f, want_root_T=False):
    """Leaf stage (Section 4.2: same local problems, per-leaf size) and the
    nonuniform merges, bottom-up."""
    q = p - 2
    leaves = sort_leaves(leaves)
    root, nodes = build_tree(leaves)
    side = float(hi[0] - lo[0])
    lT, lh, lY, lv = [], [], [], []
    for n, (lev, ix) in enumerate(leaves):
        hlen = side / 2 ** lev
        T, h, Y, v = lf.dtn_leaf(3, p, q, hlen, a[n], [bk[n] for bk in b], c[n], f[n])
        lT.append(T); lh.append(h); lY.append(Y); lv.append(v)
    merges = {}

    def up(nd):
        if nd.leaf_id >= 0:
            return lT[nd.leaf_id], lh[nd.leaf_id]
        Th = [up(ch) for ch in nd.children]
        plans, n_ext, n_int = _merge_plan(nd, q)
        is_root = nd.level == 0
        T, h, S, gt = merge_nonuniform([t for t, _ in Th], [hh for _, hh in Th], plans, n_ext, n_int,
                                       want_T=(not is_root) or want_root_T)
        merges[(nd.level, nd.idx)] = {"S": S, "gt": gt, "plans": plans}
        return T, h

    up(root)
    return AdaptiveSolver(p, leaves, root, lT, lh, lY, lv, merges)


def solve_adaptive(s: AdaptiveSolver, g):
    """Algorithm "down pass" with the projections undone by interpolation."""
    u = [None] * len(s.leaves)

    def down(nd, gN):
        if nd.leaf_id >= 0:
            u[nd.leaf_id] = s.leaf_Y[nd.leaf_id] @ gN + s.leaf_v[nd.leaf_id]
            return
        m = s.merges[(nd.level, nd.idx)]
        gint = m["S"] @ gN + m["gt"]
        for ch, pl in zip(nd.children, m["plans"]):
            e = pl["ext"] >= 0
            gp = np.zeros(len(pl["ext"]), dtype=np.result_type(gN, gint))
            gp[e] = gN[pl["ext"][e]]
            gp[~e] = gint[pl["var"][~e]]
            down(ch, pl["Pc"] @ gp)

    down(s.root, np.asarray(g))
    return np.array(u, dtype=object) if False else u


def sample_adaptive(problem, leaves, p):
    lo, hi = problem.lo, problem.hi
    x = all_leaf_nodes(leaves, lo, hi, p)
    nl, npl = len(leaves), p ** 3
    cf = problem.coeffs(x)
    a = cf["a"].reshape(nl, npl)
    b = [bk.reshape(nl, npl) for bk in cf["b"]]
    c = cf["c"].reshape(nl, npl)
    f = problem.source(x).reshape(nl, npl)
    xb = root_boundary_points(leaves, lo, hi, p - 2)
    g = problem.boundary(xb)
    return x, a, b, c, f, g
