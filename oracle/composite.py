"""O2: brute-force dense solve of the composite collocation system.

HPS eliminates a composite spectral collocation system exactly (up to
rounding): the leaf equations of Section 3.2 together with the interface
conditions used by the merges (Appendix A.2: the outward normal derivatives
of neighbouring leaves sum to zero; Appendix B.2: the incoming impedance of
one leaf is minus the outgoing impedance of its neighbour).  This module
writes that system out for a whole uniform tree and solves it with one dense
LU, with no merge recursion and no block formulas, so it is an independent
check of O1 on small trees.

DtN unknowns: every leaf's interior Chebyshev values and the Gauss values on
every interior leaf side (face).  Equations per leaf:
    L_ii u_i + L_ie P g_leaf = f_i,
and per interior panel (leaves alpha, beta on either side):
    (Q u^alpha)_panel + (Q u^beta)_panel = 0,  u = [P g_leaf on I_e; u_i on I_i].

ItI unknowns: every leaf's full p^2 values.  Equations per leaf:
    L(I_i, :) u = f_i,   G u = P g_in,
with g_in = root data on boundary panels and g_in = -(Q H u^beta)_panel on a
panel shared with leaf beta.
"""

from __future__ import annotations

import numpy as np

from . import geometry as geo
from . import leaf as lf


def _leaf_panels(dim, L):
    """For each leaf (Morton order) and each side/face slot, either
    ('root', position in the canonical root boundary) or
    ('int', panel id, orientation) with a shared interior panel id."""
    n1 = 2 ** L
    nl = n1 ** dim
    corners = []
    for m in range(nl):
        idx = [0] * dim
        for lev in range(L):
            c = (m >> (dim * (L - 1 - lev))) & ((1 << dim) - 1)
            for k in range(dim):
                idx[k] = idx[k] * 2 + ((c >> k) & 1)
        corners.append(tuple(idx))
    slots = geo.SIDES_2D if dim == 2 else geo.FACES_3D
    # canonical root panel positions
    root_pos = {}
    if dim == 2:
        for s, (axis, side) in enumerate(geo.SIDES_2D):
            for i in range(n1):
                root_pos[(axis, side, (i,))] = s * n1 + i
    else:
        order = geo._face_panel_order(L)
        for s, (axis, side) in enumerate(geo.FACES_3D):
            for k, (i1, i2) in enumerate(order):
                root_pos[(axis, side, (i1, i2))] = s * len(order) + k
    panel_ids = {}
    out = []
    for m, idx in enumerate(corners):
        row = []
        for axis, side in slots:
            tang = tuple(idx[k] for k in range(dim) if k != axis)
            on_root = (idx[axis] == 0 and side == 0) or (idx[axis] == n1 - 1 and side == 1)
            if on_root:
                row.append(("root", root_pos[(axis, side, tang)]))
            else:
                plane = idx[axis] + side        # index of the grid plane
                key = (axis, plane, tang)
                if key not in panel_ids:
                    panel_ids[key] = len(panel_ids)
                row.append(("int", panel_ids[key]))
        out.append(row)
    return out, len(panel_ids)


def solve_dtn(dim, p, L, lo, hi, a, b, c, f, g):
    A, rhs, unpack = assemble_dtn(dim, p, L, lo, hi, a, b, c, f, g)
    return unpack(np.linalg.solve(A, rhs), g)


def assemble_dtn(dim, p, L, lo, hi, a, b, c, f, g):
    """The composite DtN system (A, rhs) and unpack(sol, g) -> u on the leaf
    nodes ([n_leaves][p^dim])."""
    q = p - 2
    corners, hvec = geo.uniform_leaf_boxes(dim, lo, hi, L)
    hlen = float(hvec[0])
    ops = lf.reference_ops(dim, p, q)
    Ie, Ii = ops["Ie"], ops["Ii"]
    P, Q = lf.dtn_P_Q(dim, p, q, hlen)
    npan = q ** (dim - 1)
    nslot = 2 * dim
    panels, nint = _leaf_panels(dim, L)
    nl = len(panels)
    ni = len(Ii)
    N = nl * ni + nint * npan
    dt = np.result_type(f, g, float)
    A = np.zeros((N, N), dt)
    rhs = np.zeros(N, dt)
    off_g = nl * ni

    def gcols(slot_entry):
        kind, k = slot_entry
        return kind, k

    for m in range(nl):
        Lm = lf.assemble_L(dim, p, hlen, a[m], [bk[m] for bk in b], c[m])
        Lii = Lm[np.ix_(Ii, Ii)]
        LieP = Lm[np.ix_(Ii, Ie)] @ P
        r0 = m * ni
        A[r0:r0 + ni, r0:r0 + ni] = Lii
        rhs[r0:r0 + ni] = f[m][Ii]
        for s, ent in enumerate(panels[m]):
            blk = LieP[:, s * npan:(s + 1) * npan]
            kind, k = gcols(ent)
            if kind == "root":
                rhs[r0:r0 + ni] -= blk @ g[k * npan:(k + 1) * npan]
            else:
                A[r0:r0 + ni, off_g + k * npan:off_g + (k + 1) * npan] += blk
    # flux balance rows, one block per interior panel (sum over its 2 leaves)
    QP = Q[:, Ie] @ P              # boundary-data part of Q u
    QI = Q[:, Ii]                  # interior part of Q u
    for m in range(nl):
        for s, ent in enumerate(panels[m]):
            kind, k = ent
            if kind != "int":
                continue
            rows = slice(off_g + k * npan, off_g + (k + 1) * npan)
            srows = slice(s * npan, (s + 1) * npan)
            A[rows, m * ni:(m + 1) * ni] += QI[srows, :]
            for s2, ent2 in enumerate(panels[m]):
                blk = QP[srows, s2 * npan:(s2 + 1) * npan]
                if ent2[0] == "root":
                    rhs[rows] -= blk @ g[ent2[1] * npan:(ent2[1] + 1) * npan]
                else:
                    k2 = ent2[1]
                    A[rows, off_g + k2 * npan:off_g + (k2 + 1) * npan] += blk

    def unpack(sol, g):
        dt2 = np.result_type(sol, g)
        u = np.zeros((nl, p ** dim), dt2)
        for m in range(nl):
            gl = np.zeros(nslot * npan, dt2)
            for s, (kind, k) in enumerate(panels[m]):
                src = g if kind == "root" else sol[off_g:]
                gl[s * npan:(s + 1) * npan] = src[k * npan:(k + 1) * npan]
            u[m, Ie] = P @ gl
            u[m, Ii] = sol[m * ni:(m + 1) * ni]
        return u

    unpack.info = {"panels": panels, "off_g": off_g, "ni": ni, "npan": npan, "Ie": Ie, "Ii": Ii, "P": P,
                   "nl": nl, "npts": p ** dim}
    return A, rhs, unpack


def solve_iti(p, L, lo, hi, a, b, c, f, g, eta):
    A, rhs = assemble_iti(p, L, lo, hi, a, b, c, f, g, eta)
    nl = (2 ** L) ** 2
    return np.linalg.solve(A, rhs).reshape(nl, p * p)


def assemble_iti(p, L, lo, hi, a, b, c, f, g, eta):
    """The composite ItI system (A, rhs); the solution is u on the leaf nodes
    ([n_leaves][p^2]) flattened."""
    dim = 2
    q = p - 2
    corners, hvec = geo.uniform_leaf_boxes(dim, lo, hi, L)
    hlen = float(hvec[0])
    ops = lf.reference_ops(dim, p, q)
    Ii = ops["Ii"]
    P, G, H, Qb = lf.iti_ops(p, q, hlen, eta)
    QH = Qb @ H
    panels, _ = _leaf_panels(dim, L)
    nl = len(panels)
    npl = p * p
    nown = G.shape[0]
    N = nl * npl
    A = np.zeros((N, N), complex)
    rhs = np.zeros(N, complex)
    # neighbour lookup for interior panels
    owners = {}
    for m in range(nl):
        for s, (kind, k) in enumerate(panels[m]):
            if kind == "int":
                owners.setdefault(k, []).append((m, s))
    for m in range(nl):
        Lm = lf.assemble_L(dim, p, hlen, a[m], [bk[m] for bk in b], c[m])
        r0 = m * npl
        cols = slice(m * npl, (m + 1) * npl)
        A[r0:r0 + nown, cols] = G
        A[r0 + nown:r0 + npl, cols] = Lm[Ii, :]
        rhs[r0 + nown:r0 + npl] = f[m][Ii]
        for s, (kind, k) in enumerate(panels[m]):
            Ps = P[:, s * q:(s + 1) * q]
            if kind == "root":
                rhs[r0:r0 + nown] += Ps @ g[k * q:(k + 1) * q]
            else:
                (mb, sb), = [o for o in owners[k] if o[0] != m]
                # G u^m = P_s g_in,  g_in = -(QH u^mb) on the neighbour's slot sb
                A[r0:r0 + nown, mb * npl:(mb + 1) * npl] += Ps @ QH[sb * q:(sb + 1) * q, :]
    return A, rhs


def solve_dtn_adaptive(leaves, p, lo, hi, a, b, c, f, g):
    """O2 on an adaptive 2:1 octree (Section 4.2 discretisation): the
    composite system with interface unknowns on the coarser panel of every
    leaf-leaf interface.  A fine leaf takes its face data from the coarse
    panel by interpolation; the flux balance on a coarse panel adds the
    coarse side's normal derivative and the L2 projection of the four fine
    sides' normal derivatives."""
    from . import adaptive as ad
    q = p - 2
    q2 = q * q
    leaves = ad.sort_leaves(leaves)
    C2F, F2C = ad.panel_projections(q)
    side_len = float(hi[0] - lo[0])
    ops = lf.reference_ops(3, p, q)
    Ie, Ii = ops["Ie"], ops["Ii"]
    ni = len(Ii)
    leafset = {(lv, tuple(ix)): n for n, (lv, ix) in enumerate(leaves)}
    internal = set()
    for lv, ix in leaves:
        internal.update(ad._ancestors(lv, ix))
    root, _ = ad.build_tree(leaves)
    root_off, o = {}, 0
    for fi in range(6):
        for pn in root.faces[fi]:
            root_off[(fi, pn)] = o
            o += q2
    # classify every leaf face: ('root', off) | ('panel', key) | ('coarse', key, quadrant)
    faces_of = []
    panel_ids = {}
    for lv, ix in leaves:
        row = []
        n1 = 2 ** lv
        for fi, (axis, sd) in enumerate(ad.FACES):
            t1, t2 = ad.tangential(axis)
            pos = (ix[t1], ix[t2])
            nb = list(ix)
            nb[axis] += 1 if sd else -1
            if nb[axis] < 0 or nb[axis] >= n1:
                row.append(("root", root_off[(fi, (lv, pos))]))
                continue
            nb = tuple(nb)
            plane = ix[axis] + sd
            if (lv, nb) in leafset or (lv, nb) in internal:
                key = (lv, axis, plane, pos)
                panel_ids.setdefault(key, len(panel_ids))
                row.append(("panel", key))
            else:
                # the neighbour is a coarser leaf: use its face panel
                key = (lv - 1, axis, plane // 2, (pos[0] // 2, pos[1] // 2))
                panel_ids.setdefault(key, len(panel_ids))
                quad = (pos[0] & 1) + 2 * (pos[1] & 1)
                row.append(("coarse", key, quad))
        faces_of.append(row)
    nl = len(leaves)
    npan = len(panel_ids)
    N = nl * ni + npan * q2
    dt = np.result_type(f, g, float)
    A = np.zeros((N, N), dt)
    rhs = np.zeros(N, dt)
    og = nl * ni

    def gmap(ent):
        """(columns into the unknown vector, matrix) so that g_face = M x[cols],
        or the root data."""
        if ent[0] == "root":
            return None, g[ent[1]:ent[1] + q2]
        pid = panel_ids[ent[1]]
        cols = np.arange(og + pid * q2, og + (pid + 1) * q2)
        if ent[0] == "panel":
            return cols, np.eye(q2)
        return cols, C2F[ent[2] * q2:(ent[2] + 1) * q2]

    for n, (lv, ix) in enumerate(leaves):
        hlen = side_len / 2 ** lv
        P_, Q = lf.dtn_P_Q(3, p, q, hlen)
        Lm = lf.assemble_L(3, p, hlen, a[n], [bk[n] for bk in b], c[n])
        LieP = Lm[np.ix_(Ii, Ie)] @ P_
        r0 = n * ni
        A[r0:r0 + ni, r0:r0 + ni] = Lm[np.ix_(Ii, Ii)]
        rhs[r0:r0 + ni] = f[n][Ii]
        QP = Q[:, Ie] @ P_
        QI = Q[:, Ii]
        for fi, ent in enumerate(faces_of[n]):
            cols, M = gmap(ent)
            blk = LieP[:, fi * q2:(fi + 1) * q2]
            if cols is None:
                rhs[r0:r0 + ni] -= blk @ M
            else:
                A[r0:r0 + ni, cols] += blk @ M
        # flux rows: this leaf's normal derivative on every non-root face
        for fi, ent in enumerate(faces_of[n]):
            if ent[0] == "root":
                continue
            pid = panel_ids[ent[1]]
            rows = slice(og + pid * q2, og + (pid + 1) * q2)
            Wr = np.eye(q2) if ent[0] == "panel" else F2C[:, ent[2] * q2:(ent[2] + 1) * q2]
            A[rows, r0:r0 + ni] += Wr @ QI[fi * q2:(fi + 1) * q2]
            for fj, ent2 in enumerate(faces_of[n]):
                cols, M = gmap(ent2)
                blk = Wr @ QP[fi * q2:(fi + 1) * q2, fj * q2:(fj + 1) * q2]
                if cols is None:
                    rhs[rows] -= blk @ M
                else:
                    A[rows, cols] += blk @ M
    sol = np.linalg.solve(A, rhs)
    u = np.zeros((nl, p ** 3), dt)
    for n in range(nl):
        P_, _ = lf.dtn_P_Q(3, p, q, side_len / 2 ** leaves[n][0])
        gl = np.zeros(6 * q2, dt)
        for fi, ent in enumerate(faces_of[n]):
            cols, M = gmap(ent)
            gl[fi * q2:(fi + 1) * q2] = M if cols is None else M @ sol[cols]
        u[n, Ie] = P_ @ gl
        u[n, Ii] = sol[n * ni:(n + 1) * ni]
    return u
