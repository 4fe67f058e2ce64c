"""O1: plain HPS build and solve on uniform trees (Sections 3.2-3.4).

build():  leaf stage for every leaf (Algorithm "local solve"), then the merge
          loop level by level (Algorithm "merge").
solve():  downward pass from the root to the leaves and the leaf output
          u = Y g + v (Algorithm "down pass").

Inputs are arrays sampled at the leaf nodes (leaf-major, Morton leaf order,
tensor node order x fastest) and root boundary data in the canonical order of
``oracle.geometry``.  Everything runs in float64 / complex128.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import geometry as geo
from . import leaf as lf
from . import merge as mg


@dataclass
class OracleSolver:
    dim: int
    kind: str
    p: int
    q: int
    L: int
    lo: tuple
    hi: tuple
    eta: float | None
    leaf_T: list = field(default_factory=list)
    leaf_h: list = field(default_factory=list)
    leaf_Y: list = field(default_factory=list)
    leaf_v: list = field(default_factory=list)
    # levels[l] = list over nodes at tree level l (0 = root) of dicts
    levels: dict = field(default_factory=dict)

    @property
    def n_leaves(self):
        return 2 ** (self.dim * self.L)


def _labels(dim):
    return (geo.LABELS_2D, geo.MORTON_2D) if dim == 2 else (geo.LABELS_3D, geo.MORTON_3D)


def build(dim, kind, p, q, L, lo, hi, a, b, c, f, eta=None, iti_direct=False,
          want_root_T=True) -> OracleSolver:
    """a, c, f: arrays (n_leaves, p^dim); b: list of dim such arrays."""
    if q != p - 2:
        raise ValueError("the paper's choice q = p - 2 is required")
    if kind == "iti" and dim != 2:
        raise ValueError("ItI is defined for 2D only")
    s = OracleSolver(dim=dim, kind=kind, p=p, q=q, L=L, lo=tuple(lo), hi=tuple(hi), eta=eta)
    corners, hvec = geo.uniform_leaf_boxes(dim, lo, hi, L)
    hlen = float(hvec[0])
    if not np.allclose(hvec, hlen):
        raise ValueError("leaves must be cubes (equal side lengths)")
    nl = s.n_leaves
    for i in range(nl):
        bi = [bk[i] for bk in b]
        if kind == "dtn":
            T, h, Y, v = lf.dtn_leaf(dim, p, q, hlen, a[i], bi, c[i], f[i])
        else:
            T, h, Y, v = lf.iti_leaf(p, q, hlen, a[i], bi, c[i], f[i], eta)
        s.leaf_T.append(T)
        s.leaf_h.append(h)
        s.leaf_Y.append(Y)
        s.leaf_v.append(v)
    labels, morton = _labels(dim)
    nch = 2 ** dim
    cur_T, cur_h = s.leaf_T, s.leaf_h
    for lev in range(L - 1, -1, -1):
        nodes = []
        new_T, new_h = [], []
        for j in range(nch ** lev):
            Ts = {lab: cur_T[nch * j + morton[lab]] for lab in labels}
            hs = {lab: cur_h[nch * j + morton[lab]] for lab in labels}
            if dim == 2 and kind == "dtn":
                T, h, S, gt, perm = mg.merge_2d_dtn(Ts, hs)
            elif dim == 2:
                T, h, S, gt, perm = mg.merge_2d_iti(Ts, hs, iti_direct=iti_direct)
            else:
                T, h, S, gt, perm = mg.merge_3d_dtn(Ts, hs, want_T=(lev > 0 or want_root_T))
            nodes.append({"S": S, "gt": gt, "perm": perm, "T": T, "h": h})
            new_T.append(T)
            new_h.append(h)
        s.levels[lev] = nodes
        cur_T, cur_h = new_T, new_h
    return s


def solve(s: OracleSolver, g: np.ndarray) -> np.ndarray:
    """Downward pass and leaf output.  Returns u with shape (n_leaves, p^dim)."""
    labels, morton = _labels(s.dim)
    nch = 2 ** s.dim
    gs = [np.asarray(g)]
    for lev in range(0, s.L):
        nxt = [None] * (nch ** (lev + 1))
        for j, node in enumerate(s.levels[lev]):
            if s.dim == 2 and s.kind == "dtn":
                kids = mg.children_g_2d_dtn(gs[j], node["S"], node["gt"], node["perm"])
            elif s.dim == 2:
                kids = mg.children_g_2d_iti(gs[j], node["S"], node["gt"], node["perm"])
            else:
                kids = mg.children_g_3d_dtn(gs[j], node["S"], node["gt"], node["perm"])
            for lab in labels:
                nxt[nch * j + morton[lab]] = kids[lab]
        gs = nxt
    u = [s.leaf_Y[i] @ gs[i] + s.leaf_v[i] for i in range(s.n_leaves)]
    return np.array(u)


def leaf_boundary_data(s: OracleSolver, g: np.ndarray):
    """The incoming boundary data of every leaf after the downward pass
    (used by tests that check interface consistency)."""
    labels, morton = _labels(s.dim)
    nch = 2 ** s.dim
    gs = [np.asarray(g)]
    for lev in range(0, s.L):
        nxt = [None] * (nch ** (lev + 1))
        for j, node in enumerate(s.levels[lev]):
            fn = {(2, "dtn"): mg.children_g_2d_dtn, (2, "iti"): mg.children_g_2d_iti,
                  (3, "dtn"): mg.children_g_3d_dtn}[(s.dim, s.kind)]
            kids = fn(gs[j], node["S"], node["gt"], node["perm"])
            for lab in labels:
                nxt[nch * j + morton[lab]] = kids[lab]
        gs = nxt
    return gs


def sample_problem(problem, p, q, L):
    """Sample a workloads.Problem on the oracle's own nodes.  Returns the leaf
    arrays a, b, c, f and the root boundary data g."""
    dim = problem.dim
    x = geo.leaf_nodes(dim, problem.lo, problem.hi, L, p)
    nl = 2 ** (dim * L)
    npl = p ** dim
    cf = problem.coeffs(x)
    a = cf["a"].reshape(nl, npl)
    b = [bk.reshape(nl, npl) for bk in cf["b"]]
    c = cf["c"].reshape(nl, npl)
    f = problem.source(x).reshape(nl, npl)
    xb = geo.root_boundary_points(dim, problem.lo, problem.hi, L, q)
    g = problem.boundary(xb)
    return x, a, b, c, f, g


def solve_problem(problem, p, L, **kw):
    """Build and solve ``problem`` at order p, depth L.  Returns (x, u)."""
    q = p - 2
    x, a, b, c, f, g = sample_problem(problem, p, q, L)
    s = build(problem.dim, problem.kind, p, q, L, problem.lo, problem.hi, a, b, c, f,
              eta=problem.eta, **kw)
    return x, solve(s, g).reshape(-1)
