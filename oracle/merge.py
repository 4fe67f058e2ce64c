"""Merge stage of the oracle (Section 3.3, Algorithm "merge", Eqs. merge
linear system / merge outputs 1-2) with the block formulas of Appendix A.2
(2D DtN), B.2 (2D ItI) and C.2 (3D DtN).

Every merged node returns its T and h in the canonical boundary order of
``oracle.geometry`` (sides S, E, N, W / faces -x..+z).  Internally the merge
works in the paper's section order; ``S`` maps section-ordered exterior data
to the interior unknowns, and the permutation between the two orders is kept
with the node so the downward pass can undo it.

Readings:
* Section k (exterior) lists child k's exterior sides (faces) in the
  canonical side (face) order; an interior section lists the shared side in
  its canonical point order (the same on both children).
* ItI interface rows use the matrix form of Appendix B.2 (the expanded
  scalar equation there is garbled): the equation of g^(a)_5 is
  0 = g^(a)_5 + T^(b)_{5,2} g_2 + T^(b)_{5,5} g^(b)_5 + T^(b)_{5,6} g^(b)_6 + h^(b)_5.
* D^{-1} for ItI is formed through W = I - D12 D21 (Eq. ItI D inverse); a
  direct LU solve with D is available as a cross-check (``iti_direct``).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

# ---------------------------------------------------------------------------
# 2D: sides of a child, indices into its [S, E, N, W] boundary vector
# ---------------------------------------------------------------------------
_S, _E, _N, _W = 0, 1, 2, 3

# section -> list of (side) per child label, in the order they are stacked
_SEC2D = {
    "a": {1: [_S, _W], 5: [_E], 8: [_N]},
    "b": {2: [_S, _E], 5: [_W], 6: [_N]},
    "c": {3: [_E, _N], 6: [_S], 7: [_W]},
    "d": {4: [_N, _W], 7: [_E], 8: [_S]},
}
# canonical parent boundary: (child, side) blocks for S, E, N, W
_CANON2D = [("a", _S), ("b", _S), ("b", _E), ("c", _E),
            ("d", _N), ("c", _N), ("a", _W), ("d", _W)]
_EXTSEC2D = [("a", _S), ("a", _W), ("b", _S), ("b", _E),
             ("c", _E), ("c", _N), ("d", _N), ("d", _W)]


def _sub2d(T, n, rows, cols):
    r = np.concatenate([np.arange(s * n, (s + 1) * n) for s in rows])
    c = np.concatenate([np.arange(s * n, (s + 1) * n) for s in cols])
    return T[np.ix_(r, c)]


def _vec2d(h, n, rows):
    r = np.concatenate([np.arange(s * n, (s + 1) * n) for s in rows])
    return h[r]


def canon_perm_2d(n):
    """perm such that T_canon = T_sec[perm][:, perm]."""
    pos = {blk: i for i, blk in enumerate(_EXTSEC2D)}
    return np.concatenate([np.arange(pos[b] * n, (pos[b] + 1) * n) for b in _CANON2D])


def merge_2d_dtn(Ts, hs):
    """Appendix A.2.  Ts, hs: dicts over labels a..d of the children's
    canonical T (4n x 4n) and h (4n).  Returns T, h (canonical), S, gt and the
    canonical permutation."""
    n = Ts["a"].shape[0] // 4

    def t(ch, i, j):
        return _sub2d(Ts[ch], n, _SEC2D[ch][i], _SEC2D[ch][j])

    def hv(ch, i):
        return _vec2d(hs[ch], n, _SEC2D[ch][i])

    Z = lambda r, c: np.zeros((r, c), dtype=Ts["a"].dtype)  # noqa: E731
    n2 = 2 * n
    A = sla.block_diag(t("a", 1, 1), t("b", 2, 2), t("c", 3, 3), t("d", 4, 4))
    B = np.block([
        [t("a", 1, 5), Z(n2, n), Z(n2, n), t("a", 1, 8)],
        [t("b", 2, 5), t("b", 2, 6), Z(n2, n), Z(n2, n)],
        [Z(n2, n), t("c", 3, 6), t("c", 3, 7), Z(n2, n)],
        [Z(n2, n), Z(n2, n), t("d", 4, 7), t("d", 4, 8)],
    ])
    C = np.block([
        [t("a", 5, 1), t("b", 5, 2), Z(n, n2), Z(n, n2)],
        [Z(n, n2), t("b", 6, 2), t("c", 6, 3), Z(n, n2)],
        [Z(n, n2), Z(n, n2), t("c", 7, 3), t("d", 7, 4)],
        [t("a", 8, 1), Z(n, n2), Z(n, n2), t("d", 8, 4)],
    ])
    D = np.block([
        [t("a", 5, 5) + t("b", 5, 5), t("b", 5, 6), Z(n, n), t("a", 5, 8)],
        [t("b", 6, 5), t("b", 6, 6) + t("c", 6, 6), t("c", 6, 7), Z(n, n)],
        [Z(n, n), t("c", 7, 6), t("c", 7, 7) + t("d", 7, 7), t("d", 7, 8)],
        [t("a", 8, 5), Z(n, n), t("d", 8, 7), t("d", 8, 8) + t("a", 8, 8)],
    ])
    h_ext = np.concatenate([hv("a", 1), hv("b", 2), hv("c", 3), hv("d", 4)])
    h_int = np.concatenate([hv("a", 5) + hv("b", 5), hv("b", 6) + hv("c", 6),
                            hv("c", 7) + hv("d", 7), hv("d", 8) + hv("a", 8)])
    lu = sla.lu_factor(D)
    DinvC = sla.lu_solve(lu, C)
    Dinvh = sla.lu_solve(lu, h_int)
    T = A - B @ DinvC
    h = h_ext - B @ Dinvh
    S = -DinvC
    gt = -Dinvh
    perm = canon_perm_2d(n)
    return T[np.ix_(perm, perm)], h[perm], S, gt, perm


def children_g_2d_dtn(g_canon, S, gt, perm):
    """Downward step (Algorithm "down pass") for a 2D DtN node: returns the
    children's canonical boundary data."""
    n = len(g_canon) // 8
    g_sec = np.empty_like(g_canon)
    g_sec[perm] = g_canon
    gi = S @ g_sec + gt
    blk = lambda v, k: v[k * n:(k + 1) * n]  # noqa: E731
    ext = {b: blk(g_sec, i) for i, b in enumerate(_EXTSEC2D)}
    g5, g6, g7, g8 = (blk(gi, k) for k in range(4))
    return {
        "a": np.concatenate([ext[("a", _S)], g5, g8, ext[("a", _W)]]),
        "b": np.concatenate([ext[("b", _S)], ext[("b", _E)], g6, g5]),
        "c": np.concatenate([g6, ext[("c", _E)], ext[("c", _N)], g7]),
        "d": np.concatenate([g8, g7, ext[("d", _N)], ext[("d", _W)]]),
    }


def merge_2d_iti(Ts, hs, iti_direct=False):
    """Appendix B.2.  g_int = [g5a, g8a, g6c, g7c, g5b, g6b, g7d, g8d]."""
    n = Ts["a"].shape[0] // 4

    def t(ch, i, j):
        return _sub2d(Ts[ch], n, _SEC2D[ch][i], _SEC2D[ch][j])

    def hv(ch, i):
        return _vec2d(hs[ch], n, _SEC2D[ch][i])

    Z = lambda r, c: np.zeros((r, c), dtype=complex)  # noqa: E731
    n2 = 2 * n
    A = sla.block_diag(t("a", 1, 1), t("b", 2, 2), t("c", 3, 3), t("d", 4, 4))
    z2 = Z(n2, n)
    B = np.block([
        [t("a", 1, 5), t("a", 1, 8), z2, z2, z2, z2, z2, z2],
        [z2, z2, z2, z2, t("b", 2, 5), t("b", 2, 6), z2, z2],
        [z2, z2, t("c", 3, 6), t("c", 3, 7), z2, z2, z2, z2],
        [z2, z2, z2, z2, z2, z2, t("d", 4, 7), t("d", 4, 8)],
    ])
    zc = Z(n, n2)
    C = np.block([
        [zc, t("b", 5, 2), zc, zc],
        [zc, zc, zc, t("d", 8, 4)],
        [zc, t("b", 6, 2), zc, zc],
        [zc, zc, zc, t("d", 7, 4)],
        [t("a", 5, 1), zc, zc, zc],
        [zc, zc, t("c", 6, 3), zc],
        [zc, zc, t("c", 7, 3), zc],
        [t("a", 8, 1), zc, zc, zc],
    ])
    z = Z(n, n)
    M = np.block([
        [z, z, z, z, t("b", 5, 5), t("b", 5, 6), z, z],
        [z, z, z, z, z, z, t("d", 8, 7), t("d", 8, 8)],
        [z, z, z, z, t("b", 6, 5), t("b", 6, 6), z, z],
        [z, z, z, z, z, z, t("d", 7, 7), t("d", 7, 8)],
        [t("a", 5, 5), t("a", 5, 8), z, z, z, z, z, z],
        [z, z, t("c", 6, 6), t("c", 6, 7), z, z, z, z],
        [z, z, t("c", 7, 6), t("c", 7, 7), z, z, z, z],
        [t("a", 8, 5), t("a", 8, 8), z, z, z, z, z, z],
    ])
    D = np.eye(8 * n) + M
    h_ext = np.concatenate([hv("a", 1), hv("b", 2), hv("c", 3), hv("d", 4)])
    h_int = np.concatenate([hv("b", 5), hv("d", 8), hv("b", 6), hv("d", 7),
                            hv("a", 5), hv("c", 6), hv("c", 7), hv("a", 8)])
    R = np.concatenate([C, h_int[:, None]], axis=1)
    if iti_direct:
        X = np.linalg.solve(D, R)
    else:
        m = 4 * n
        D12 = D[:m, m:]
        D21 = D[m:, :m]
        W = np.eye(m) - D12 @ D21
        luW = sla.lu_factor(W)
        Winv = lambda Y: sla.lu_solve(luW, Y)  # noqa: E731
        # D^{-1} = [[W^-1, -W^-1 D12], [-D21 W^-1, I + D21 W^-1 D12]]
        R1, R2 = R[:m], R[m:]
        X1 = Winv(R1) - Winv(D12 @ R2)
        X2 = -D21 @ Winv(R1) + R2 + D21 @ Winv(D12 @ R2)
        X = np.concatenate([X1, X2], axis=0)
    DinvC, Dinvh = X[:, :-1], X[:, -1]
    T = A - B @ DinvC
    h = h_ext - B @ Dinvh
    S = -DinvC
    gt = -Dinvh
    perm = canon_perm_2d(n)
    return T[np.ix_(perm, perm)], h[perm], S, gt, perm


def children_g_2d_iti(g_canon, S, gt, perm):
    n = len(g_canon) // 8
    g_sec = np.empty_like(g_canon)
    g_sec[perm] = g_canon
    gi = S @ g_sec + gt
    blk = lambda v, k: v[k * n:(k + 1) * n]  # noqa: E731
    ext = {b: blk(g_sec, i) for i, b in enumerate(_EXTSEC2D)}
    g5a, g8a, g6c, g7c, g5b, g6b, g7d, g8d = (blk(gi, k) for k in range(8))
    return {
        "a": np.concatenate([ext[("a", _S)], g5a, g8a, ext[("a", _W)]]),
        "b": np.concatenate([ext[("b", _S)], ext[("b", _E)], g6b, g5b]),
        "c": np.concatenate([g6c, ext[("c", _E)], ext[("c", _N)], g7c]),
        "d": np.concatenate([g8d, g7d, ext[("d", _N)], ext[("d", _W)]]),
    }


# ---------------------------------------------------------------------------
# 3D (Appendix C.2): faces 0..5 = -x, +x, -y, +y, -z, +z
# ---------------------------------------------------------------------------
_FACE_SEC3D = {
    "a": {0: 1, 1: 9, 2: 1, 3: 12, 4: 1, 5: 17},
    "b": {0: 9, 1: 2, 2: 2, 3: 10, 4: 2, 5: 18},
    "c": {0: 11, 1: 3, 2: 10, 3: 3, 4: 3, 5: 19},
    "d": {0: 4, 1: 11, 2: 12, 3: 4, 4: 4, 5: 20},
    "e": {0: 5, 1: 13, 2: 5, 3: 16, 4: 17, 5: 5},
    "f": {0: 13, 1: 6, 2: 6, 3: 14, 4: 18, 5: 6},
    "g": {0: 15, 1: 7, 2: 14, 3: 7, 4: 19, 5: 7},
    "h": {0: 8, 1: 15, 2: 16, 3: 8, 4: 20, 5: 8},
}
_CHILD_OF_EXT = {k + 1: ch for k, ch in enumerate("abcdefgh")}
# interior section -> the two children that share it (paper's h_int order)
_INT_PAIRS = {9: "ab", 10: "bc", 11: "cd", 12: "da", 13: "ef", 14: "fg", 15: "gh",
              16: "he", 17: "ae", 18: "bf", 19: "cg", 20: "dh"}
# canonical parent faces: children in Morton order over the tangential axes
_CANON3D_FACES = [("adeh", 0), ("bcfg", 1), ("abef", 2), ("dchg", 3), ("abdc", 4), ("efhg", 5)]


def _faces_of(ch, sec):
    return [f for f in range(6) if _FACE_SEC3D[ch][f] == sec]


def _sub3d(T, n, rows, cols):
    r = np.concatenate([np.arange(f * n, (f + 1) * n) for f in rows])
    c = np.concatenate([np.arange(f * n, (f + 1) * n) for f in cols])
    return T[np.ix_(r, c)]


def canon_perm_3d(n):
    ext_blocks = []
    for sec in range(1, 9):
        ch = _CHILD_OF_EXT[sec]
        ext_blocks += [(ch, f) for f in _faces_of(ch, sec)]
    pos = {b: i for i, b in enumerate(ext_blocks)}
    canon = [(ch, f) for chs, f in _CANON3D_FACES for ch in chs]
    return np.concatenate([np.arange(pos[b] * n, (pos[b] + 1) * n) for b in canon]), ext_blocks


def merge_3d_dtn(Ts, hs, want_T=True):
    """Appendix C.2.  Blocks of A, B, C, D follow the printed matrices: block
    (r, s) of B is T^(k)_{k,s} for the child k of exterior section r when k
    touches interior section s; C and D likewise (D sums both children of a
    shared interface on its diagonal)."""
    n = Ts["a"].shape[0] // 6

    def t(ch, i, j):
        return _sub3d(Ts[ch], n, _faces_of(ch, i), _faces_of(ch, j))

    def hv(ch, i):
        return np.concatenate([hs[ch][f * n:(f + 1) * n] for f in _faces_of(ch, i)])

    ints = list(range(9, 21))
    touches = {s: set(_INT_PAIRS[s]) for s in ints}
    dt = Ts["a"].dtype
    A = sla.block_diag(*[t(_CHILD_OF_EXT[k], k, k) for k in range(1, 9)])
    B = np.zeros((24 * n, 12 * n), dt)
    C = np.zeros((12 * n, 24 * n), dt)
    D = np.zeros((12 * n, 12 * n), dt)
    for k in range(1, 9):
        ch = _CHILD_OF_EXT[k]
        for j, s in enumerate(ints):
            if ch in touches[s]:
                B[(k - 1) * 3 * n:k * 3 * n, j * n:(j + 1) * n] = t(ch, k, s)
                C[j * n:(j + 1) * n, (k - 1) * 3 * n:k * 3 * n] = t(ch, s, k)
    for i, s in enumerate(ints):
        for j, s2 in enumerate(ints):
            for ch in touches[s] & touches[s2]:
                D[i * n:(i + 1) * n, j * n:(j + 1) * n] += t(ch, s, s2)
    h_ext = np.concatenate([hv(_CHILD_OF_EXT[k], k) for k in range(1, 9)])
    h_int = np.concatenate([hv(_INT_PAIRS[s][0], s) + hv(_INT_PAIRS[s][1], s) for s in ints])
    lu = sla.lu_factor(D)
    DinvC = sla.lu_solve(lu, C)
    Dinvh = sla.lu_solve(lu, h_int)
    perm, _ = canon_perm_3d(n)
    S = -DinvC
    gt = -Dinvh
    if want_T:
        T = A - B @ DinvC
        h = h_ext - B @ Dinvh
        return T[np.ix_(perm, perm)], h[perm], S, gt, perm
    return None, None, S, gt, perm


def children_g_3d_dtn(g_canon, S, gt, perm):
    n = len(g_canon) // 24
    g_sec = np.empty_like(g_canon)
    g_sec[perm] = g_canon
    gi = S @ g_sec + gt
    _, ext_blocks = canon_perm_3d(n)
    out = {}
    for ch in "abcdefgh":
        parts = []
        for f in range(6):
            sec = _FACE_SEC3D[ch][f]
            if sec <= 8:
                b = ext_blocks.index((ch, f))
                parts.append(g_sec[b * n:(b + 1) * n])
            else:
                j = sec - 9
                parts.append(gi[j * n:(j + 1) * n])
        out[ch] = np.concatenate(parts)
    return out
