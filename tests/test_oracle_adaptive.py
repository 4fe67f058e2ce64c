"""Pins for the adaptive 3D oracle (Section 4.2): 4-to-1 panel projections,
the refinement interpolation, the level restriction, polynomial exactness on
2:1 trees, the uniform special case and the brute-force composite solve."""

import numpy as np
import pytest

import workloads as W
from workloads.problems import Problem, _const_coeffs
from oracle import adaptive as ad
from oracle import composite, hps
from oracle.spectral import cheb_points, gauss_legendre


def rel(u, v):
    return np.abs(u - v).max() / np.abs(v).max()


@pytest.mark.parametrize("q", [2, 4, 6, 10])
def test_panel_projections_exact_on_Q(q):
    C2F, F2C = ad.panel_projections(q)
    xc, _ = gauss_legendre(q, 0.0, 1.0)
    xh = [gauss_legendre(q, 0.0, 0.5)[0], gauss_legendre(q, 0.5, 1.0)[0]]
    rng = np.random.default_rng(q)
    for deg in (0, q - 1):
        c = rng.standard_normal((deg + 1, deg + 1))
        fun = lambda s, t: np.polynomial.polynomial.polyval2d(s, t, c)  # noqa: E731
        B, A = np.meshgrid(xc, xc, indexing="ij")
        coarse = fun(A.ravel(), B.ravel())
        fine = []
        for quad in range(4):
            a, b = quad & 1, quad >> 1
            Bf, Af = np.meshgrid(xh[b], xh[a], indexing="ij")
            fine.append(fun(Af.ravel(), Bf.ravel()))
        fine = np.concatenate(fine)
        assert np.allclose(C2F @ coarse, fine, atol=1e-11)
        assert np.allclose(F2C @ fine, coarse, atol=1e-11)
    assert np.allclose(F2C @ C2F, np.eye(q * q), atol=1e-12)
    # degree q is not carried exactly by the coarse panel
    B, A = np.meshgrid(xc, xc, indexing="ij")
    fine = np.concatenate([
        np.meshgrid(xh[quad >> 1], xh[quad & 1], indexing="ij")[1].ravel() ** q for quad in range(4)])
    assert np.abs(C2F @ (A.ravel() ** q) - fine).max() > 1e-8


@pytest.mark.parametrize("p", [4, 6, 8])
def test_child_interpolation_exact(p):
    rng = np.random.default_rng(p)
    c = rng.standard_normal((p, p, p))
    x0 = ad.leaf_nodes((-1, -1, -1), (1, 1, 1), 0, (0, 0, 0), p)
    x1 = ad.eight_child_nodes((-1, -1, -1), (1, 1, 1), 0, (0, 0, 0), p)
    fun = lambda x: np.polynomial.polynomial.polyval3d(x[:, 0], x[:, 1], x[:, 2], c)  # noqa: E731
    assert np.allclose(ad.L8f1_apply(p, fun(x0)), fun(x1), atol=1e-10 * np.abs(c).sum())


def _is_balanced(leaves):
    cells = {}
    for lv, ix in leaves:
        cells[(lv, tuple(ix))] = True
    maxl = max(lv for lv, _ in leaves)
    # map every finest-level cell to its leaf level, then compare face neighbours
    n = 2 ** maxl
    lev = np.full((n, n, n), -1)
    for lv, ix in leaves:
        s = 2 ** (maxl - lv)
        lev[ix[0] * s:(ix[0] + 1) * s, ix[1] * s:(ix[1] + 1) * s, ix[2] * s:(ix[2] + 1) * s] = lv
    assert (lev >= 0).all()
    for axis in range(3):
        a = np.take(lev, range(n - 1), axis=axis)
        b = np.take(lev, range(1, n), axis=axis)
        if np.abs(a - b).max() > 1:
            return False
    return True


def test_balance_enforces_level_restriction():
    rng = np.random.default_rng(0)
    leaves = [(1, (i, j, k)) for i in range(2) for j in range(2) for k in range(2)]
    for _ in range(12):
        lv, ix = leaves.pop(rng.integers(len(leaves)))
        if lv < 4:
            leaves += ad.children_of(lv, ix)
        else:
            leaves.append((lv, ix))
    out = ad.balance(leaves)
    assert _is_balanced(out)
    vol = sum(8.0 ** -lv for lv, _ in out)
    assert abs(vol - 1.0) < 1e-12


def test_refine_keeps_polynomials_coarse_and_splits_a_sharp_source():
    P = W.polynomial_field(3, 4, 1, tensor=True)
    leaves = ad.refine([P.value], (-1,) * 3, (1,) * 3, 6, 1e-6, 1, 4)
    assert all(lv == 1 for lv, _ in leaves) and len(leaves) == 8
    pr = W.sharp_source_3d(seed=3, width=0.1)
    leaves = ad.refine([pr.source], pr.lo, pr.hi, 6, 1e-3, 1, 4)
    levels = [lv for lv, _ in leaves]
    assert max(levels) == 4 and min(levels) <= 2
    assert _is_balanced(leaves)
    assert abs(sum(8.0 ** -lv for lv in levels) - 1.0) < 1e-12
    # the finest leaves sit around the source centre
    z = np.array(pr.info["centre"])
    fine = [ix for lv, ix in leaves if lv == 4]
    centres = np.array([(-1 + (np.array(ix) + 0.5) * 2 / 16) for ix in fine])
    assert np.min(np.linalg.norm(centres - z, axis=1)) < 0.2


def test_uniform_tree_equals_uniform_oracle():
    pr = W.elliptic_3d()
    p = 6
    leaves = ad.sort_leaves([(1, (i, j, k)) for i in range(2) for j in range(2) for k in range(2)])
    x, a, b, c, f, g = ad.sample_adaptive(pr, leaves, p)
    x2, a2, b2, c2, f2, g2 = hps.sample_problem(pr, p, p - 2, 1)
    assert np.array_equal(x, x2) and np.array_equal(g, g2)
    u = np.array(ad.solve_adaptive(ad.build_adaptive(leaves, p, pr.lo, pr.hi, a, b, c, f), g))
    uo = hps.solve(hps.build(3, "dtn", p, p - 2, 1, pr.lo, pr.hi, a2, b2, c2, f2), g2)
    assert rel(u, uo) < 1e-13


def _two_one_tree():
    leaves = [(1, (i, j, k)) for i in range(2) for j in range(2) for k in range(2) if (i, j, k) != (0, 0, 0)]
    leaves += ad.children_of(1, (0, 0, 0))
    # refine one more cell inside the refined corner, then balance
    leaves.remove((2, (1, 1, 1)))
    leaves += ad.children_of(2, (1, 1, 1))
    return ad.sort_leaves(ad.balance(leaves))


@pytest.mark.parametrize("p", [6, 8])
def test_polynomial_exactness_on_2to1_tree(p):
    leaves = _two_one_tree()
    assert len(set(lv for lv, _ in leaves)) == 3
    for deg, exact in ((p - 3, True), (p - 2, False)):
        P = W.polynomial_field(3, deg, 5 + deg, tensor=True)
        pr = Problem("p3", 3, (-1,) * 3, (1,) * 3, "dtn", None, _const_coeffs(3, c=0.7),
                     lambda x: P.lap(x) + 0.7 * P.value(x), P.value, P.value)
        x, a, b, c, f, g = ad.sample_adaptive(pr, leaves, p)
        u = np.array(ad.solve_adaptive(ad.build_adaptive(leaves, p, pr.lo, pr.hi, a, b, c, f), g))
        err = rel(u.reshape(-1), P.value(x))
        assert (err < 1e-11) if exact else (err > 1e-9)


def test_adaptive_matches_composite_solve():
    leaves = _two_one_tree()
    pr = W.elliptic_3d()
    p = 6
    x, a, b, c, f, g = ad.sample_adaptive(pr, leaves, p)
    u = np.array(ad.solve_adaptive(ad.build_adaptive(leaves, p, pr.lo, pr.hi, a, b, c, f), g))
    u2 = composite.solve_dtn_adaptive(leaves, p, pr.lo, pr.hi, a, b, c, f, g)
    assert rel(u, u2) < 1e-12


def test_adaptive_root_boundary_points_are_on_the_box():
    leaves = _two_one_tree()
    q = 4
    xb = ad.root_boundary_points(leaves, (-1,) * 3, (1,) * 3, q)
    on = (np.abs(np.abs(xb) - 1.0) < 1e-14).sum(axis=1)
    assert (on == 1).all()
    root, _ = ad.build_tree(leaves)
    panels = [pn for face in root.faces for pn in face]
    assert len(xb) == q * q * len(panels)
    # the panels tile the six faces of [-1, 1]^3 (total area 24)
    assert abs(sum(4.0 ** (1 - lv) for lv, _ in panels) - 24.0) < 1e-12
