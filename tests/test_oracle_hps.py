"""Pins for the oracle's leaf stage, merges and downward pass.

Each pin is something the paper or the mathematics fixes independently of
the oracle: exactness on polynomial solutions, closed forms of DtN maps,
the brute-force composite solve (O2), the paper's hp-convergence rate
(Section 5.1), the ItI D^{-1} identity (Appendix B.2) and the top-level D
sizes of Table "merge_sizes" (Section 4.2).
"""

import json
import os

import numpy as np
import pytest

import workloads as W
from workloads.problems import Problem, _const_coeffs, box_normals
from oracle import composite, geometry as geo, hps, leaf as lf, merge as mg

HERE = os.path.dirname(__file__)


def rel(u, v):
    return np.abs(u - v).max() / np.abs(v).max()


# ---------------------------------------------------------------- leaf ----

@pytest.mark.parametrize("p", [6, 8, 12])
def test_dtn_laplace_leaf_closed_forms(p):
    """Laplace DtN of one leaf: T 1 = 0 and T (x at the Gauss points) = n_x."""
    q = p - 2
    lo, hi = (-0.5, 0.25), (0.0, 0.75)
    xb = geo.root_boundary_points(2, lo, hi, 0, q)
    n = box_normals(xb, lo, hi)
    one = np.ones(p * p)
    zero = np.zeros(p * p)
    T, h, Y, v = lf.dtn_leaf(2, p, q, 0.5, one, [zero, zero], zero, zero)
    assert np.abs(T @ np.ones(4 * q)).max() < 1e-10
    assert np.allclose(T @ xb[:, 0], n[:, 0], atol=1e-10)
    assert np.allclose(T @ xb[:, 1], n[:, 1], atol=1e-10)
    assert np.abs(h).max() == 0.0


def _poly_problem(dim, deg, seed, kind="dtn", eta=2.0, cval=0.0):
    P = W.polynomial_field(dim, deg, seed, tensor=True)
    lo, hi = (-1.0,) * dim, (1.0,) * dim
    if kind == "dtn":
        return Problem("poly", dim, lo, hi, "dtn", seed, _const_coeffs(dim, c=cval),
                       lambda x: P.lap(x) + cval * P.value(x), P.value, P.value), P

    def g(xb):
        nn = box_normals(xb, lo, hi)
        gr = P.grad(xb)
        return sum(nn[:, k] * gr[k] for k in range(dim)) + 1j * eta * P.value(xb)

    return Problem("poly", dim, lo, hi, "iti", seed, _const_coeffs(dim, c=cval),
                   lambda x: (P.lap(x) + cval * P.value(x)).astype(complex), g,
                   P.value, eta=eta), P


@pytest.mark.parametrize("dim,kind,p,L", [(2, "dtn", 8, 0), (2, "dtn", 8, 2), (2, "dtn", 12, 1),
                                          (2, "iti", 8, 0), (2, "iti", 8, 2), (2, "iti", 10, 1),
                                          (3, "dtn", 6, 0), (3, "dtn", 6, 1)])
def test_polynomial_exactness(dim, kind, p, L):
    """u in Q_{p-3} (tensor degree p-3) is reproduced to roundoff; degree
    p-2 is not (negative control)."""
    pr, P = _poly_problem(dim, p - 3, 10 + p, kind, cval=1.5)
    x, u = hps.solve_problem(pr, p, L)
    assert rel(u, P.value(x)) < 1e-11
    pr2, P2 = _poly_problem(dim, p - 2, 20 + p, kind, cval=1.5)
    x, u2 = hps.solve_problem(pr2, p, max(L, 1))
    assert rel(u2, P2.value(x)) > 1e-9



@pytest.mark.parametrize("dim,kind,p,L", [(2, "dtn", 8, 0), (2, "dtn", 8, 2), (2, "dtn", 12, 1),
                                          (2, "iti", 8, 0), (2, "iti", 8, 2), (2, "iti", 10, 1),
                                          (3, "dtn", 6, 0), (3, "dtn", 6, 1)])
def test_polynomial_exactness_variable_coefficients(dim, kind, p, L):
    """The same exactness with seeded non-constant a(x), b(x), c(x): f is
    formed from u's closed-form derivatives, so the collocation equations
    hold exactly for u in Q_{p-3} whatever the coefficients are.  This pins
    how a, b and c enter the leaf operator (Section 3.2: diag(a) times the
    spectral Laplacian, diag(b_k) times the k-th derivative, diag(c))."""
    pr = W.poly_varcoef(dim, p - 3, 10 + p, kind)
    x, u = hps.solve_problem(pr, p, L)
    assert rel(u, pr.u_exact(x)) < 1e-11
    pr2 = W.poly_varcoef(dim, p - 2, 20 + p, kind)
    x, u2 = hps.solve_problem(pr2, p, max(L, 1))
    assert rel(u2, pr2.u_exact(x)) > 1e-9

# ------------------------------------------------------- O1 against O2 ----

@pytest.mark.parametrize("L,p", [(1, 8), (2, 8), (2, 10)])
def test_o1_matches_composite_dtn_2d(L, p):
    pr = W.e1_dtn_2d()
    q = p - 2
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, L)
    s = hps.build(2, "dtn", p, q, L, pr.lo, pr.hi, a, b, c, f)
    u1 = hps.solve(s, g)
    u2 = composite.solve_dtn(2, p, L, pr.lo, pr.hi, a, b, c, f, g)
    assert rel(u1, u2) < 1e-12


@pytest.mark.parametrize("L,p,which", [(1, 8, "e2"), (2, 8, "e2"), (2, 8, "bumps")])
def test_o1_matches_composite_iti(L, p, which):
    pr = W.e2_iti_2d() if which == "e2" else W.helmholtz_bumps_2d(k=10.0)
    q = p - 2
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, L)
    s = hps.build(2, "iti", p, q, L, pr.lo, pr.hi, a, b, c, f, eta=pr.eta)
    u1 = hps.solve(s, g)
    u2 = composite.solve_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, pr.eta)
    assert rel(u1, u2) < 1e-11


@pytest.mark.parametrize("p", [6, 8])
def test_o1_matches_composite_dtn_3d(p):
    pr = W.elliptic_3d()
    q = p - 2
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, 1)
    s = hps.build(3, "dtn", p, q, 1, pr.lo, pr.hi, a, b, c, f)
    u1 = hps.solve(s, g)
    u2 = composite.solve_dtn(3, p, 1, pr.lo, pr.hi, a, b, c, f, g)
    assert rel(u1, u2) < 1e-12


def test_iti_w_route_equals_direct_solve():
    """Eq. "ItI D inverse": D^{-1} through W = I - D12 D21 equals a direct
    LU solve with D."""
    pr = W.helmholtz_bumps_2d(k=15.0)
    p, q, L = 8, 6, 2
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, L)
    s1 = hps.build(2, "iti", p, q, L, pr.lo, pr.hi, a, b, c, f, eta=pr.eta)
    s2 = hps.build(2, "iti", p, q, L, pr.lo, pr.hi, a, b, c, f, eta=pr.eta, iti_direct=True)
    assert rel(hps.solve(s1, g), hps.solve(s2, g)) < 1e-12
    for lev in s1.levels:
        for n1, n2 in zip(s1.levels[lev], s2.levels[lev]):
            assert rel(n1["S"], n2["S"]) < 1e-11


def test_laplace_node_maps_annihilate_constants():
    """For Lap u = 0 the merged DtN map of every node sends constants to 0."""
    pr = W.poisson_poly_2d(seed=0)
    p, q, L = 8, 6, 2
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, L)
    s = hps.build(2, "dtn", p, q, L, pr.lo, pr.hi, a, b, c, f)
    for lev, nodes in s.levels.items():
        for node in nodes:
            T = node["T"]
            assert np.abs(T @ np.ones(T.shape[1])).max() < 1e-9 * np.abs(T).max()


def test_interior_continuity_after_down_pass():
    """After the downward pass, the two leaves sharing an interior side get
    the same Dirichlet data (DtN) and opposite-normal impedance relations (ItI:
    g_a = -(outgoing of b))."""
    pr = W.helmholtz_bumps_2d(k=12.0)
    p, q, L = 8, 6, 1
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, L)
    s = hps.build(2, "iti", p, q, L, pr.lo, pr.hi, a, b, c, f, eta=pr.eta)
    gl = hps.leaf_boundary_data(s, g)
    # leaf 0 = SW (a), leaf 1 = SE (b): a's E side faces b's W side
    out_b = s.leaf_T[1] @ gl[1] + s.leaf_h[1]
    assert np.allclose(gl[0][q:2 * q], -out_b[3 * q:4 * q], atol=1e-9 * np.abs(out_b).max())


# ------------------------------------------------------ convergence -------

def test_e1_hp_convergence():
    """Section 5.1: errors decay like O(h^{p-2}) (observed order within 1.5)."""
    pr = W.e1_dtn_2d()
    p = 8
    errs = []
    for L in (3, 4):
        x, u = hps.solve_problem(pr, p, L)
        errs.append(rel(u, pr.u_exact(x)))
    order = np.log2(errs[0] / errs[1])
    assert order > (p - 2) - 1.5
    assert errs[1] < 5e-5


def test_e2_hp_convergence():
    pr = W.e2_iti_2d()
    p = 8
    errs = []
    for L in (3, 4):
        x, u = hps.solve_problem(pr, p, L)
        errs.append(rel(u, pr.u_exact(x)))
    order = np.log2(errs[0] / errs[1])
    assert order > (p - 2) - 1.5
    assert errs[1] < 1e-2


def test_e1_spectral_convergence_in_p():
    """Section 5.1 at a fixed tree: for the smooth E1 solution the error
    falls faster than any fixed power of p (spectral convergence).  At depth
    3 each step of 4 in p gains a growing factor: more than 30x from 8 to 12
    and more than 300x from 12 to 16; an algebraic rate p^-k would give a
    shrinking gain, (8/12)^k then (12/16)^k."""
    pr = W.e1_dtn_2d()
    errs = {}
    for p in (8, 12, 16):
        x, u = hps.solve_problem(pr, p, 3)
        errs[p] = rel(u, pr.u_exact(x))
    assert errs[12] / errs[8] < 1 / 30
    assert errs[16] / errs[12] < 1 / 300
    assert errs[16] < 1e-7



def test_top_merge_sizes_match_table():
    """Table "merge_sizes": the top-level D of a uniform octree of depth L has
    12 q^2 4^(L-1) rows.  The oracle's D for small trees follows the same
    count, and the printed uniform sizes follow from it."""
    with open(os.path.join(HERE, "golden", "table_merge_sizes.json")) as fh:
        tab = json.load(fh)
    for method, p, err, nleaves, dsize in tab["rows"]:
        if method != "uniform":
            continue
        L = round(np.log(nleaves) / np.log(8))
        q = p - 2
        assert 8 ** L == nleaves
        assert 12 * q * q * 4 ** (L - 1) == dsize
    # the oracle's own D has that size: S maps 24 n exterior to 12 n interior
    pr = W.elliptic_3d()
    p, q = 6, 4
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, 1)
    s = hps.build(3, "dtn", p, q, 1, pr.lo, pr.hi, a, b, c, f)
    S = s.levels[0][0]["S"]
    assert S.shape == (12 * q * q, 24 * q * q)


# ----------------------------------------------- planted mistakes --------

def test_planted_sign_error_in_v_is_caught(monkeypatch):
    """With the printed minus sign in v (Algorithm "2D DtN local solve") the
    polynomial pin fails: the reading v = +L_ii^{-1} f_i is the right one."""
    orig = lf.dtn_leaf

    def bad(dim, p, q, hlen, a, b, c, f):
        T, h, Y, v = orig(dim, p, q, hlen, a, b, c, f)
        return T, -h, Y, -v

    monkeypatch.setattr(lf, "dtn_leaf", bad)
    pr, P = _poly_problem(2, 5, 3)
    x, u = hps.solve_problem(pr, 8, 1)
    assert rel(u, P.value(x)) > 1e-2


def test_planted_transposed_block_is_caught(monkeypatch):
    """Transposing one child's T before the merge breaks agreement with O2."""
    orig = mg.merge_2d_dtn

    def bad(Ts, hs):
        Ts = dict(Ts)
        Ts["c"] = Ts["c"].T.copy()
        return orig(Ts, hs)

    pr = W.e1_dtn_2d()
    p, q, L = 8, 6, 1
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, L)
    u2 = composite.solve_dtn(2, p, L, pr.lo, pr.hi, a, b, c, f, g)
    monkeypatch.setattr(mg, "merge_2d_dtn", bad)
    s = hps.build(2, "dtn", p, q, L, pr.lo, pr.hi, a, b, c, f)
    assert rel(hps.solve(s, g), u2) > 1e-6


@pytest.mark.parametrize("mistake", ["a_on_columns", "a_on_one_derivative", "b_on_columns"])
def test_planted_coefficient_mistakes_are_caught(monkeypatch, mistake):
    """A plausible slip in how the coefficients enter L -- a scaling columns
    instead of rows, a multiplying only one second derivative, b scaling
    columns -- leaves every constant-coefficient pin green but fails the
    variable-coefficient exactness pin."""
    def bad(dim, p, hlen, a, b, c):
        Ds = lf.derivative_matrices(dim, p, hlen)
        n = p ** dim
        if mistake == "a_on_columns":
            L = sum(Dk @ Dk for Dk in Ds) * a[None, :] + c[:, None] * np.eye(n)
        elif mistake == "a_on_one_derivative":
            L = a[:, None] * (Ds[0] @ Ds[0]) + sum(Dk @ Dk for Dk in Ds[1:]) + c[:, None] * np.eye(n)
        else:
            L = a[:, None] * sum(Dk @ Dk for Dk in Ds) + c[:, None] * np.eye(n)
        for k in range(dim):
            L = L + (Ds[k] * b[k][None, :] if mistake == "b_on_columns" else b[k][:, None] * Ds[k])
        return L

    pr = W.poly_varcoef(2, 5, 18, "dtn")
    x, u = hps.solve_problem(pr, 8, 1)
    assert rel(u, pr.u_exact(x)) < 1e-11
    monkeypatch.setattr(lf, "assemble_L", bad)
    x, u = hps.solve_problem(pr, 8, 1)
    assert rel(u, pr.u_exact(x)) > 1e-4
