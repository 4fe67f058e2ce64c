"""Pins of the oracle adjoint (oracle/adjoint.py): the coefficient gradient
against central finite differences of the oracle's forward solve, and the
adjoint identity Re<ubar, u(g, f)> = Re<gbar, g> + Re<fbar, f>."""

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA
from oracle import composite as O2
from oracle import hps as O

CASES = [
    ("dtn2d", lambda: W.elliptic_2d(seed=4), 6, 1),
    ("iti", lambda: W.helmholtz_bumps_2d(seed=1), 8, 1),
    ("dtn3d", lambda: W.elliptic_3d(seed=2), 5, 1),
]


def _setup(mk, p, L, seed=3):
    pr = mk()
    x, a, b, c, f, g = O.sample_problem(pr, p, p - 2, L)
    rng = np.random.default_rng(seed)
    cplx = pr.kind == "iti"
    ubar = rng.standard_normal(f.shape) + (1j * rng.standard_normal(f.shape) if cplx else 0.0)
    if cplx:
        f = f.astype(complex)
        g = g.astype(complex)
    return pr, a, b, c, f, g, ubar


def _forward(pr, p, L, a, b, c, f, g):
    if pr.kind == "iti":
        return O2.solve_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, pr.eta)
    return O2.solve_dtn(pr.dim, p, L, pr.lo, pr.hi, a, b, c, f, g)


def _adjoint(pr, p, L, a, b, c, f, g, ubar):
    if pr.kind == "iti":
        return OA.adjoint_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, ubar, pr.eta)
    return OA.adjoint_dtn(pr.dim, p, L, pr.lo, pr.hi, a, b, c, f, g, ubar)


@pytest.mark.parametrize("name,mk,p,L", CASES, ids=[c[0] for c in CASES])
def test_coefficient_gradient_matches_finite_differences(name, mk, p, L):
    pr, a, b, c, f, g, ubar = _setup(mk, p, L)
    gbar, fbar, grad_c, u = _adjoint(pr, p, L, a, b, c, f, g, ubar)
    J = lambda cc: float(np.real(np.vdot(ubar, _forward(pr, p, L, a, b, cc, f, g))))  # noqa: E731
    rng = np.random.default_rng(11)
    interior = np.nonzero(grad_c.reshape(-1))[0]
    assert interior.size > 0
    hstep = 1e-6
    for j in rng.choice(interior, 5, replace=False):
        cp, cm = c.copy().reshape(-1), c.copy().reshape(-1)
        cp[j] += hstep
        cm[j] -= hstep
        fd = (J(cp.reshape(c.shape)) - J(cm.reshape(c.shape))) / (2 * hstep)
        assert abs(fd - grad_c.reshape(-1)[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, grad_c.reshape(-1)[j])
    # boundary nodes carry no coefficient dependence
    assert np.count_nonzero(grad_c) <= grad_c.size


@pytest.mark.parametrize("name,mk,p,L", CASES, ids=[c[0] for c in CASES])
def test_adjoint_identity(name, mk, p, L):
    pr, a, b, c, f, g, ubar = _setup(mk, p, L)
    gbar, fbar, grad_c, u = _adjoint(pr, p, L, a, b, c, f, g, ubar)
    lhs = np.real(np.vdot(ubar, u))
    rhs = np.real(np.vdot(gbar, g)) + np.real(np.vdot(fbar, f))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def test_planted_sign_error_in_the_gradient_is_caught(monkeypatch):
    """A gradient with the wrong sign must fail the finite-difference pin."""
    pr, a, b, c, f, g, ubar = _setup(CASES[0][1], 6, 1)
    gbar, fbar, grad_c, u = _adjoint(pr, 6, 1, a, b, c, f, g, ubar)
    j = int(np.nonzero(grad_c.reshape(-1))[0][0])
    J = lambda cc: float(np.real(np.vdot(ubar, _forward(pr, 6, 1, a, b, cc, f, g))))  # noqa: E731
    cp, cm = c.copy().reshape(-1), c.copy().reshape(-1)
    cp[j] += 1e-6
    cm[j] -= 1e-6
    fd = (J(cp.reshape(c.shape)) - J(cm.reshape(c.shape))) / 2e-6
    assert abs(fd + grad_c.reshape(-1)[j]) > 1e-3 * abs(fd)


def test_grid_interpolation_is_exact_on_cubics():
    """The theta-to-node interpolation of the differentiation workload
    reproduces tensor cubics exactly (it is the standard 4-point Lagrange
    rule per axis)."""
    x = np.random.default_rng(0).uniform(-1, 1, (200, 2))
    n = 64
    g1 = np.linspace(-1, 1, n)
    X, Y = np.meshgrid(g1, g1, indexing="ij")
    f = lambda a, b: 1 + a - 2 * b + a * b + a ** 3 - b ** 3 + a ** 2 * b + a ** 3 * b ** 3  # noqa: E731
    I = W.grid_interp_matrix(x, n)
    assert np.abs(I @ f(X, Y).reshape(-1, order="F") - f(x[:, 0], x[:, 1])).max() < 1e-12
    # a quartic is not reproduced (the rule is cubic)
    q = lambda a, b: a ** 4  # noqa: E731
    assert np.abs(I @ q(X, Y).reshape(-1, order="F") - q(x[:, 0], x[:, 1])).max() > 1e-9
