"""The size-independent residual checks (tests/residuals.py) accept the
oracle's solution and reject a perturbed one, so they can stand in for the
oracle at sizes where it is too slow."""

import numpy as np
import pytest

import workloads as W
from oracle import hps
from residuals import check_dtn, check_iti


@pytest.mark.parametrize("dim,p,L", [(2, 8, 2), (3, 6, 1)])
def test_dtn_residuals(dim, p, L):
    pr = W.e1_dtn_2d() if dim == 2 else W.elliptic_3d()
    q = p - 2
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, L)
    s = hps.build(dim, "dtn", p, q, L, pr.lo, pr.hi, a, b, c, f)
    u = hps.solve(s, g)
    nl = 2 ** (dim * L)
    sample = range(nl)
    assert check_dtn(dim, p, L, pr.lo, pr.hi, a, b, c, f, g, u, sample) < 1e-12
    u2 = u.copy()
    u2[1, 3] += 1e-6 * np.abs(u).max()
    assert check_dtn(dim, p, L, pr.lo, pr.hi, a, b, c, f, g, u2, sample) > 1e-9


def test_iti_residuals():
    pr = W.helmholtz_bumps_2d(k=12.0)
    p, q, L = 8, 6, 2
    x, a, b, c, f, g = hps.sample_problem(pr, p, q, L)
    s = hps.build(2, "iti", p, q, L, pr.lo, pr.hi, a, b, c, f, eta=pr.eta)
    u = hps.solve(s, g)
    sample = range(16)
    assert check_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, u, pr.eta, sample) < 1e-12
    u2 = u.copy()
    u2[5, 0] += 1e-6 * np.abs(u).max()
    assert check_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, u2, pr.eta, sample) > 1e-9
