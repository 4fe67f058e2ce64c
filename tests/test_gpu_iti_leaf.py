"""The two ItI leaf solvers (hps_options.iti_leaf): the complex LU of the whole
leaf matrix B (1, the paper's Algorithm "2D ItI local solve") and the
elimination of the interior nodes (2: real LU of L(I_i, I_i) and a complex
Schur complement on the boundary).  Both are held to the parity bar against
the oracle, for the build-time source, a new source, and the adjoint."""

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA
from test_gpu_parity import P, TOL, dev, oracle_solve, rel, sample_inputs  # noqa: F401

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    ("helmholtz_p16_L3", lambda: W.helmholtz_bumps_2d(seed=1), 16, 3),
    ("helmholtz_p12_L4", lambda: W.helmholtz_bumps_2d(seed=1), 12, 4),
    ("e2_p8_L3", W.e2_iti_2d, 8, 3),
    ("e2_single_leaf", W.e2_iti_2d, 10, 0),
]


def _solve(P, pr, p, inputs, mode, f_solve=None, lazy=False):
    t, x, a, b, c, f, g = inputs
    h = P.hps_build(t, p, p - 2, P.HPS_ITI, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    eta=pr.eta, iti_leaf=mode, lazy_root=lazy)
    u = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
    P.hps_solve(h, dev(g), u, f=None if f_solve is None else dev(f_solve))
    torch.cuda.synchronize()
    P.hps_free(h)
    return u.cpu().numpy()


@pytest.mark.parametrize("mode", [1, 2], ids=["dense_B", "interior_elimination"])
@pytest.mark.parametrize("name,mk,p,L", CASES, ids=[c[0] for c in CASES])
def test_iti_leaf_modes_match_oracle(P, name, mk, p, L, mode):
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    uo = oracle_solve(pr, p, L, inputs)
    assert rel(_solve(P, pr, p, inputs, mode), uo) <= TOL


@pytest.mark.parametrize("mode", [1, 2], ids=["dense_B", "interior_elimination"])
def test_iti_leaf_modes_new_source(P, mode):
    pr = W.helmholtz_bumps_2d(seed=1)
    p, L = 12, 3
    inputs = sample_inputs(P, pr, p, L)
    rng = np.random.default_rng(4)
    f2 = rng.standard_normal(inputs[5].shape) + 1j * rng.standard_normal(inputs[5].shape)
    ug = _solve(P, pr, p, inputs, mode, f_solve=f2, lazy=True)
    assert rel(ug, oracle_solve(pr, p, L, inputs, f_override=f2)) <= TOL


@pytest.mark.parametrize("mode", [1, 2], ids=["dense_B", "interior_elimination"])
def test_iti_leaf_modes_adjoint(P, mode):
    pr = W.helmholtz_bumps_2d(seed=1)
    p, L = 8, 2
    inputs = sample_inputs(P, pr, p, L)
    t, x, a, b, c, f, g = inputs
    rng = np.random.default_rng(3)
    ubar = rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)
    h = P.hps_build(t, p, p - 2, P.HPS_ITI, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    eta=pr.eta, iti_leaf=mode)
    u = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
    P.hps_solve(h, dev(g), u, f=dev(f))
    gb = torch.zeros(g.shape, dtype=torch.complex128, device="cuda")
    fb = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
    P.hps_solve_adjoint(h, dev(ubar), gb, fb)
    gc = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    P.hps_coeff_gradient(h, u, fb, gc=gc)
    torch.cuda.synchronize()
    P.hps_free(h)
    og, of, oc, ou = OA.adjoint_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, ubar, pr.eta)
    assert rel(gb.cpu().numpy(), og) <= TOL
    assert rel(fb.cpu().numpy(), of) <= TOL
    assert rel(gc.cpu().numpy(), oc) <= TOL


def test_automatic_choice_uses_elimination_for_small_leaves(P):
    """The benchmark workload (leaf side 1/32, k = 20) is far from leaf
    resonance, so the automatic choice eliminates the interior; the result
    equals the dense-B solve."""
    from residuals import check_iti
    pr = W.helmholtz_bumps_2d(seed=1)
    p, L = 16, 5
    inputs = sample_inputs(P, pr, p, L)
    ua = _solve(P, pr, p, inputs, 0)
    ud = _solve(P, pr, p, inputs, 1)
    # each solver is held to the 1e-10 bar, so the two may differ by twice it
    assert rel(ua, ud) <= 2 * TOL
    t, x, a, b, c, f, g = inputs
    rng = np.random.default_rng(2)
    sample = sorted(set(rng.choice(1024, 16, replace=False).tolist()) | {0, 1023})
    assert check_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, ua, pr.eta, sample) < 1e-10
