"""GPU parity of the lazy-root option (hps_options.lazy_root).

With lazy_root the top merge keeps [C | h_int] and the factors of D instead
of forming S = -D^{-1} C and the particular part (the top-level merge
formulas of Section 3.2); the solve applies D^{-1} to C g + h_int.  The result
is the same solution of the same linear system, so it is held to the same bar
as the default path: relative L-infinity error <= 1e-10 against the oracle.
"""

import numpy as np
import pytest

import workloads as W
from test_gpu_parity import P, TOL, dev, oracle_solve, rel, sample_inputs  # noqa: F401
from residuals import check_iti

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    ("poisson2d_p8_L2", lambda: W.poisson_poly_2d(seed=0), 8, 2),
    ("e1_dtn_p12_L3", W.e1_dtn_2d, 12, 3),
    ("helmholtz_iti_p16_L3", lambda: W.helmholtz_bumps_2d(seed=1), 16, 3),
    ("e2_iti_p8_L1", W.e2_iti_2d, 8, 1),
    ("elliptic3d_p6_L2", lambda: W.elliptic_3d(seed=2), 6, 2),
    ("elliptic3d_single_leaf", lambda: W.elliptic_3d(seed=2), 8, 0),
]


def lazy_solve(P, pr, p, inputs, f_solve=None, nrhs=None, G=None, F=None):
    t, x, a, b, c, f, g = inputs
    kind = P.HPS_ITI if pr.kind == "iti" else P.HPS_DTN
    h = P.hps_build(t, p, p - 2, kind, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    eta=pr.eta or 0.0, lazy_root=True)
    dt = torch.complex128 if pr.kind == "iti" else torch.float64
    try:
        if nrhs is None:
            u = torch.zeros(f.shape, dtype=dt, device="cuda")
            P.hps_solve(h, dev(g), u, f=None if f_solve is None else dev(f_solve))
        else:
            u = torch.zeros((nrhs,) + f.shape, dtype=dt, device="cuda")
            P.hps_solve_batched(h, nrhs, dev(G), u, f=None if F is None else dev(F))
        torch.cuda.synchronize()
        return u.cpu().numpy()
    finally:
        P.hps_free(h)


def _rand(rng, shape, cplx):
    v = rng.standard_normal(shape)
    return v + 1j * rng.standard_normal(shape) if cplx else v


@pytest.mark.parametrize("name,mk,p,L", CASES, ids=[c[0] for c in CASES])
def test_lazy_root_build_source(P, name, mk, p, L):
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    assert rel(lazy_solve(P, pr, p, inputs), oracle_solve(pr, p, L, inputs)) <= TOL


@pytest.mark.parametrize("name,mk,p,L", [CASES[0], CASES[2], CASES[4]], ids=["dtn2d", "iti", "dtn3d"])
def test_lazy_root_new_source(P, name, mk, p, L):
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    f2 = _rand(np.random.default_rng(42), inputs[5].shape, pr.kind == "iti")
    ug = lazy_solve(P, pr, p, inputs, f_solve=f2)
    assert rel(ug, oracle_solve(pr, p, L, inputs, f_override=f2)) <= TOL


@pytest.mark.parametrize("name,mk,p,L", [CASES[1], CASES[3]], ids=["dtn2d", "iti"])
def test_lazy_root_batched_matches_oracle(P, name, mk, p, L):
    """Several right-hand sides at once (boundary data and sources), each
    against its own oracle solve."""
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    rng = np.random.default_rng(7)
    cp = pr.kind == "iti"
    G = _rand(rng, (3, inputs[6].size), cp)
    F = _rand(rng, (3,) + inputs[5].shape, cp)
    U = lazy_solve(P, pr, p, inputs, nrhs=3, G=G, F=F)
    for k in range(3):
        ik = inputs[:5] + (F[k], G[k])
        assert rel(U[k], oracle_solve(pr, p, L, ik)) <= TOL


def test_lazy_root_noalloc_rejected(P):
    pr = W.poisson_poly_2d(seed=0)
    t, x, a, b, c, f, g = sample_inputs(P, pr, 8, 2)
    h = P.hps_build(t, 8, 6, P.HPS_DTN, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    lazy_root=True)
    u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        P.hps_solve_noalloc(h, dev(g), u)
    P.hps_free(h)


def test_lazy_root_full_size_helmholtz_residuals(P):
    """Benchmark workload (4096 leaves, p = 16, k = 20) with the lazy root:
    sampled composite-system residuals and agreement with the default path."""
    pr = W.helmholtz_bumps_2d(seed=1)
    p, L = 16, 6
    inputs = sample_inputs(P, pr, p, L)
    ul = lazy_solve(P, pr, p, inputs)
    t, x, a, b, c, f, g = inputs
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.choice(4096, 24, replace=False).tolist()) | {0, 4095, 1365})
    assert check_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, ul, pr.eta, sample) < 1e-10
    h = P.hps_build(t, p, p - 2, P.HPS_ITI, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    eta=pr.eta)
    u = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
    P.hps_solve(h, dev(g), u)
    torch.cuda.synchronize()
    P.hps_free(h)
    assert rel(ul, u.cpu().numpy()) <= 1e-11


@pytest.mark.parametrize("lazy", [False, True], ids=["explicit", "lazy"])
def test_graph_solve_replays_match_eager(P, lazy):
    """hps_options.graph_solve: the third and later calls replay a captured
    graph; results for changing data behind the same pointers equal eager
    solves (the graph takes the blocked triangular solves at a lazy root,
    so agreement is to roundoff, not bitwise)."""
    pr = W.helmholtz_bumps_2d(seed=1)
    p, L = 12, 3
    t, x, a, b, c, f, g = sample_inputs(P, pr, p, L)
    args = dict(a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f), eta=pr.eta, lazy_root=lazy)
    hg = P.hps_build(t, p, p - 2, P.HPS_ITI, graph_solve=True, **args)
    he = P.hps_build(t, p, p - 2, P.HPS_ITI, **args)
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(9)
    gd = torch.zeros(g.shape, dtype=torch.complex128, device="cuda")
    fd = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
    ug = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
    ue = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
    with torch.cuda.stream(stream):
        for k in range(5):
            gd.copy_(dev(_rand(rng, g.shape, True)))
            fd.copy_(dev(_rand(rng, f.shape, True)))
            P.hps_solve(hg, gd, ug, f=fd if k % 2 else None, stream=stream.cuda_stream)
            P.hps_solve(he, gd, ue, f=fd if k % 2 else None, stream=stream.cuda_stream)
            stream.synchronize()
            assert rel(ug.cpu().numpy(), ue.cpu().numpy()) <= 1e-12
    P.hps_free(hg)
    P.hps_free(he)
