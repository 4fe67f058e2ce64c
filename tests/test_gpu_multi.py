"""Apply-only solves of several different operators in shared launches
(hps_solve_multi): 2D DtN, 2D ItI and 3D DtN operators of different depths
and orders, explicit and lazy roots, one or two right-hand sides each, solved
together.  Every result must equal the operator's own hps_solve to 1e-12 and
the oracle to 1e-10."""

import numpy as np
import pytest

import workloads as W
from oracle import hps as O
from test_gpu_parity import P, dev, rel, sample_inputs  # noqa: F401

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OPS = [  # name, problem, p, L, lazy root, right-hand sides
    ("dtn2d_p8_L2", lambda: W.e1_dtn_2d(), 8, 2, False, 2),
    ("iti_p12_L3_lazy", lambda: W.helmholtz_bumps_2d(seed=1), 12, 3, True, 1),
    ("dtn3d_p6_L1", lambda: W.elliptic_3d(seed=2), 6, 1, False, 1),
    ("iti_p16_L2", lambda: W.helmholtz_bumps_2d(seed=1), 16, 2, False, 2),
    ("dtn2d_p12_L3_lazy", lambda: W.elliptic_2d(seed=4), 12, 3, True, 1),
    ("iti_p8_L0", lambda: W.e2_iti_2d(), 8, 0, False, 1),
]


def _build(P, pr, p, inputs, lazy):
    t, x, a, b, c, f, g = inputs
    kind = P.HPS_ITI if pr.kind == "iti" else P.HPS_DTN
    return P.hps_build(t, p, p - 2, kind, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                       eta=pr.eta or 0.0, lazy_root=lazy)


def test_multi_operator_solve_matches_single_and_oracle(P):
    rng = np.random.default_rng(9)
    hs, gs, us, refs, nr, oracle = [], [], [], [], [], []
    for name, mk, p, L, lazy, k in OPS:
        pr = mk()
        inputs = sample_inputs(P, pr, p, L)
        t, x, a, b, c, f, g = inputs
        cp = pr.kind == "iti"
        G = np.stack([g] + [g * (1.0 + 0.5 * j) + rng.standard_normal(g.shape) * (1j if cp else 1.0)
                            for j in range(1, k)])
        h = _build(P, pr, p, inputs, lazy)
        dt = torch.complex128 if cp else torch.float64
        U = torch.zeros((k,) + f.shape, dtype=dt, device="cuda")
        R = torch.zeros((k,) + f.shape, dtype=dt, device="cuda")
        P.hps_solve_batched(h, k, dev(G), R)
        hs.append(h); gs.append(dev(G)); us.append(U); refs.append(R); nr.append(k)
        s = O.build(pr.dim, pr.kind, p, p - 2, L, pr.lo, pr.hi, a, b, c, f, eta=pr.eta)
        oracle.append([O.solve(s, G[j]) for j in range(k)])
    P.hps_solve_multi(hs, gs, us, nrhs=nr)
    # a second round reuses the workspaces
    P.hps_solve_multi(hs, gs, us, nrhs=nr)
    torch.cuda.synchronize()
    for i, (name, *_rest) in enumerate(OPS):
        U = us[i].cpu().numpy()
        R = refs[i].cpu().numpy()
        assert rel(U, R) <= 1e-12, (name, rel(U, R))
        for j in range(nr[i]):
            assert rel(U[j], oracle[i][j]) <= 1e-10, (name, j, rel(U[j], oracle[i][j]))
    for h in hs:
        P.hps_free(h)


def test_multi_operator_solve_rejects_bad_arguments(P):
    pr = W.e1_dtn_2d()
    inputs = sample_inputs(P, pr, 8, 1)
    h = _build(P, pr, 8, inputs, False)
    g = dev(inputs[6])
    u = torch.zeros(inputs[5].shape, dtype=torch.float64, device="cuda")
    from paper_2503_17535_gb300 import HPSError
    with pytest.raises(HPSError):
        P.hps_solve_multi([h, h], [g, g], [u, u])          # repeated handle
    with pytest.raises(HPSError):
        P.hps_solve_multi([h], [inputs[6]], [u])            # host g
    P.hps_free(h)
