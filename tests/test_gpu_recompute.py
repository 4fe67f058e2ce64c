"""Subtree recomputation under a device-memory budget (Section 4.1,
Algorithm "our_recomputation", on the device).

A build whose planned footprint exceeds hps_options.recompute_budget_mb
keeps only the merges above the largest complete subtrees that fit and the
subtrees' root maps; every solve rebuilds the subtrees.  The results must
equal the unbudgeted build's (the same operations, rounding aside) and the
oracle's (relative L-infinity <= 1e-10), the handle must hold fewer device
bytes, and a budget no subtree depth fits is refused with HPS_ERR_OOM.
"""

import numpy as np
import pytest

import workloads as W
from oracle import hps as O
from test_gpu_parity import P, TOL, dev, rel, sample_inputs  # noqa: F401

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [  # name, problem, p, L, lazy root, budget as a fraction of the plain plan
    ("dtn2d_p8_L4", W.e1_dtn_2d, 8, 4, False, 0.52),
    ("iti_p12_L4_lazy", lambda: W.helmholtz_bumps_2d(seed=1), 12, 4, True, 0.35),
    ("dtn3d_p6_L2", lambda: W.elliptic_3d(seed=2), 6, 2, False, 0.9),
]


def _build(P, pr, p, inputs, **kw):
    t, x, a, b, c, f, g = inputs
    kind = P.HPS_ITI if pr.kind == "iti" else P.HPS_DTN
    return P.hps_build(t, p, p - 2, kind, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                       eta=pr.eta or 0.0, **kw)


@pytest.mark.parametrize("name,mk,p,L,lazy,frac", CASES, ids=[c[0] for c in CASES])
def test_recomputed_solves_match_plain_and_oracle(P, name, mk, p, L, lazy, frac):
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    t, x, a, b, c, f, g = inputs
    cp = pr.kind == "iti"
    kind = P.HPS_ITI if cp else P.HPS_DTN
    dt = torch.complex128 if cp else torch.float64
    plan = P.hps_plan_bytes(t, p, p - 2, kind)
    budget_mb = max(1, int(frac * plan) >> 20)
    h0 = _build(P, pr, p, inputs, lazy_root=lazy)
    h1 = _build(P, pr, p, inputs, lazy_root=lazy, recompute_budget_mb=budget_mb)
    b0, b1 = P.hps_device_bytes(h0), P.hps_device_bytes(h1)
    assert b1 < b0 and b1 <= budget_mb << 20, (b0, b1, budget_mb)
    rng = np.random.default_rng(17)
    z = (lambda s: rng.standard_normal(s) + 1j * rng.standard_normal(s)) if cp else rng.standard_normal
    G = np.stack([g, z(g.shape)])
    F2 = z(f.shape)
    outs = []
    for h in (h0, h1):
        u = torch.zeros((2,) + f.shape, dtype=dt, device="cuda")
        P.hps_solve_batched(h, 2, dev(G), u)                 # build-time source, two right-hand sides
        un = torch.zeros(f.shape, dtype=dt, device="cuda")
        P.hps_solve(h, dev(G[1]), un, f=dev(F2))             # a new source through the upward pass
        uh = np.zeros(f.shape, f.dtype if cp else np.float64)
        P.hps_solve(h, G[0], uh)                             # host buffers
        torch.cuda.synchronize()
        outs.append((u.cpu().numpy(), un.cpu().numpy(), uh))
    # the subtree builds batch fewer leaves, so some of their products and
    # factorisations take other (equally valid) paths: equal up to rounding
    for k in range(3):
        assert rel(outs[1][k], outs[0][k]) <= TOL, (k, rel(outs[1][k], outs[0][k]))
    s_b = O.build(pr.dim, pr.kind, p, p - 2, L, pr.lo, pr.hi, a, b, c, f, eta=pr.eta)
    s_n = O.build(pr.dim, pr.kind, p, p - 2, L, pr.lo, pr.hi, a, b, c, F2, eta=pr.eta)
    assert rel(outs[1][0][0], O.solve(s_b, G[0])) <= TOL
    assert rel(outs[1][0][1], O.solve(s_b, G[1])) <= TOL
    assert rel(outs[1][1], O.solve(s_n, G[1])) <= TOL
    print(f"{name}: plain {b0 / 2**20:.1f} MiB, recomputing {b1 / 2**20:.1f} MiB (budget {budget_mb} MiB), "
          f"saved {(b0 - b1) / 2**20:.1f} MiB")
    P.hps_free(h0)
    P.hps_free(h1)


def test_budget_no_subtree_fits_is_refused(P):
    from paper_2503_17535_gb300 import HPSError, _capi
    pr = W.e1_dtn_2d()
    inputs = sample_inputs(P, pr, 8, 3)
    with pytest.raises(HPSError) as ei:
        _build(P, pr, 8, inputs, recompute_budget_mb=1)
    assert ei.value.status == _capi.HPS_ERR_OOM


def test_recomputing_handle_refuses_other_entry_points(P):
    from paper_2503_17535_gb300 import HPSError
    pr = W.e1_dtn_2d()
    inputs = sample_inputs(P, pr, 8, 4)
    t = inputs[0]
    budget_mb = max(1, int(0.52 * P.hps_plan_bytes(t, 8, 6, P.HPS_DTN)) >> 20)
    h = _build(P, pr, 8, inputs, recompute_budget_mb=budget_mb)
    f = inputs[5]
    u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(HPSError):
        P.hps_solve_adjoint(h, dev(np.ones(f.shape)), torch.zeros_like(dev(inputs[6])), torch.zeros_like(u))
    with pytest.raises(HPSError):
        P.hps_solve_noalloc(h, dev(inputs[6]), u)
    P.hps_free(h)


def test_benchmark_operator_under_a_budget(P):
    """The Helmholtz benchmark operator (4096 leaves, p = 16, complex128)
    built under a 4 GiB budget: its solve equals the unbudgeted one within
    the rounding floor of this operator at depth 6 (two FP64 builds that
    round the leaf operators differently differ by up to ~6e-10 there; the
    element-wise oracle parity test of this operator measures that floor),
    held here to 2e-9."""
    pr = W.helmholtz_bumps_2d(seed=1)
    p, L = 16, 6
    inputs = sample_inputs(P, pr, p, L)
    t, x, a, b, c, f, g = inputs
    h0 = _build(P, pr, p, inputs, lazy_root=True)
    h1 = _build(P, pr, p, inputs, lazy_root=True, recompute_budget_mb=4096)
    assert P.hps_device_bytes(h1) <= 4096 << 20 < P.hps_device_bytes(h0)
    us = []
    for h in (h0, h1):
        u = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
        P.hps_solve(h, dev(g), u)
        torch.cuda.synchronize()
        us.append(u.cpu().numpy())
    print(f"helmholtz depth 6: recomputing vs plain {rel(us[1], us[0]):.2e}")
    assert rel(us[1], us[0]) <= 2e-9, rel(us[1], us[0])
    print(f"helmholtz depth 6: plain {P.hps_device_bytes(h0) / 2**30:.2f} GiB, "
          f"recomputing {P.hps_device_bytes(h1) / 2**30:.2f} GiB")
    P.hps_free(h0)
    P.hps_free(h1)
