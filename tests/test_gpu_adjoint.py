"""GPU adjoint solve and coefficient gradients against the oracle adjoint
(dense composite system), the adjoint identity at larger sizes, and the
differentiation workload (Helmholtz, 1024 leaves, p = 16, theta on
a 64 x 64 grid) against central finite differences through the
torch.autograd.Function."""

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA
from test_gpu_parity import P, dev, rel, sample_inputs  # noqa: F401

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-10

SMALL = [
    ("dtn2d_L1", lambda: W.elliptic_2d(seed=4), 6, 1),
    ("dtn2d_L2", lambda: W.elliptic_2d(seed=4), 8, 2),
    ("iti_L1", lambda: W.helmholtz_bumps_2d(seed=1), 8, 1),
    ("iti_L2", lambda: W.helmholtz_bumps_2d(seed=1), 8, 2),
    ("dtn3d_L1", lambda: W.elliptic_3d(seed=2), 6, 1),
]


def _gpu_adjoint(P, pr, p, inputs, ubar, lazy=False):
    t, x, a, b, c, f, g = inputs
    cp = pr.kind == "iti"
    kind = P.HPS_ITI if cp else P.HPS_DTN
    dt = torch.complex128 if cp else torch.float64
    h = P.hps_build(t, p, p - 2, kind, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    eta=pr.eta or 0.0, lazy_root=lazy)
    u = torch.zeros(f.shape, dtype=dt, device="cuda")
    P.hps_solve(h, dev(g), u, f=dev(f))
    gbar = torch.zeros(g.shape, dtype=dt, device="cuda")
    fbar = torch.zeros(f.shape, dtype=dt, device="cuda")
    P.hps_solve_adjoint(h, dev(ubar), gbar, fbar)
    gc = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    P.hps_coeff_gradient(h, u, fbar, gc=gc)
    torch.cuda.synchronize()
    P.hps_free(h)
    return gbar.cpu().numpy(), fbar.cpu().numpy(), gc.cpu().numpy(), u.cpu().numpy()


@pytest.mark.parametrize("lazy", [False, True], ids=["explicit", "lazy"])
@pytest.mark.parametrize("name,mk,p,L", SMALL, ids=[c[0] for c in SMALL])
def test_adjoint_matches_oracle_adjoint(P, name, mk, p, L, lazy):
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    t, x, a, b, c, f, g = inputs
    cp = pr.kind == "iti"
    rng = np.random.default_rng(3)
    ubar = rng.standard_normal(f.shape) + (1j * rng.standard_normal(f.shape) if cp else 0.0)
    gb, fb, gc, u = _gpu_adjoint(P, pr, p, inputs, ubar, lazy=lazy)
    if cp:
        og, of, oc, ou = OA.adjoint_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, ubar, pr.eta)
    else:
        og, of, oc, ou = OA.adjoint_dtn(pr.dim, p, L, pr.lo, pr.hi, a, b, c, f, g, ubar, with_gbar=pr.dim == 2)
    assert rel(u, ou) <= TOL
    if og is not None:
        assert rel(gb, og) <= TOL, rel(gb, og)
    assert rel(fb, of) <= TOL, rel(fb, of)
    assert rel(gc, oc) <= TOL, rel(gc, oc)


@pytest.mark.parametrize("lazy", [False, True], ids=["explicit", "lazy"])
@pytest.mark.parametrize("name,mk,p,L", [
    ("dtn2d", W.e1_dtn_2d, 12, 3),
    ("iti", lambda: W.helmholtz_bumps_2d(seed=1), 16, 3),
    ("dtn3d", lambda: W.elliptic_3d(seed=2), 6, 2),
], ids=["dtn2d", "iti", "dtn3d"])
def test_adjoint_identity_two_rhs(P, name, mk, p, L, lazy):
    """Re<ubar, u(g, f)> = Re<gbar, g> + Re<fbar, f> for two columns at once."""
    pr = mk()
    t, x, a, b, c, f, g = sample_inputs(P, pr, p, L)
    cp = pr.kind == "iti"
    kind = P.HPS_ITI if cp else P.HPS_DTN
    dt = torch.complex128 if cp else torch.float64
    h = P.hps_build(t, p, p - 2, kind, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    eta=pr.eta or 0.0, lazy_root=lazy)
    rng = np.random.default_rng(5)
    z = (lambda s: rng.standard_normal(s) + 1j * rng.standard_normal(s)) if cp else rng.standard_normal
    G, F, UB = z((2, g.size)), z((2,) + f.shape), z((2,) + f.shape)
    U = torch.zeros((2,) + f.shape, dtype=dt, device="cuda")
    P.hps_solve_batched(h, 2, dev(G), U, f=dev(F))
    GB = torch.zeros((2, g.size), dtype=dt, device="cuda")
    FB = torch.zeros((2,) + f.shape, dtype=dt, device="cuda")
    P.hps_solve_adjoint(h, dev(UB), GB, FB, nrhs=2)
    torch.cuda.synchronize()
    P.hps_free(h)
    U, GB, FB = U.cpu().numpy(), GB.cpu().numpy(), FB.cpu().numpy()
    for k in range(2):
        lhs = np.real(np.vdot(UB[k], U[k]))
        rhs = np.real(np.vdot(GB[k], G[k])) + np.real(np.vdot(FB[k], F[k]))
        assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs)), (lhs, rhs)


def test_differentiation_workload_matches_finite_differences(P):
    """Helmholtz coefficient fit: J(theta) = ||u(theta) - u(theta_true)||^2, 1024 leaves,
    p = 16, complex128; autograd gradient (adjoint kernels) against central
    differences (h = 1e-6) on 16 seeded grid entries and one seeded direction."""
    from paper_2503_17535_gb300.autograd import hps_solve_fn
    d = W.helmholtz_theta_2d(seed=5)
    pr, k = d["problem"], d["k"]
    p, L = 16, 5
    t = P.uniform_tree(2, L, pr.lo, pr.hi)
    x, xb = P.hps_nodes(t, p, p - 2)
    nl, ppl, nr = P.hps_sizes(t, p, p - 2)
    I = W.grid_interp_matrix(x, d["n"]).tocoo()
    Imat = torch.sparse_coo_tensor(np.vstack([I.row, I.col]), I.data, I.shape, dtype=torch.float64,
                                   device="cuda")
    f = dev(pr.source(x).reshape(nl, ppl).astype(np.complex128))
    g = dev(pr.boundary(xb).astype(np.complex128))

    def forward(theta):
        c = (k ** 2 * (1.0 - torch.sparse.mm(Imat, theta[:, None])[:, 0])).reshape(nl, ppl)
        return hps_solve_fn(c, g, f, t, p, P.HPS_ITI, eta=pr.eta)

    with torch.no_grad():
        u_obs = forward(dev(d["theta_true"]))
    theta = dev(d["theta_0"]).requires_grad_(True)
    J = ((forward(theta) - u_obs).abs() ** 2).sum()
    J.backward()
    grad = theta.grad.detach().cpu().numpy()

    def Jval(th):
        with torch.no_grad():
            return float(((forward(dev(th)) - u_obs).abs() ** 2).sum().item())

    th0 = d["theta_0"]
    J0 = Jval(th0)
    scale = np.abs(grad).max()
    assert scale > 0

    def fd(v, h):
        return (Jval(th0 + h * v) - Jval(th0 - h * v)) / (2 * h)

    # Central differences carry the solver's rounding (relative ~1e-11 of J,
    # deterministic in theta but not smooth) divided by h: at h = 1e-6 that
    # floor is ~1e-5 |J| per unit of theta, so the check there allows it; at
    # h = 1e-4 the floor is 100x lower and the truncation error O(h^2) is
    # still negligible, so the agreement must be tight.
    for j in d["probe"]:
        e = np.zeros_like(th0)
        e[j] = 1.0
        assert abs(fd(e, 1e-6) - grad[j]) <= 1e-10 * abs(J0) / 1e-6 + 1e-6 * scale, (j, grad[j])
        assert abs(fd(e, 1e-4) - grad[j]) <= 1e-10 * abs(J0) / 1e-4 + 1e-6 * scale, (j, grad[j])
    v = d["direction"]
    ad = float(grad @ v)
    assert abs(fd(v, 1e-6) - ad) <= 1e-10 * abs(J0) / 1e-6 + 1e-6 * scale
    assert abs(fd(v, 1e-4) - ad) <= 1e-10 * abs(J0) / 1e-4 + 1e-6 * scale, (fd(v, 1e-4), ad, J0)


@pytest.mark.parametrize("name,mk,p,L", [SMALL[2], SMALL[1]], ids=["iti_L1", "dtn2d_L2"])
def test_autograd_backward_twice_reuses_the_factors(P, name, mk, p, L):
    """Two backward passes through one graph (retain_graph=True, then
    torch.autograd.grad) reuse the handle built in forward; both coefficient
    gradients of J = Re<ubar, u> equal the oracle adjoint's."""
    from paper_2503_17535_gb300.autograd import hps_solve_fn
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    t, x, a, b, c, f, g = inputs
    cp = pr.kind == "iti"
    rng = np.random.default_rng(7)
    ubar = rng.standard_normal(f.shape) + (1j * rng.standard_normal(f.shape) if cp else 0.0)
    if cp:
        _, _, oc, _ = OA.adjoint_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, ubar, pr.eta)
    else:
        _, _, oc, _ = OA.adjoint_dtn(pr.dim, p, L, pr.lo, pr.hi, a, b, c, f, g, ubar, with_gbar=False)
    cd = dev(c).requires_grad_(True)
    u = hps_solve_fn(cd, dev(g), dev(f), t, p, P.HPS_ITI if cp else P.HPS_DTN, a=dev(a),
                     b=[dev(bk) for bk in b], eta=pr.eta or 0.0)
    J = (torch.conj(dev(ubar)) * u).real.sum()
    J.backward(retain_graph=True)
    g1 = cd.grad.detach().cpu().numpy().copy()
    (g2,) = torch.autograd.grad(J, cd)
    g2 = g2.detach().cpu().numpy()
    assert rel(g1, oc) <= TOL, rel(g1, oc)
    assert rel(g2, oc) <= TOL, rel(g2, oc)
