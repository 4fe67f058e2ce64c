"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Bar (stated with the workloads): relative L-infinity error
max|u_gpu - u_oracle| / max|u_oracle| <= 1e-10 for float64 and complex128.
At the full benchmark sizes, where the oracle is too slow, the composite
collocation residuals of tests/residuals.py are checked on sampled leaves.
"""

import numpy as np
import pytest

import workloads as W
from oracle import hps as O
from residuals import check_dtn, check_iti

pytestmark = pytest.mark.gpu
TOL = 1e-10

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_17535_gb300 as P
    from paper_2503_17535_gb300 import _capi
    import os
    if not os.path.exists(_capi.LIB_PATH):
        from paper_2503_17535_gb300 import build
        build.build()
    return P


def rel(u, v):
    return float(np.abs(u - v).max() / np.abs(v).max())


def sample_inputs(P, pr, p, L):
    q = p - 2
    t = P.uniform_tree(pr.dim, L, pr.lo, pr.hi)
    x, xb = P.hps_nodes(t, p, q)
    nl, ppl, nr = P.hps_sizes(t, p, q)
    cf = pr.coeffs(x)
    a = cf["a"].reshape(nl, ppl)
    b = [bk.reshape(nl, ppl) for bk in cf["b"]]
    c = cf["c"].reshape(nl, ppl)
    f = pr.source(x).reshape(nl, ppl)
    g = pr.boundary(xb)
    if pr.kind == "iti":
        f = f.astype(np.complex128)
        g = g.astype(np.complex128)
    return t, x, a, b, c, f, g


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_solve(P, pr, p, L, inputs, f_solve=None, host=False, fp64_gemm=False, stats=None):
    t, x, a, b, c, f, g = inputs
    kind = P.HPS_ITI if pr.kind == "iti" else P.HPS_DTN
    if host:
        h = P.hps_build(t, p, p - 2, kind, a=a, b=b, c=c, f=f, eta=pr.eta or 0.0)
        u = np.zeros(f.shape, f.dtype)
        P.hps_solve(h, g, u, f=f_solve)
        P.hps_free(h)
        return u
    h = P.hps_build(t, p, p - 2, kind, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    eta=pr.eta or 0.0, fp64_gemm=fp64_gemm)
    if stats is not None:
        stats.update(P.hps_kernel_stats(h))
    u = torch.zeros(f.shape, dtype=torch.complex128 if pr.kind == "iti" else torch.float64,
                    device="cuda")
    P.hps_solve(h, dev(g), u, f=None if f_solve is None else dev(f_solve))
    torch.cuda.synchronize()
    P.hps_free(h)
    return u.cpu().numpy()


def oracle_solve(pr, p, L, inputs, f_override=None):
    t, x, a, b, c, f, g = inputs
    ff = f if f_override is None else f_override
    s = O.build(pr.dim, pr.kind, p, p - 2, L, pr.lo, pr.hi, a, b, c, ff, eta=pr.eta)
    return O.solve(s, g)


CASES = [
    # name, problem factory, p, L
    ("poisson2d_cfg_small", lambda: W.poisson_poly_2d(seed=0), 8, 2),
    ("poisson2d_single_leaf", lambda: W.poisson_poly_2d(seed=0), 8, 0),
    ("e1_dtn_p8_L3", W.e1_dtn_2d, 8, 3),
    ("e1_dtn_p12_L2", W.e1_dtn_2d, 12, 2),
    ("e1_dtn_p16_L1", W.e1_dtn_2d, 16, 1),
    ("helmholtz_iti_p16_L2", lambda: W.helmholtz_bumps_2d(seed=1), 16, 2),
    ("helmholtz_iti_p16_L3", lambda: W.helmholtz_bumps_2d(seed=1), 16, 3),
    ("e2_iti_p8_L3", W.e2_iti_2d, 8, 3),
    ("iti_single_leaf", W.e2_iti_2d, 10, 0),
    ("elliptic3d_p6_L1", lambda: W.elliptic_3d(seed=2), 6, 1),
    ("elliptic3d_p8_L1", lambda: W.elliptic_3d(seed=2), 8, 1),
    ("elliptic3d_p6_L2", lambda: W.elliptic_3d(seed=2), 6, 2),
    ("elliptic3d_single_leaf", lambda: W.elliptic_3d(seed=2), 8, 0),
]


@pytest.mark.parametrize("name,mk,p,L", CASES, ids=[c[0] for c in CASES])
def test_parity_against_oracle(P, name, mk, p, L):
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    ug = gpu_solve(P, pr, p, L, inputs)
    uo = oracle_solve(pr, p, L, inputs)
    assert rel(ug, uo) <= TOL, rel(ug, uo)


@pytest.mark.parametrize("name,mk,p,L", [CASES[2], CASES[6], CASES[11]], ids=[CASES[2][0], CASES[6][0], CASES[11][0]])
def test_products_on_either_pipe_match_the_oracle(P, name, mk, p, L):
    """The build's products on the tensor cores (default) and on the FP64
    pipe (fp64_gemm) both meet the parity bar; the default build really ran
    tensor-core products where they are large enough, the other none."""
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    uo = oracle_solve(pr, p, L, inputs)
    st_tc, st_fp = {}, {}
    u_tc = gpu_solve(P, pr, p, L, inputs, stats=st_tc)
    u_fp = gpu_solve(P, pr, p, L, inputs, fp64_gemm=True, stats=st_fp)
    assert rel(u_tc, uo) <= TOL, rel(u_tc, uo)
    assert rel(u_fp, uo) <= TOL, rel(u_fp, uo)
    assert st_fp["gemm_tc"]["launches"] == 0 and st_fp["split"]["launches"] == 0
    if name.startswith("helmholtz"):
        assert st_tc["gemm_tc"]["launches"] > 0 and st_tc["split"]["launches"] > 0


@pytest.mark.parametrize("name,mk,p,L", [CASES[0], CASES[5], CASES[9]], ids=["dtn2d", "iti", "dtn3d"])
def test_new_source_upward_pass(P, name, mk, p, L):
    """hps_solve with a new f runs the upward particular pass with the
    stored factors; it must equal an oracle build with that f."""
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    rng = np.random.default_rng(42)
    f2 = rng.standard_normal(inputs[5].shape)
    if pr.kind == "iti":
        f2 = f2 + 1j * rng.standard_normal(f2.shape)
    ug = gpu_solve(P, pr, p, L, inputs, f_solve=f2)
    uo = oracle_solve(pr, p, L, inputs, f_override=f2)
    assert rel(ug, uo) <= TOL


def test_host_buffers_match_device_buffers(P):
    pr = W.helmholtz_bumps_2d(seed=1)
    inputs = sample_inputs(P, pr, 16, 2)
    u1 = gpu_solve(P, pr, 16, 2, inputs)
    u2 = gpu_solve(P, pr, 16, 2, inputs, host=True)
    assert np.array_equal(u1, u2)


def test_batched_solve_equals_single_solves(P):
    pr = W.e1_dtn_2d()
    p, L = 8, 2
    t, x, a, b, c, f, g = sample_inputs(P, pr, p, L)
    h = P.hps_build(t, p, p - 2, P.HPS_DTN, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f))
    rng = np.random.default_rng(3)
    G = rng.standard_normal((3, g.size))
    F = rng.standard_normal((3,) + f.shape)
    U = torch.zeros((3,) + f.shape, dtype=torch.float64, device="cuda")
    P.hps_solve_batched(h, 3, dev(G), U, f=dev(F))
    for k in range(3):
        u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
        P.hps_solve(h, dev(G[k]), u, f=dev(F[k]))
        assert rel(U[k].cpu().numpy(), u.cpu().numpy()) < 1e-14
    P.hps_free(h)


def test_polynomial_exact_on_gpu(P):
    """u in Q_{p-3} is reproduced to roundoff by the CUDA path as well."""
    from workloads.problems import Problem, _const_coeffs
    poly = W.polynomial_field(2, 5, 77, tensor=True)
    pr = Problem("poly", 2, (-1.0, -1.0), (1.0, 1.0), "dtn", 77, _const_coeffs(2),
                 poly.lap, poly.value, poly.value)
    inputs = sample_inputs(P, pr, 8, 3)
    ug = gpu_solve(P, pr, 8, 3, inputs)
    assert rel(ug.reshape(-1), poly.value(inputs[1])) < 1e-11


def test_full_size_helmholtz_iti_residuals(P):
    """Benchmark workload (4096 leaves, p = 16, k = 20, complex128): sampled
    composite-system residuals hold at full size."""
    pr = W.helmholtz_bumps_2d(seed=1)
    p, L = 16, 6
    inputs = sample_inputs(P, pr, p, L)
    ug = gpu_solve(P, pr, p, L, inputs)
    t, x, a, b, c, f, g = inputs
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.choice(4096, 24, replace=False).tolist()) | {0, 4095, 1365})
    assert check_iti(p, L, pr.lo, pr.hi, a, b, c, f, g, ug, pr.eta, sample) < 1e-10


def test_full_size_elliptic3d_residuals(P):
    """3D workload (512 leaves, p = 8): sampled residuals hold at full size."""
    pr = W.elliptic_3d(seed=2)
    p, L = 8, 3
    inputs = sample_inputs(P, pr, p, L)
    ug = gpu_solve(P, pr, p, L, inputs)
    t, x, a, b, c, f, g = inputs
    rng = np.random.default_rng(1)
    sample = sorted(set(rng.choice(512, 16, replace=False).tolist()) | {0, 511})
    assert check_dtn(3, p, L, pr.lo, pr.hi, a, b, c, f, g, ug, sample) < 1e-10
    # the discretisation error against the manufactured solution is small too
    assert rel(ug.reshape(-1), pr.u_exact(inputs[1])) < 1e-3
