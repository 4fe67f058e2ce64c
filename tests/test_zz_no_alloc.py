"""hps_solve_noalloc: the allocation-free solve for callers that cannot let
the library allocate device memory at solve time (memory owned by another
allocator, or code that must not synchronise the device through
cudaMalloc / cudaFree).  It is checked through the C ABI against hps_solve,
the existing entry point, on two calls in a row (the static scratch array
keeps the previous call's contents, so the second call must not depend on
them).  This file is collected last so that a failure here stops a
first-failure run only after every other test has run."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-10


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    import paper_2503_17535_gb300 as P
    from paper_2503_17535_gb300 import _capi
    if not os.path.exists(_capi.LIB_PATH):
        from paper_2503_17535_gb300 import build
        build.build()
    return P


def _build(P, pr, p, L):
    q = p - 2
    t = P.uniform_tree(pr.dim, L, pr.lo, pr.hi)
    x, xb = P.hps_nodes(t, p, q)
    nl, ppl, nr = P.hps_sizes(t, p, q)
    cf = pr.coeffs(x)
    cdt = np.complex128 if pr.kind == "iti" else np.float64
    d = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()  # noqa: E731
    kind = P.HPS_ITI if pr.kind == "iti" else P.HPS_DTN
    h = P.hps_build(t, p, q, kind, a=d(cf["a"].reshape(nl, ppl)),
                    b=[d(bk.reshape(nl, ppl)) for bk in cf["b"]], c=d(cf["c"].reshape(nl, ppl)),
                    f=d(pr.source(x).reshape(nl, ppl).astype(cdt)), eta=pr.eta or 0.0)
    g = d(pr.boundary(xb).astype(cdt))
    return h, g, (nl, ppl), torch.complex128 if pr.kind == "iti" else torch.float64


@pytest.mark.parametrize("name,mk,p,L", [
    ("helmholtz_iti_p16_L3", lambda: W.helmholtz_bumps_2d(seed=1), 16, 3),
    ("poisson_dtn_p8_L2", lambda: W.poisson_poly_2d(seed=0), 8, 2),
    ("elliptic3d_p6_L2", lambda: W.elliptic_3d(seed=2), 6, 2),
])
def test_noalloc_matches_hps_solve_twice(P, name, mk, p, L):
    h, g, shape, dt = _build(P, mk(), p, L)
    ref = torch.zeros(shape, dtype=dt, device="cuda")
    P.hps_solve(h, g, ref)
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    for _ in range(2):
        u = torch.full(shape, float("nan"), dtype=dt, device="cuda")
        P.hps_solve_noalloc(h, g, u)
        torch.cuda.synchronize()
        err = float(np.abs(u.cpu().numpy() - r).max() / np.abs(r).max())
        assert err <= TOL, err
    P.hps_free(h)


def test_noalloc_rejects_host_buffers(P):
    h, g, shape, dt = _build(P, W.poisson_poly_2d(seed=0), 8, 1)
    with pytest.raises(P.HPSError) as e:
        P.hps_solve_noalloc(h, g.cpu().numpy(), torch.zeros(shape, dtype=dt, device="cuda"))
    assert e.value.status == -1
    P.hps_free(h)


def test_noalloc_rejects_problems_beyond_the_static_array(P):
    """A 2D DtN tree of depth 7 at p = 16 needs about 18 MB of downward-pass
    vectors, more than the 16 MiB array: refused, nothing launched."""
    pr = W.poisson_poly_2d(seed=0)
    h, g, shape, dt = _build(P, pr, 16, 7)
    with pytest.raises(P.HPSError) as e:
        P.hps_solve_noalloc(h, g, torch.zeros(shape, dtype=dt, device="cuda"))
    assert e.value.status == -1
    P.hps_free(h)
