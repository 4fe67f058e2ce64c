"""Allocation failures in hps_build unwind cleanly (host-side injection).

hps_debug_fail_alloc(k) makes the k-th handle allocation fail as if cudaMalloc
had run out of memory; no device fault is involved.  For every k up to the
number of allocations a build makes, the build must return HPS_ERR_OOM,
return no handle and give its memory back, and a later build must still
produce the same solution.
"""

import numpy as np
import pytest

import workloads as W
from test_gpu_parity import dev, rel, sample_inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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
    torch.cuda.init()
    return P


def _build_solve(P, pr, p, inputs):
    t, x, a, b, c, f, g = inputs
    kind = P.HPS_ITI if pr.kind == "iti" else P.HPS_DTN
    h = P.hps_build(t, p, p - 2, kind, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    eta=pr.eta or 0.0)
    u = torch.zeros(f.shape, dtype=torch.complex128 if pr.kind == "iti" else torch.float64, device="cuda")
    P.hps_solve(h, dev(g), u)
    torch.cuda.synchronize()
    P.hps_free(h)
    return u.cpu().numpy()


@pytest.mark.parametrize("name,mk,p,L", [
    ("dtn2d", W.e1_dtn_2d, 8, 2),
    ("iti2d", W.e2_iti_2d, 8, 2),
], ids=["dtn2d", "iti2d"])
def test_every_allocation_failure_unwinds(P, name, mk, p, L):
    from paper_2503_17535_gb300 import HPSError, _capi
    pr = mk()
    inputs = sample_inputs(P, pr, p, L)
    t, x, a, b, c, f, g = inputs
    kind = P.HPS_ITI if pr.kind == "iti" else P.HPS_DTN
    ref = _build_solve(P, pr, p, inputs)
    da, db, dc, df = dev(a), [dev(bk) for bk in b], dev(c), dev(f)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n0 = P.hps_debug_alloc_count()
    h = P.hps_build(t, p, p - 2, kind, a=da, b=db, c=dc, f=df, eta=pr.eta or 0.0)
    n_alloc = P.hps_debug_alloc_count() - n0
    P.hps_free(h)
    assert n_alloc > 5
    try:
        for k in range(1, n_alloc + 1):
            P.hps_debug_fail_alloc(k)
            with pytest.raises(HPSError) as ei:
                P.hps_build(t, p, p - 2, kind, a=da, b=db, c=dc, f=df, eta=pr.eta or 0.0)
            assert ei.value.status == _capi.HPS_ERR_OOM, (k, ei.value.status)
    finally:
        P.hps_debug_fail_alloc(0)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 64 << 20
    assert rel(_build_solve(P, pr, p, inputs), ref) <= 1e-14


def test_zero_pivot_reports_singular_with_node(P):
    """All-zero coefficients make every leaf matrix zero: the panel LU records
    the zero pivot in its status word (no trap), hps_build returns
    HPS_ERR_SINGULAR without a handle, and the node is readable afterwards."""
    from paper_2503_17535_gb300 import HPSError, _capi
    pr = W.e1_dtn_2d()
    p, L = 8, 2
    t, x, a, b, c, f, g = sample_inputs(P, pr, p, L)
    z = np.zeros_like(a)
    with pytest.raises(HPSError) as ei:
        P.hps_build(t, p, p - 2, P.HPS_DTN, a=dev(z), b=[dev(z), dev(z)], c=dev(z), f=dev(f))
    assert ei.value.status == _capi.HPS_ERR_SINGULAR
    node = P.hps_last_error_detail(None)
    nl = P.hps_sizes(t, p, p - 2)[0]
    assert 0 <= node < nl + nl, node
    # the library stays usable
    assert rel(_build_solve(P, pr, p, (t, x, a, b, c, f, g)), _build_solve(P, pr, p, (t, x, a, b, c, f, g))) == 0.0
