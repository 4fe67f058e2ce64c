"""Bounded device waits give up with a status instead of hanging the GPU.

Each of the library's device-side waits -- the inter-CTA barrier of the
cooperative panel LU, the flag wait of the flag-ordered triangular solves
and the mbarrier wait of the tensor-core product pipeline -- is run by
hps_debug_wait_timeout on a word that nothing writes, with a short poll
limit: the call must report HPS_ERR_TIMEOUT, the same wait on a satisfied
word must pass, and afterwards the same device must still build and solve
correctly (the context stays usable).  No fault, trap or endless loop is
involved: the waits are bounded by construction.
"""

import time

import numpy as np
import pytest

import workloads as W
from oracle import hps as O
from test_gpu_parity import dev, rel, sample_inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WAITS = [(0, "group_barrier"), (1, "trsv_flag"), (2, "tc_mbarrier")]


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


@pytest.mark.parametrize("which,name", WAITS, ids=[w[1] for w in WAITS])
def test_wait_on_a_flag_nothing_sets_times_out(P, which, name):
    st = torch.cuda.current_stream().cuda_stream
    assert P.hps_debug_wait_timeout(which, True, 100000, st) == P.HPS_OK
    t0 = time.perf_counter()
    s = P.hps_debug_wait_timeout(which, False, 100000, st)
    dt = time.perf_counter() - t0
    assert s == P._capi.HPS_ERR_TIMEOUT, s
    assert dt < 10.0
    # the device is still usable: a build + solve after the timeouts matches the oracle
    pr = W.helmholtz_bumps_2d(seed=1)
    p, L = 8, 2
    t, x, a, b, c, f, g = sample_inputs(P, pr, p, L)
    h = P.hps_build(t, p, p - 2, P.HPS_ITI, a=dev(a), b=[dev(bk) for bk in b], c=dev(c), f=dev(f),
                    eta=pr.eta, lazy_root=True)
    u = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
    P.hps_solve(h, dev(g), u)
    torch.cuda.synchronize()
    P.hps_free(h)
    s_o = O.build(2, "iti", p, p - 2, L, pr.lo, pr.hi, a, b, c, f, eta=pr.eta)
    assert rel(u.cpu().numpy(), O.solve(s_o, g)) <= 1e-10
