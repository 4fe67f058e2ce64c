"""GPU tests of the request server (include/hps_serve.h).

The server must return, for every request, the same solution as the plain
path (hps_build + hps_solve of the same operator, one request at a time)
and as the oracle, within the parity bar (relative L-infinity <= 1e-10),
whatever batches, operator groups and streams the request shared; builds are
admitted by device footprint.
"""

import numpy as np
import pytest

import workloads as W
from oracle import hps as O
from test_gpu_parity import TOL, rel, sample_inputs

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


def _problem(P, mk, p, L):
    pr = mk()
    t, x, a, b, c, f, g = sample_inputs(P, pr, p, L)
    cc = np.ascontiguousarray
    a, b, c, f, g = cc(a), [cc(bk) for bk in b], cc(c), cc(f), cc(g)
    kind = P.HPS_ITI if pr.kind == "iti" else P.HPS_DTN
    return dict(pr=pr, t=t, p=p, L=L, kind=kind, a=a, b=b, c=c, f=f, g=g, eta=pr.eta or 0.0)


def _rand_like(rng, x):
    v = rng.standard_normal(x.shape)
    if np.iscomplexobj(x):
        v = v + 1j * rng.standard_normal(x.shape)
    return np.ascontiguousarray(v)


def _alone(P, op, g, f):
    """The plain path: its own build, then one solve."""
    h = P.hps_build(op["t"], op["p"], op["p"] - 2, op["kind"], a=op["a"], b=op["b"], c=op["c"], f=op["f"],
                    eta=op["eta"])
    u = np.zeros(op["f"].shape, op["f"].dtype)
    P.hps_solve(h, g, u, f=f)
    P.hps_free(h)
    return u


_ORACLE_OPS = {}


def _oracle(op, g, f):
    """The oracle's u for the operator's coefficients, boundary data g and
    source f (the build-time source when f is None)."""
    pr = op["pr"]
    key = (id(op), None if f is None else f.tobytes())
    if key not in _ORACLE_OPS:
        _ORACLE_OPS[key] = O.build(pr.dim, pr.kind, op["p"], op["p"] - 2, op["L"], pr.lo, pr.hi, op["a"],
                                   op["b"], op["c"], op["f"] if f is None else f, eta=pr.eta)
    return O.solve(_ORACLE_OPS[key], g)


def _submit_build(S, slot, op):
    return S.submit_build(slot, op["t"], op["p"], op["p"] - 2, op["kind"], a=op["a"], b=op["b"], c=op["c"],
                          f=op["f"], eta=op["eta"])


def test_results_same_alone_and_in_mix(P):
    ops = [
        _problem(P, W.e1_dtn_2d, 8, 3),
        _problem(P, W.e2_iti_2d, 8, 2),
        _problem(P, lambda: W.poisson_poly_2d(seed=0), 12, 2),
        _problem(P, lambda: W.elliptic_3d(seed=2), 6, 1),
    ]
    rebuilt = _problem(P, lambda: W.helmholtz_bumps_2d(seed=5), 8, 2)
    rng = np.random.default_rng(123)
    reqs = []  # (ticket, op dict, g, f, u)
    with P.Server(n_slots=4, n_streams=3, max_batch=4) as S:
        builds = [_submit_build(S, i, op) for i, op in enumerate(ops)]
        for k in range(40):
            if k == 20:
                builds.append(_submit_build(S, 1, rebuilt))
            slot = int(rng.integers(0, 4))
            op = rebuilt if (slot == 1 and k >= 20) else ops[slot]
            g = _rand_like(rng, op["g"])
            f = _rand_like(rng, op["f"]) if rng.random() < 0.4 else None
            u = np.zeros(op["f"].shape, op["f"].dtype)
            reqs.append((S.submit_solve(slot, g, u, f=f), op, g, f, u))
        infos = [S.wait(t, check=False) for t, *_ in reqs]
        binfos = [S.wait(t, check=False) for t in builds]
        st = S.stats()
    assert all(i["status"] == 0 for i in binfos), binfos
    assert all(i["status"] == 0 for i in infos), [(t, i) for (t, *_), i in zip(reqs, infos) if i["status"]]
    assert st["solves"] == 40 and st["builds"] == 5
    assert max(i["batch"] for i in infos) >= 2, "no request was batched"
    for (t, op, g, f, u), info in zip(reqs, infos):
        assert info["status"] == 0
        ua = _alone(P, op, g, f)
        assert rel(u, ua) <= TOL, (info, rel(u, ua))
        uo = _oracle(op, g, f)
        assert rel(u, uo) <= TOL, (info, rel(u, uo))


def test_apply_only_solves_of_different_operators_share_launches(P):
    """Apply-only requests queued on operators of different kinds, depths
    and orders are served by one grouped solve; each result equals the
    oracle's and the plain path's."""
    ops = [
        _problem(P, W.e1_dtn_2d, 8, 3),
        _problem(P, W.e2_iti_2d, 12, 2),
        _problem(P, lambda: W.elliptic_3d(seed=2), 6, 1),
        _problem(P, lambda: W.helmholtz_bumps_2d(seed=1), 16, 2),
        _problem(P, lambda: W.poisson_poly_2d(seed=0), 8, 0),
    ]
    rng = np.random.default_rng(77)
    with P.Server(n_slots=len(ops), n_streams=1, max_batch=3, max_group=8) as S:
        for t in [_submit_build(S, i, op) for i, op in enumerate(ops)]:
            S.wait(t)
        reqs = []
        for k in range(30):
            slot = k % len(ops)
            op = ops[slot]
            g = _rand_like(rng, op["g"])
            u = np.zeros(op["f"].shape, op["f"].dtype)
            reqs.append((S.submit_solve(slot, g, u), op, g, u))
        infos = [S.wait(t) for t, *_ in reqs]
        st = S.stats()
    assert st["multi_batches"] >= 1 and st["max_group_seen"] >= 2, st
    for (t, op, g, u), info in zip(reqs, infos):
        assert info["status"] == 0
        assert rel(u, _alone(P, op, g, None)) <= TOL
        assert rel(u, _oracle(op, g, None)) <= TOL


def test_queued_solves_share_one_batch(P):
    op = _problem(P, W.e1_dtn_2d, 8, 2)
    rng = np.random.default_rng(5)
    with P.Server(n_slots=1, n_streams=2, max_batch=8) as S:
        _submit_build(S, 0, op)
        gs = [_rand_like(rng, op["g"]) for _ in range(8)]
        us = [np.zeros(op["f"].shape) for _ in range(8)]
        ts = [S.submit_solve(0, g, u) for g, u in zip(gs, us)]
        infos = [S.wait(t) for t in ts]
    assert all(i["batch"] == 8 for i in infos)
    for g, u in zip(gs, us):
        assert rel(u, _alone(P, op, g, None)) <= TOL


def test_build_beyond_budget_is_refused(P):
    op = _problem(P, W.e1_dtn_2d, 8, 2)
    assert P.hps_plan_bytes(op["t"], 8, 6, P.HPS_DTN) > 1 << 16
    with P.Server(n_slots=1, n_streams=1, max_batch=1, hbm_budget=1 << 16) as S:
        t = _submit_build(S, 0, op)
        info = S.wait(t, check=False)
        assert info["status"] == -2  # HPS_ERR_OOM
        u = np.zeros(op["f"].shape)
        t2 = S.submit_solve(0, op["g"], u)
        assert S.wait(t2, check=False)["status"] == -1  # no operator in the slot


def test_server_operator_matches_plain_build(P):
    op = _problem(P, W.e2_iti_2d, 8, 2)
    with P.Server(n_slots=2) as S:
        S.wait(_submit_build(S, 1, op))
        h = S.operator(1)
        assert S.operator(0) is None
        u = np.zeros(op["f"].shape, op["f"].dtype)
        P.hps_solve(h, op["g"], u)
        assert rel(u, _alone(P, op, op["g"], None)) <= TOL
