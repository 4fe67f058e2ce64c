"""GPU parity of the adaptive 3D path (Section 4.2) against the adaptive
oracle: 2:1 trees with three leaf levels, a tree refined around a sharp
source by the library's own refinement (compared with the oracle's
refinement), polynomial exactness and the upward pass with a new source.
Bar: relative L-infinity error <= 1e-10."""

import numpy as np
import pytest

import workloads as W
from workloads.problems import Problem, _const_coeffs
from oracle import adaptive as ad

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


def rel(u, v):
    return float(np.abs(u - v).max() / np.abs(v).max())


def two_one_tree():
    leaves = [(1, (i, j, k)) for i in range(2) for j in range(2) for k in range(2) if (i, j, k) != (0, 0, 0)]
    leaves += ad.children_of(1, (0, 0, 0))
    leaves.remove((2, (1, 1, 1)))
    leaves += ad.children_of(2, (1, 1, 1))
    return ad.sort_leaves(ad.balance(leaves))


def d(v):
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


def gpu_solve(P, pr, leaves, p, f_solve=None, lazy=False):
    t = P.adaptive_tree(leaves, pr.lo, pr.hi)
    x, xb = P.hps_nodes(t, p, p - 2)
    nl, ppl, nr = P.hps_sizes(t, p, p - 2)
    cf = pr.coeffs(x)
    a = cf["a"].reshape(nl, ppl)
    b = [bk.reshape(nl, ppl) for bk in cf["b"]]
    c = cf["c"].reshape(nl, ppl)
    f = pr.source(x).reshape(nl, ppl)
    g = pr.boundary(xb)
    h = P.hps_build(t, p, p - 2, P.HPS_DTN, a=d(a), b=[d(bk) for bk in b], c=d(c), f=d(f), lazy_root=lazy)
    u = torch.zeros((nl, ppl), dtype=torch.float64, device="cuda")
    P.hps_solve(h, d(g), u, f=None if f_solve is None else d(f_solve))
    torch.cuda.synchronize()
    P.hps_free(h)
    return u.cpu().numpy(), (x, a, b, c, f, g)


@pytest.mark.parametrize("lazy", [False, True], ids=["explicit", "lazy"])
@pytest.mark.parametrize("p", [6, 8])
def test_adaptive_parity_two_one_tree(P, p, lazy):
    pr = W.elliptic_3d(seed=2)
    leaves = two_one_tree()
    ug, (x, a, b, c, f, g) = gpu_solve(P, pr, leaves, p, lazy=lazy)
    uo = np.array(ad.solve_adaptive(ad.build_adaptive(leaves, p, pr.lo, pr.hi, a, b, c, f), g))
    assert rel(ug, uo) <= TOL


def test_adaptive_polynomial_exact_on_gpu(P):
    p = 6
    poly = W.polynomial_field(3, p - 3, 9, tensor=True)
    pr = Problem("p3", 3, (-1.0,) * 3, (1.0,) * 3, "dtn", 9, _const_coeffs(3, c=0.7),
                 lambda x: poly.lap(x) + 0.7 * poly.value(x), poly.value, poly.value)
    leaves = two_one_tree()
    ug, inputs = gpu_solve(P, pr, leaves, p)
    assert rel(ug.reshape(-1), poly.value(inputs[0])) < 1e-11


@pytest.mark.parametrize("lazy", [False, True], ids=["explicit", "lazy"])
def test_adaptive_new_source(P, lazy):
    pr = W.elliptic_3d(seed=2)
    p = 6
    leaves = two_one_tree()
    rng = np.random.default_rng(5)
    nl = len(leaves)
    f2 = rng.standard_normal((nl, p ** 3))
    ug, (x, a, b, c, f, g) = gpu_solve(P, pr, leaves, p, f_solve=f2, lazy=lazy)
    uo = np.array(ad.solve_adaptive(ad.build_adaptive(leaves, p, pr.lo, pr.hi, a, b, c, f2), g))
    assert rel(ug, uo) <= TOL


def test_library_refinement_matches_oracle_and_solves(P):
    """hps_refine (device interpolation check + 2:1 balance) gives the same
    tree as the oracle's refinement; the solve on it matches the oracle."""
    pr = W.sharp_source_3d(seed=3, width=0.15)
    p = 6
    lib_leaves = P.hps_refine(pr.lo, pr.hi, p, 1e-3, 1, 3, [pr.source])
    orc_leaves = ad.refine([pr.source], pr.lo, pr.hi, p, 1e-3, 1, 3)
    assert [(lv, tuple(ix)) for lv, ix in lib_leaves] == [(lv, tuple(ix)) for lv, ix in orc_leaves]
    assert len(set(lv for lv, _ in lib_leaves)) >= 2
    prob = W.elliptic_3d(seed=2)
    ug, (x, a, b, c, f, g) = gpu_solve(P, prob, lib_leaves, p)
    uo = np.array(ad.solve_adaptive(ad.build_adaptive(lib_leaves, p, prob.lo, prob.hi, a, b, c, f), g))
    assert rel(ug, uo) <= TOL


def test_uniform_octree_through_adaptive_path(P):
    """A uniform depth-2 octree given as an adaptive leaf list equals the
    uniform path."""
    pr = W.elliptic_3d(seed=2)
    p = 6
    leaves = ad.sort_leaves([(2, (i, j, k)) for i in range(4) for j in range(4) for k in range(4)])
    ua, _ = gpu_solve(P, pr, leaves, p)
    t = P.uniform_tree(3, 2, pr.lo, pr.hi)
    x, xb = P.hps_nodes(t, p, p - 2)
    cf = pr.coeffs(x)
    h = P.hps_build(t, p, p - 2, P.HPS_DTN, a=d(cf["a"].reshape(64, -1)),
                    b=[d(bk.reshape(64, -1)) for bk in cf["b"]], c=d(cf["c"].reshape(64, -1)),
                    f=d(pr.source(x).reshape(64, -1)))
    u = torch.zeros((64, p ** 3), dtype=torch.float64, device="cuda")
    P.hps_solve(h, d(pr.boundary(xb)), u)
    torch.cuda.synchronize()
    P.hps_free(h)
    assert rel(ua, u.cpu().numpy()) <= TOL


def test_adaptive_workload_full_size(P):
    """Workload 3b at full size: the operator of the 3D workload with a sharp
    seeded source, tree from hps_refine (eps 1e-4, depths 2..5); parity with
    the oracle on the same tree (the oracle takes about a minute here)."""
    pr = W.adaptive_3d()
    p = 8
    fa = lambda x: pr.coeffs(x)["a"]  # noqa: E731
    fc = lambda x: pr.coeffs(x)["c"]  # noqa: E731
    leaves = P.hps_refine(pr.lo, pr.hi, p, 1e-4, 2, 5, [pr.source, fa, fc])
    assert sorted(set(lv for lv, _ in leaves)) == [2, 3, 4, 5]
    ug, (x, a, b, c, f, g) = gpu_solve(P, pr, leaves, p)
    uo = np.array(ad.solve_adaptive(ad.build_adaptive(leaves, p, pr.lo, pr.hi, a, b, c, f), g))
    assert rel(ug, uo) <= TOL
