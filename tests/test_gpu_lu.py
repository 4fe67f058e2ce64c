"""The batched LU with partial pivoting (hps_getrf) against LAPACK.

Every merge of the build factors D (Sec. 3.3) and every leaf factors its
local operator (Sec. 2.2-2.3) with this routine; the paper leaves both to its
library.  Here it is run alone through the C ABI and compared with LAPACK's
getrf (scipy.linalg.lu_factor):

* the interchanges must be identical -- the same pivot in every column,
  including exact ties, which both break by the lowest position in the row
  order reached so far;
* the factors must agree to the rounding floor of the factorisation: the
  bar is max(1e-12, 8 x the difference between LAPACK's factors of A and of A
  with every entry perturbed by one rounding unit), relative to max |LU|.

The shapes exercise each panel path: one CTA per matrix (large batches), a
thread-block cluster per matrix (few, tall matrices: the merges near the
root, up to the 6912-row root of the 3D workload), and the cooperative
kernel used when the cluster form is switched off.
"""

import numpy as np
import pytest
import scipy.linalg as sla

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
    return P


def random_batch(n, batch, cplx, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((batch, n, n))
    if cplx:
        A = A + 1j * rng.standard_normal((batch, n, n))
    return A


def gpu_lu(P, A, mode):
    """A: (batch, n, n) numpy, row-major items; returns (LU items, ipiv, info)
    in the same layout."""
    At = torch.from_numpy(np.ascontiguousarray(np.transpose(A, (0, 2, 1)))).cuda()  # column-major items
    _, ipiv, info = P.hps_getrf(At, mode=mode)
    LU = np.transpose(At.cpu().numpy(), (0, 2, 1))
    return LU, ipiv.cpu().numpy(), info.cpu().numpy()


def lapack_lu(a):
    lu, piv = sla.lu_factor(a, check_finite=False)
    return lu, piv


def floor_of(a, lu_ref, seed):
    rng = np.random.default_rng(seed)
    ap = a * (1.0 + 2.0 ** -53 * rng.uniform(-1.0, 1.0, a.shape))
    lu2, _ = lapack_lu(ap)
    return float(np.abs(lu2 - lu_ref).max() / np.abs(lu_ref).max())


def check(P, A, mode, n_floor=2):
    LU, ipiv, info = gpu_lu(P, A, mode)
    worst = 0.0
    for b in range(A.shape[0]):
        lu_ref, piv_ref = lapack_lu(A[b])
        assert np.array_equal(ipiv[b], piv_ref), (b, np.nonzero(ipiv[b] != piv_ref)[0][:10])
        assert info[b] == 0
        err = float(np.abs(LU[b] - lu_ref).max() / np.abs(lu_ref).max())
        if b < n_floor:
            bar = max(1e-12, 8.0 * floor_of(A[b], lu_ref, 7 + b))
        worst = max(worst, err)
        assert err <= bar, (b, err, bar)
    return worst


@pytest.fixture
def tune(P):
    """Restore the LU shape table after a test that changes it."""
    keys = list(P.TUNE_PARAMS)
    saved = {k: P.hps_tune_get(k) for k in keys}
    yield P
    for k, v in saved.items():
        P.hps_tune_set(k, v)


@pytest.mark.parametrize("mode", [0, 1], ids=["tc", "fp64"])
@pytest.mark.parametrize("n,batch,cplx", [(120, 400, False), (196, 320, True), (196, 64, False), (449, 4, True),
                                          (1000, 1, False)])
def test_batched_lu_matches_lapack(P, n, batch, cplx, mode):
    """One CTA per matrix (400 and 320 items), clusters of 2-8 CTAs (64 and
    4 items, ragged 449), and a single 1000-row matrix."""
    A = random_batch(n, batch, cplx, seed=n + batch)
    check(P, A, mode)


@pytest.mark.parametrize("n,cplx", [(1792, True), (3456, False), (6912, False)])
def test_root_sized_lu_matches_lapack(P, n, cplx):
    """The lazy root's W of the 2D Helmholtz workload (1792, complex), and
    the 3D workload's level-1 and root D (3456 and 6912 rows, real)."""
    A = random_batch(n, 1, cplx, seed=n)
    check(P, A, 0, n_floor=1)


def test_narrow_panels_for_few_matrices_match_lapack(tune):
    """The tuned panel width of few-matrix batches (16 instead of 32 for real
    data): the same interchanges and factors."""
    P = tune
    P.hps_tune_set("lu_panel_nb_few", 16)
    A = random_batch(3456, 1, False, seed=17)
    check(P, A, 0, n_floor=1)


def test_cooperative_panel_matches_lapack(tune):
    """The same results with the thread-block-cluster panel switched off."""
    P = tune
    P.hps_tune_set("lu_cluster_panel", 0)
    A = random_batch(700, 2, False, seed=3)
    check(P, A, 0)


def tie_matrix(n, rng):
    """Column 0 has one nonzero, 1 at row 300, so step 0 swaps rows 0 and 300
    and eliminates nothing (every multiplier is 0: no rounding anywhere).
    Column 1 then holds the largest magnitude, 1, in rows 0 (now at position
    300), 100 and 500: LAPACK's pivot is the lowest current position, row 100,
    although row 0 has the lowest index."""
    A = rng.uniform(-0.5, 0.5, (n, n))
    A[:, 0] = 0.0
    A[300, 0] = 1.0
    A[0, 1] = 1.0
    A[100, 1] = -1.0
    A[500, 1] = 1.0
    return A


@pytest.mark.parametrize("path", ["cluster", "cooperative", "one_cta"])
def test_ties_break_by_current_position(tune, path):
    P = tune
    rng = np.random.default_rng(5)
    if path == "one_cta":
        A = np.stack([tie_matrix(640, rng) for _ in range(200)])  # many items: one CTA each
    else:
        A = tie_matrix(1000, rng)[None]
        if path == "cooperative":
            P.hps_tune_set("lu_cluster_panel", 0)
    _, piv = lapack_lu(A[0])
    assert piv[0] == 300 and piv[1] == 100
    check(P, A, 0)


def test_exactly_singular_column(P):
    """A zero column k: info = k + 1 as in LAPACK, no interchange at step k,
    and the remaining columns are still factored."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((2, 600, 600))
    A[:, :, 200] = 0.0
    LU, ipiv, info = gpu_lu(P, A, 0)
    for b in range(2):
        lu_ref, piv_ref = lapack_lu(A[b])
        assert info[b] == 201
        assert np.array_equal(ipiv[b], piv_ref)
        assert np.abs(LU[b] - lu_ref).max() / np.abs(lu_ref).max() < 1e-10


def test_invalid_arguments(P):
    A = torch.zeros((1, 4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        P.hps_getrf(A)
    A = torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        P.hps_getrf(A, mode=3)
