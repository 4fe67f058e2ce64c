"""GPU tests of the tensor-core FP64 product (hps_gemm mode 0): exact
digit-slice products accumulated in fp32 and recombined in integers.

References: every entry is checked against the FP64 product (numpy) within
the error bound of both computations, and sampled entries against the exact
rational value of the dot product (fractions), where the digit-slice error
bound itself is checked:

  |C - exact| <= (K 2^-57 + chunks 2^-lsb) 2^(e_i + f_j) + 2^-52 |exact|

with 2^e_i the power of two above the largest |A(i, :)|, 2^f_j that above
the largest |B(:, j)|, lsb = 62 - ceil(log2 K) fixed-point fraction bits and
chunks = ceil(K / 256) exact accumulation chunks (operand rounding
K 2^-60, dropped digit pairs about K 2^-58.7, half a fixed-point unit per
chunk, the final rounding to FP64).
"""

import math
from fractions import Fraction

import numpy as np
import pytest

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


def _colmajor(x):
    """(batch, rows, cols) numpy -> device tensor (batch, cols, rows) contiguous."""
    return torch.from_numpy(np.ascontiguousarray(np.swapaxes(x, 1, 2))).cuda()


def _back(t):
    return np.swapaxes(t.cpu().numpy(), 1, 2)


def _run(P, A, B, C0, alpha, beta, mode):
    C = _colmajor(C0)
    P.hps_gemm(_colmajor(A), _colmajor(B), C, alpha=alpha, beta=beta, mode=mode)
    torch.cuda.synchronize()
    return _back(C)


def _pow2_above(x):
    """2^e with max |x| < 2^e (e = frexp exponent); 1 for zero."""
    out = np.ones_like(x)
    nz = x > 0
    out[nz] = np.ldexp(1.0, np.frexp(x[nz])[1])
    return out


def _bound(A, B, K):
    lsb = 62 - math.ceil(math.log2(max(K, 1)))
    chunks = -(-K // 256)
    ea = _pow2_above(np.abs(A).max(axis=2))          # (batch, m)
    fb = _pow2_above(np.abs(B).max(axis=1))          # (batch, n)
    return (K * 2.0 ** -57 + chunks * 2.0 ** -lsb) * ea[:, :, None] * fb[:, None, :]


def _exact(a_row, b_col):
    return sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a_row, b_col))


def _check(A, B, C0, C, alpha, beta, rng, nsample=24):
    batch, m, K = A.shape
    n = B.shape[2]
    ref = alpha * np.matmul(A, B) + beta * C0
    # FP64 product error bound: K u sum |a||b| (plus the epilogue roundings)
    fp64_err = (K + 4) * 2.0 ** -53 * (np.abs(alpha) * np.matmul(np.abs(A), np.abs(B)) + abs(beta) * np.abs(C0))
    tol = abs(alpha) * _bound(A, B, K) + 2.0 ** -51 * np.abs(ref) + fp64_err
    err = np.abs(C - ref)
    assert np.all(err <= tol), float((err / tol).max())
    # sampled entries against the exact rational value
    for _ in range(nsample):
        b, i, j = int(rng.integers(batch)), int(rng.integers(m)), int(rng.integers(n))
        ex = Fraction(alpha) * _exact(A[b, i, :], B[b, :, j]) + Fraction(beta) * Fraction(float(C0[b, i, j]))
        d = abs(Fraction(float(C[b, i, j])) - ex)
        lim = abs(alpha) * _bound(A[b:b + 1, i:i + 1], B[b:b + 1, :, j:j + 1], K)[0, 0, 0] + \
            2.0 ** -52 * abs(float(ex)) + 2.0 ** -52 * abs(beta * C0[b, i, j])
        assert float(d) <= lim, (b, i, j, float(d), lim)


# A product whose transposed tiling (C^T = B^T A^T in 128 x 48 tiles of C^T)
# takes fewer waves of CTAs over the SMs runs transposed: the few-row shapes
# of the recursive LU and triangular solves with many items (32 x 114 x 400,
# 48 x 225 x 200, 40 x 1000 x 20 items); everything that fits one wave stays
# in the normal form.
SHAPES = [
    (1, 1, 1, 1),
    (130, 50, 17, 3),      # ragged M, N and K tiles
    (128, 48, 256, 2),     # exactly one tile and one accumulation chunk
    (200, 97, 449, 2),     # ragged K tail
    (300, 130, 700, 1),    # three accumulation chunks
    (64, 33, 32, 5),
    (32, 114, 32, 400),    # transposed: one 128 x 48 tile of C^T per item
    (48, 225, 56, 200),    # transposed, two 128-row tiles of C^T per item
    (40, 1000, 300, 20),   # transposed, eight 128-row tiles of C^T, two chunks
]

@pytest.mark.parametrize("m,n,k,batch", SHAPES, ids=[f"{s[0]}x{s[1]}x{s[2]}b{s[3]}" for s in SHAPES])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0), (0.5, -2.0)], ids=["set", "sub", "general"])
def test_real_product_within_bound(P, m, n, k, batch, alpha, beta):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((batch, m, k))
    B = rng.standard_normal((batch, k, n))
    C0 = rng.standard_normal((batch, m, n))
    C = _run(P, A, B, C0, alpha, beta, 0)
    _check(A, B, C0, C, alpha, beta, rng)


def test_wide_dynamic_range_and_zero_rows(P):
    """Rows and columns scaled by 2^-40 .. 2^40, entries 1e-12 next to 1, and
    zero rows / columns: the bound is relative to each row's / column's
    largest entry."""
    rng = np.random.default_rng(11)
    batch, m, n, k = 2, 150, 70, 300
    A = rng.standard_normal((batch, m, k)) * np.ldexp(1.0, rng.integers(-40, 41, (batch, m, 1)))
    B = rng.standard_normal((batch, k, n)) * np.ldexp(1.0, rng.integers(-40, 41, (batch, 1, n)))
    A[:, 5, :] = 0.0
    B[:, :, 7] = 0.0
    A[:, :, ::3] *= 1e-12
    C0 = np.zeros((batch, m, n))
    C = _run(P, A, B, C0, 1.0, 0.0, 0)
    assert np.all(C[:, 5, :] == 0.0) and np.all(C[:, :, 7] == 0.0)
    _check(A, B, C0, C, 1.0, 0.0, rng)


@pytest.mark.parametrize("m,n,k,batch", [(130, 60, 470, 2), (200, 60, 300, 2), (32, 114, 32, 400)],
                         ids=["ragged", "normal", "transposed"])
def test_complex_product(P, m, n, k, batch):
    """Complex products run as one launch per component of C, two real
    digit-slice products into shared accumulators: Re = Ar Br - Ai Bi, Im =
    Ar Bi + Ai Br (in the transposed tiling the A slot holds B's parts and the
    B slot A's).  The parts of a row of A (column of B) share one scale, so
    each component is the real product [Ar Ai] [Br; -Bi] (resp. [Bi; Br]) of
    inner dimension 2K, and the bound is that product's."""
    rng = np.random.default_rng(3 + m)
    z = lambda s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    A, B, C0 = z((batch, m, k)), z((batch, k, n)), z((batch, m, n))
    Ar, Ai, Br, Bi = A.real, A.imag, B.real, B.imag
    mag = np.matmul(np.abs(A), np.abs(B))
    for alpha, beta in [(1.0, 0.0), (-1.0, 1.0)]:
        C = _run(P, A, B, C0, alpha, beta, 0)
        ref = alpha * np.matmul(A, B) + beta * C0
        slack = (2 * k + 8) * 2.0 ** -53 * 2 * (mag + np.abs(C0)) + 2.0 ** -51 * np.abs(ref)
        Acat = np.concatenate([Ar, Ai], axis=2)
        tol_re = _bound(Acat, np.concatenate([Br, -Bi], axis=1), 2 * k) + slack
        tol_im = _bound(Acat, np.concatenate([Bi, Br], axis=1), 2 * k) + slack
        assert np.all(np.abs(C.real - ref.real) <= tol_re)
        assert np.all(np.abs(C.imag - ref.imag) <= tol_im)


def test_modes_agree_and_fp64_mode_is_native(P):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 257, 129))
    B = rng.standard_normal((3, 129, 95))
    C0 = np.zeros((3, 257, 95))
    c_tc = _run(P, A, B, C0, 1.0, 0.0, 0)
    c_fp = _run(P, A, B, C0, 1.0, 0.0, 1)
    ref = np.matmul(A, B)
    mag = np.matmul(np.abs(A), np.abs(B))
    assert np.all(np.abs(c_fp - ref) <= 140 * 2.0 ** -53 * mag)
    assert np.all(np.abs(c_tc - c_fp) <= 300 * 2.0 ** -53 * mag + 2.0 ** -50 * np.abs(ref))


def test_invalid_arguments(P):
    from paper_2503_17535_gb300 import HPSError
    A = torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(HPSError):
        P.hps_gemm(A, A, A, mode=7)
    with pytest.raises(ValueError):
        P.hps_gemm(A, torch.zeros((1, 3, 5), dtype=torch.float64, device="cuda"), A)


@pytest.mark.parametrize("m,batch", [(32, 160), (300, 7)], ids=["transposed", "normal"])
@pytest.mark.parametrize("shared", ["A", "B"])
@pytest.mark.parametrize("cplx", [False, True], ids=["real", "complex"])
def test_operand_shared_by_every_item(P, shared, cplx, m, batch):
    """An operand given with item stride 0 (the same matrix for every item,
    as the leaf stage's Q and QH products are) is cut into digits once per
    call and serves every item; the products stay within the bound."""
    from paper_2503_17535_gb300 import _capi
    rng = np.random.default_rng(31 if shared == "A" else 37)
    n, k = 114, 300
    z = (lambda s: rng.standard_normal(s) + 1j * rng.standard_normal(s)) if cplx else rng.standard_normal
    A = z((1 if shared == "A" else batch, m, k))
    B = z((1 if shared == "B" else batch, k, n))
    Ad, Bd = _colmajor(A), _colmajor(B)
    Cd = _colmajor(np.zeros((batch, m, n), A.dtype))
    st = _capi.lib().hps_gemm(_capi.HPS_C128 if cplx else _capi.HPS_F64, 0, m, n, k, batch, 1.0, Ad.data_ptr(), m,
                              0 if shared == "A" else m * k, Bd.data_ptr(), k, 0 if shared == "B" else k * n, 0.0,
                              Cd.data_ptr(), m, m * n, None)
    torch.cuda.synchronize()
    assert st == 0
    C = _back(Cd)
    Af, Bf = np.broadcast_to(A, (batch, m, k)), np.broadcast_to(B, (batch, k, n))
    if not cplx:
        _check(Af, Bf, np.zeros((batch, m, n)), C, 1.0, 0.0, rng)
    else:
        ref = np.matmul(Af, Bf)
        scale = np.abs(Af).max() * np.abs(Bf).max() * k
        assert np.abs(C - ref).max() <= 1e-14 * scale
