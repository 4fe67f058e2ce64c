"""Host model of the tensor-core product's arithmetic (no GPU).

The CUDA kernels cut each row of A (column of B) into ten balanced base-64
digits of the value scaled by 2^-e and rounded to 60 fraction bits, sum the
digit products of each anti-diagonal d = p + q <= 11 exactly in fp32 over
K chunks of 256, and recombine the ten diagonal sums in a 64-bit fixed-point
integer (pairs of diagonals in 32 bits, diagonals 2..7 exactly, 8..11
rounded once per chunk) before one scaling into FP64.  This file rebuilds
those steps with Python integers and checks the facts the kernel relies on:

* the digits lie in [-64, 64] (leading) and [-32, 31] (others), so they are
  exact in bf16, and reconstruct the rounded value;
* the largest |sum of one diagonal's products| over a chunk stays below
  2^22, where the kernel's fp32-add conversion to an integer is exact;
* the 32-bit pairing, the high / low split and the final rounding reproduce
  the exact fixed-point value within the rounding the kernel documents;
* the result meets the error bound the GPU tests use,
  (K 2^-57 + chunks 2^-lsb) 2^(e_i + f_j) + 2^-52 |exact|,
  on random and adversarial inputs.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

DIG, BITS, DSUM, KC = 10, 6, 11, 256
FRAC = DIG * BITS


def row_exp(row):
    """e with max |x| < 2^e (frexp exponent); 0 for a zero row."""
    m = max(abs(float(x)) for x in row)
    return math.frexp(m)[1] if m > 0 else 0


def digits(x, e):
    """Balanced base-64 digits (most significant first) of x 2^(FRAC - e)
    rounded to an integer (ties away from zero in magnitude, as the kernel)."""
    fx = Fraction(float(x)) * Fraction(2) ** (FRAC - e)
    mag = abs(fx)
    X = int(mag + Fraction(1, 2))          # round half up in magnitude
    X = -X if fx < 0 else X
    out = [0] * DIG
    for p in range(DIG - 1, 0, -1):
        t = X + 32
        out[p] = (t & 63) - 32
        X = t >> BITS
    out[0] = X
    return out


def fixed_product(A, B):
    """The kernel's C = A B (real), entry by entry, in exact integers."""
    M, K = A.shape
    N = B.shape[1]
    lsb = 62 - math.ceil(math.log2(max(K, 1)))
    ea = [row_exp(A[i, :]) for i in range(M)]
    fb = [row_exp(B[:, j]) for j in range(N)]
    da = [[digits(A[i, k], ea[i]) for k in range(K)] for i in range(M)]
    db = [[digits(B[k, j], fb[j]) for k in range(K)] for j in range(N)]
    C = np.zeros((M, N))
    maxdiag = 0
    for i in range(M):
        for j in range(N):
            R = 0
            for c0 in range(0, K, KC):
                S = [0] * (DSUM - 1)        # diagonals d = 2..11
                for k in range(c0, min(K, c0 + KC)):
                    a, b = da[i][k], db[j][k]
                    for p in range(DIG):
                        for q in range(DIG):
                            if p + q <= DSUM - 2:
                                S[p + q] += a[p] * b[q]
                maxdiag = max(maxdiag, max(abs(v) for v in S))
                y = [S[2 * t] * 64 + S[2 * t + 1] for t in range(5)]
                assert all(abs(v) < 2 ** 31 for v in y)
                H = (y[0] << 24) + (y[1] << 12) + y[2]          # units 2^-42
                L = (y[3] << 12) + y[4]                         # units 2^-66
                sh_l = 66 - lsb
                R += (H << (lsb - 42)) + ((L + (1 << (sh_l - 1))) >> sh_l)
            assert abs(R) < 2 ** 63
            C[i, j] = float(Fraction(R) * Fraction(2) ** (ea[i] + fb[j] - lsb))
    return C, ea, fb, lsb, maxdiag


def check(A, B):
    M, K = A.shape
    N = B.shape[1]
    C, ea, fb, lsb, maxdiag = fixed_product(A, B)
    assert maxdiag < 2 ** 22
    chunks = -(-K // KC)
    for i in range(M):
        for j in range(N):
            ex = sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K))
            lim = (K * 2.0 ** -57 + chunks * 2.0 ** -lsb) * 2.0 ** (ea[i] + fb[j]) + 2.0 ** -52 * abs(float(ex))
            assert abs(float(Fraction(float(C[i, j])) - ex)) <= lim, (i, j)


def test_digits_are_exact_in_bf16_and_reconstruct():
    rng = np.random.default_rng(0)
    for x in list(rng.standard_normal(2000)) + [1.0 - 2.0 ** -53, -(1.0 - 2.0 ** -53), 0.5, 2.0 ** -60, 0.0]:
        e = row_exp([x, 1.0])
        d = digits(x, e)
        assert -64 <= d[0] <= 64 and all(-32 <= v <= 31 for v in d[1:])
        val = sum(Fraction(v) * Fraction(2) ** (-BITS * (p + 1)) for p, v in enumerate(d)) * Fraction(2) ** e
        assert abs(val - Fraction(float(x))) <= Fraction(2) ** (e - FRAC - 1)


def test_worst_diagonal_sum_stays_below_2_to_22():
    """Every entry at its row's largest magnitude with the sign pattern that
    maximises one diagonal: the bound 256 (2 64 32 + 8 32 32) < 2^22."""
    assert KC * (2 * 64 * 32 + (DIG - 2) * 32 * 32) < 2 ** 22
    assert KC * 64 * 64 < 2 ** 22
    x = 1.0 - 2.0 ** -20   # leading digit 64 after rounding, others near -32 / 31
    A = np.full((1, KC), x)
    B = np.full((KC, 1), x)
    C, *_, maxdiag = fixed_product(A, B)
    assert maxdiag < 2 ** 22


@pytest.mark.parametrize("M,N,K,seed", [(3, 4, 7, 1), (4, 3, 300, 2), (2, 2, 600, 3)])
def test_product_meets_the_documented_bound(M, N, K, seed):
    rng = np.random.default_rng(seed)
    check(rng.standard_normal((M, K)), rng.standard_normal((K, N)))


def test_product_bound_with_wide_ranges_and_zero_rows():
    rng = np.random.default_rng(7)
    M, N, K = 3, 3, 40
    A = rng.standard_normal((M, K)) * np.ldexp(1.0, rng.integers(-30, 31, (M, 1)))
    B = rng.standard_normal((K, N)) * np.ldexp(1.0, rng.integers(-30, 31, (1, N)))
    A[:, ::3] *= 1e-12
    A[1, :] = 0.0
    C, *_ = fixed_product(A, B)
    assert np.all(C[1, :] == 0.0)
    check(A, B)


def test_aligned_digits_need_every_kept_diagonal():
    """Entries whose first eight digits are all 31 (48 bits: exact in FP64;
    one entry of 0.99 fixes each row's exponent at 0): every digit product is
    positive, so each diagonal's sum grows linearly in K; dropping a kept
    diagonal (for instance d = 11, about K 2^-53.5) breaks the bound, which
    is met with all ten."""
    x = float(sum(Fraction(31) * Fraction(2) ** (-BITS * (p + 1)) for p in range(8)))
    assert digits(x, 0) == [31] * 8 + [0, 0]
    K = 200
    A = np.full((2, K), x)
    A[:, 0] = 0.99
    B = np.full((K, 2), x)
    B[0, :] = 0.99
    check(A, B)
