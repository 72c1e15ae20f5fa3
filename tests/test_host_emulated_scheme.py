"""The digit-slicing scheme of the emulated-FP64 contractions, restated on the
host in exact integer arithmetic (the GPU kernels are tested against exact dot
products in tests/test_gpu_emulated.py):

* a row scaled into (-1, 1) by a power of two and rounded to q = rint(x 2^{5S})
  has balanced base-32 digits with |d_0| <= 32, |d_j| <= 16, that sum back to q;
* the level sums of one accumulation piece (at most 8192 products of digits)
  stay integers below 2^23, so an FP32 accumulator holds them exactly;
* sum over i + j < S of 2^{-5(i+j+2)} D_i D_j^T approximates A B^T within the
  stated bound 4 (S + 1) 2^{-5S} K max|a_m| max|b_n|, and the bound is not loose
  by orders of magnitude for few digits.
"""
from fractions import Fraction

import numpy as np
import pytest

BITS = 5
PIECE_PRODUCTS = 8192


def _row_exponent(row):
    m = np.max(np.abs(row))
    return 0 if m == 0 else int(np.frexp(m)[1])


def _digits(row, S):
    """(e, D) with D[j] the j-th balanced digits of rint(row 2^{5S - e})."""
    e = _row_exponent(row)
    q = [int(round(Fraction(float(x)) * Fraction(2) ** (BITS * S - e))) for x in row]
    D = np.zeros((S, len(row)), dtype=np.int64)
    for k, v in enumerate(q):
        for j in range(S - 1, 0, -1):
            d = ((v + 16) & 31) - 16
            v = (v - d) >> BITS
            D[j, k] = d
        D[0, k] = v
    return e, D


def _emulated(A, B, S):
    """Exact value (Fraction) of the scheme's result for every (m, n)."""
    ea, DA = zip(*[_digits(a, S) for a in A])
    eb, DB = zip(*[_digits(b, S) for b in B])
    out = [[Fraction(0)] * len(B) for _ in A]
    for m in range(len(A)):
        for n in range(len(B)):
            tot = Fraction(0)
            for d in range(S):
                level = sum(int(DA[m][i] @ DB[n][d - i]) for i in range(d + 1))
                tot += Fraction(level) * Fraction(2) ** (-BITS * (d + 2))
            out[m][n] = tot * Fraction(2) ** (ea[m] + eb[n])
    return out


def test_balanced_digits_reconstruct_the_rounded_integer():
    rng = np.random.default_rng(0)
    for S in (1, 3, 11, 12):
        row = rng.standard_normal(50) * np.exp2(rng.integers(-30, 30))
        e, D = _digits(row, S)
        assert np.all(np.abs(D[0]) <= 32) and np.all(np.abs(D[1:]) <= 16)
        for k, x in enumerate(row):
            q = sum(int(D[j, k]) * 32 ** (S - 1 - j) for j in range(S))
            assert q == round(Fraction(float(x)) * Fraction(2) ** (BITS * S - e))


def test_piece_sums_fit_fp32_exactly():
    """The worst case of one piece: 8192 products of the largest digits."""
    assert PIECE_PRODUCTS * 32 * 32 <= 2 ** 23
    rng = np.random.default_rng(1)
    row_a = np.where(rng.random(PIECE_PRODUCTS) < 0.5, -1.0, 1.0) * (1 - 2.0 ** -40)
    _, DA = _digits(row_a, 11)
    s = int(DA[0] @ DA[0])
    assert abs(s) <= 2 ** 23 and float(np.float32(s)) == s


@pytest.mark.parametrize("S", [2, 3, 11])
def test_scheme_error_within_bound(S):
    rng = np.random.default_rng(S)
    M, N, K = 3, 4, 40
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-8, 9, size=(M, 1)))
    B = rng.standard_normal((N, K)) * np.exp2(rng.integers(-8, 9, size=(N, 1)))
    C = _emulated(A, B, S)
    worst = 0.0
    for m in range(M):
        for n in range(N):
            exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[m], B[n]))
            err = abs(float(C[m][n] - exact))
            bound = 4 * (S + 1) * 2.0 ** (-BITS * S) * K * np.abs(A[m]).max() * np.abs(B[n]).max()
            assert err <= bound, (m, n, err, bound)
            worst = max(worst, err / bound)
    if S <= 3:
        assert worst > 1e-4  # the bound is within a few orders of the actual error
