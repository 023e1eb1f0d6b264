"""The integer-slice scheme of the float64 tensor-core products, modelled
exactly on the CPU (numpy and rational arithmetic; no CUDA code involved).

Each operand row r is scaled by 2^-e_r (e_r the binary exponent of its
largest entry) and cut into 8 digits of 7 bits; the 36 digit pairs with
t + u <= 9 are grouped by level l = t + u, levels 2-6 combine exactly as
integers and levels 7-9 in float32, then one float64 scaling.  These tests
pin the bounds the scheme relies on."""
import math
from fractions import Fraction

import numpy as np
import pytest

SLICES, BITS = 8, 7


def row_exponent(row):
    m = max(abs(float(v)) for v in row)
    return math.frexp(m)[1] if m > 0 else None      # m < 2^e


def digits(x, e):
    """The 8 signed 7-bit digits a_t of x / 2^e (truncation toward zero)."""
    V = math.floor(abs(Fraction(x)) * 2 ** (SLICES * BITS - e))
    assert V < 2 ** (SLICES * BITS)
    ds = [(V >> (BITS * (SLICES - t))) & 127 for t in range(1, SLICES + 1)]
    return [-d if x < 0 else d for d in ds]


def spread(rng, shape, span):
    v = rng.uniform(-0.5, 0.5, shape)
    return np.ldexp(v, -rng.integers(0, span + 1, shape)) if span else v


@pytest.mark.parametrize("span", [0, 40])
def test_digits_reconstruct_within_2_pow_minus_56(span):
    rng = np.random.default_rng(span + 1)
    A = spread(rng, (6, 50), span)
    for row in A:
        e = row_exponent(row)
        for x in row:
            ds = digits(x, e)
            assert all(-127 <= d <= 127 for d in ds)
            rec = sum(Fraction(d) * Fraction(2) ** (e - BITS * t) for t, d in enumerate(ds, 1))
            assert abs(Fraction(x) - rec) < Fraction(2) ** (e - 56)


def test_float32_sums_of_digit_products_are_exact_over_1024_terms():
    """1024 products of digits in [-127, 127], summed in float32 in any
    order, equal the integer sum: every partial sum stays below 2^24."""
    assert 1024 * 127 * 127 < 2 ** 24
    rng = np.random.default_rng(3)
    cases = [np.full(1024, 127 * 127)]                       # all at the bound, one sign
    cases += [rng.integers(-127, 128, 1024) * rng.integers(-127, 128, 1024) for _ in range(20)]
    for prods in cases:
        exact = int(prods.sum())
        for order in (np.arange(1024), rng.permutation(1024)):
            acc = np.float32(0.0)
            for p in prods[order]:
                acc = np.float32(acc + np.float32(p))
            assert int(acc) == exact


def emulate(A, B):
    """A @ B by the scheme: exact level sums, int64 levels 2-6, float32
    levels 7-9, float64 scaling.  Returns (result, exact-truncated)."""
    M, K = A.shape
    N = B.shape[1]
    eA = [row_exponent(A[i]) for i in range(M)]
    eB = [row_exponent(B[:, j]) for j in range(N)]
    dA = [[digits(A[i, k], eA[i]) if eA[i] is not None else [0] * SLICES for k in range(K)]
          for i in range(M)]
    dB = [[digits(B[k, j], eB[j]) if eB[j] is not None else [0] * SLICES for k in range(K)]
          for j in range(N)]
    out = np.zeros((M, N))
    trunc = [[Fraction(0)] * N for _ in range(M)]
    for i in range(M):
        for j in range(N):
            if eA[i] is None or eB[j] is None:
                continue
            S = {}
            for l in range(2, SLICES + 2):
                S[l] = sum(dA[i][k][t - 1] * dB[j][k][l - t - 1]
                           for k in range(K) for t in range(1, l))
            H = 0
            for l in range(2, 7):
                H = H * 128 + S[l]
            assert abs(H) < 2 ** 63
            T = np.float32(0.0)
            for l in range(9, 6, -1):
                T = np.float32(np.float32(T) * np.float32(0.0078125) + np.float32(S[l]))
            h = float(T) * 0.0078125 + float(H)
            out[i, j] = math.ldexp(h, eA[i] + eB[j] - 42)
            trunc[i][j] = sum(Fraction(S[l]) * Fraction(2) ** (eA[i] + eB[j] - 7 * l)
                              for l in S)
    return out, trunc


@pytest.mark.parametrize("span,K", [(0, 300), (40, 300), (0, 1500)])
def test_emulated_product_is_float64_accurate(span, K):
    rng = np.random.default_rng(K + span)
    A = spread(rng, (4, K), span)
    B = spread(rng, (K, 3), span)
    got, trunc = emulate(A, B)
    for i in range(A.shape[0]):
        scale_r = row_exponent(A[i])
        for j in range(B.shape[1]):
            scale_c = row_exponent(B[:, j])
            exact = sum(Fraction(A[i, k]) * Fraction(B[k, j]) for k in range(K))
            unit = Fraction(2) ** (scale_r + scale_c)
            # dropped pairs and remainders: below 9 K 2^-56 of the scale
            assert abs(trunc[i][j] - exact) <= 9 * K * Fraction(2) ** -56 * unit
            # the int64 + float32 combination adds float64 rounding only
            assert abs(Fraction(got[i, j]) - trunc[i][j]) <= (
                Fraction(2) ** -52 * abs(trunc[i][j]) + Fraction(2) ** -57 * K * unit)
            # and the result is as close to the exact product as float64 sums are
            ref = float(np.dot(A[i], B[:, j]))
            assert abs(got[i, j] - ref) <= 4 * K * 2.0 ** -53 * float(unit)
