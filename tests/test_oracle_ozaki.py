"""Pins for the oracle of the emulated FP64 trailing update (slice products
after Ozaki, Ogita, Oishi and Rump 2012), no GPU:

  - the splitting is error-free and its slices are in range: sum_i q_i
    2^(E - i beta) reproduces every entry to within 2^(E - s beta - 1), with
    |q_1| <= 2^beta and |q_i| <= 2^(beta - 1);
  - on integer matrices whose bits all fit in the kept slices the update is
    exact (C - A B to the last bit, checked with Python integers);
  - on random matrices the error against the exact result (Python fractions)
    is within the bound that follows from the dropped slice pairs and the
    FP64 roundings of the level sum, and that bound is of the order of an
    FP64 DGEMM's own rounding error;
  - the oracle refuses slice parameters whose level sums could leave the
    range where FP32 accumulation is exact.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests import inputs

U64 = 2.0 ** -53


@pytest.mark.parametrize("s,beta", [(8, 7), (9, 6), (3, 5)])
def test_split_is_error_free_and_in_range(s, beta):
    g = inputs.rng(11)
    A = np.asfortranarray(g.standard_normal((40, 33)) * 2.0 ** g.integers(-30, 30, (40, 1)))
    A[3, :] = 0.0  # a zero row: exponent 0, zero slices
    E, Q = O.ozaki_split_rows(A, s, beta)
    assert np.all(np.abs(Q[0]) <= 2.0 ** beta) and np.all(np.abs(Q[1:]) <= 2.0 ** (beta - 1))
    assert np.all(Q == np.round(Q))
    assert E[3] == 0 and not Q[:, 3, :].any()
    for r in range(A.shape[0]):
        mu = np.max(np.abs(A[r]))
        if mu > 0:
            assert mu < 2.0 ** E[r] <= 2 * mu
        for c in range(A.shape[1]):
            rec = sum(Fraction(int(Q[i, r, c])) * Fraction(2) ** (int(E[r]) - (i + 1) * beta) for i in range(s))
            assert abs(rec - Fraction(A[r, c])) <= Fraction(2) ** (int(E[r]) - s * beta - 1)
    # the columns of B use the same rule on B^T's rows
    F, QB = O.ozaki_split_cols(A.T, s, beta)
    assert np.array_equal(F, E) and np.array_equal(QB, Q)


@pytest.mark.parametrize("k", [1, 64, 384])
def test_integer_inputs_are_exact(k):
    g = inputs.rng(12 + k)
    m, n = 9, 7
    A = g.integers(-(2 ** 20), 2 ** 20, (m, k)).astype(np.float64)
    B = g.integers(-(2 ** 20), 2 ** 20, (k, n)).astype(np.float64)
    Cm = g.integers(-(2 ** 30), 2 ** 30, (m, n)).astype(np.float64)
    got = O.ozaki_gemm(A, B, Cm, 8, 7)
    exact = Cm.astype(object) - A.astype(np.int64).astype(object) @ B.astype(np.int64).astype(object)
    assert all(int(got[i, j]) == exact[i, j] and float(exact[i, j]) == got[i, j]
               for i in range(m) for j in range(n))


def truncation_per_term(s, beta):
    """Bound on |a'b' - kept part| for |a'|, |b'| < 1 (units of 2^(E + F))."""
    t = 0.0
    for d in range(s + 2, 2 * s + 1):
        pairs = sum(1 for i in range(2, s + 1) if 2 <= d - i <= s)
        t += pairs * 2.0 ** (-(d - 2) * beta - 2)
    return t + 2.0 ** (-s * beta) + 2.0 ** (-2 * s * beta - 2)


@pytest.mark.parametrize("s,beta,k", [(8, 7, 64), (9, 6, 96), (8, 7, 384)])
def test_random_inputs_within_the_bound(s, beta, k):
    g = inputs.rng(20 + k)
    m, n = 5, 4
    A = inputs.uniform((m, k), seed=30 + k) * 2.0 ** g.integers(-3, 3, (m, 1))
    B = inputs.uniform((k, n), seed=31 + k)
    Cm = inputs.uniform((m, n), seed=32 + k)
    got = O.ozaki_gemm(A, B, Cm, s, beta)
    E, _ = O.ozaki_split_rows(A, s, beta)
    F, _ = O.ozaki_split_cols(B, s, beta)
    T = truncation_per_term(s, beta)
    worst_vs_dgemm = 0.0
    for i in range(m):
        for j in range(n):
            exact = Fraction(Cm[i, j]) - sum(Fraction(A[i, t]) * Fraction(B[t, j]) for t in range(k))
            scale = 2.0 ** (int(E[i]) + int(F[j]))
            bound = k * scale * (T + 4 * s * U64) + U64 * abs(float(exact))
            err = abs(Fraction(got[i, j]) - exact)
            assert err <= Fraction(bound), (i, j, float(err), bound)
            # the same order as an FP64 DGEMM's rounding bound gamma_k |A||B| + u |C|
            dgemm = k * U64 * float(np.abs(A[i]) @ np.abs(B[:, j])) + U64 * abs(Cm[i, j])
            worst_vs_dgemm = max(worst_vs_dgemm, float(err) / dgemm)
    assert worst_vs_dgemm < 1.0


def test_refuses_inexact_level_sums():
    A = np.ones((2, 410))
    B = np.ones((410, 2))
    with pytest.raises(ValueError):
        O.ozaki_gemm(A, B, np.zeros((2, 2)), 8, 7)   # k = 410 > 409 for s = 8, beta = 7
    O.ozaki_gemm(A[:, :409], B[:409], np.zeros((2, 2)), 8, 7)
    O.ozaki_gemm(A, B, np.zeros((2, 2)), 9, 6)
