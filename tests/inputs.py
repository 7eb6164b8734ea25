"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method: it only draws numbers (numpy's
PCG64 generator) and builds matrices of fixed, documented structure.  The
random system of the method itself (the 64-bit LCG of the library) is not
drawn here: each side implements it independently.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform(shape, seed: int) -> np.ndarray:
    """i.i.d. U[-0.5, 0.5) in Fortran order."""
    return np.asfortranarray(rng(seed).random(shape) - 0.5)


def dyadic_factors(n: int, seed: int, block: int = 0):
    """L0 unit lower with strictly-lower entries in {0, +1/2, -1/2}, U0 upper with
    small integers (nonzero diagonal).  A0 = L0 @ U0 is exact in FP64 and partial
    pivoting never swaps it (every subdiagonal multiplier has magnitude <= 1/2).

    With block > 0, inside each diagonal block (block x block, at multiples of
    block) the strictly-lower entries of L0 sit only in the block's lower-left
    quarter (rows of its second half, columns of its first half) and the
    strictly-upper entries of U0 only in its upper-right quarter, and U0's
    diagonal holds powers of two: each diagonal block of L0 is I + N with
    N^2 = 0 and each of U0 is D (I + N') with N'^2 = 0, so their inverses
    I - N and (I - N') D^-1 are dyadic too, as are those of every diagonal
    sub-block, and solves by explicit inverses stay exact."""
    g = rng(seed)
    L0 = np.tril(g.choice([-0.5, 0.0, 0.5], size=(n, n)), -1)
    if block > 0:
        for b0 in range(0, n, block):
            b1 = min(n, b0 + block)
            h = b0 + (b1 - b0 + 1) // 2
            D = np.zeros((b1 - b0, b1 - b0))
            D[h - b0:, :h - b0] = L0[h:b1, b0:h]
            L0[b0:b1, b0:b1] = D
    L0 = L0 + np.eye(n)
    U0 = np.triu(g.integers(-8, 9, size=(n, n)).astype(np.float64))
    d = g.integers(1, 9, size=n) * g.choice([-1, 1], size=n)
    if block > 0:
        d = 2.0 ** g.integers(0, 4, size=n) * g.choice([-1, 1], size=n)
        for b0 in range(0, n, block):
            b1 = min(n, b0 + block)
            h = b0 + (b1 - b0 + 1) // 2
            D = np.zeros((b1 - b0, b1 - b0))
            D[:h - b0, h - b0:] = U0[b0:h, h:b1]
            U0[b0:b1, b0:b1] = D
    U0[np.arange(n), np.arange(n)] = d
    A0 = L0 @ U0
    return np.asfortranarray(L0), np.asfortranarray(U0), np.asfortranarray(A0)


def wilkinson_growth(n: int) -> np.ndarray:
    """a_ii = 1, a_ij = -1 for i > j, a_in = 1 (last column), else 0."""
    A = np.tril(-np.ones((n, n)), -1) + np.eye(n)
    A[:, n - 1] = 1.0
    return np.asfortranarray(A)


def permutation_matrix(n: int, seed: int):
    p = rng(seed).permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), p] = 1.0
    return np.asfortranarray(P), p
