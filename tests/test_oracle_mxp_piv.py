"""Pins of the oracle's mixed-precision LU with partial pivoting and of its
GMRES-IR (CPU only).

The pivoted variant keeps the steps of the unpivoted one and pivots FACT as in
Sec. I (largest magnitude, first row on ties, interchanges across all columns).
It is pinned against the unpivoted oracle on diagonally dominant systems (where
partial pivoting never swaps), against exact factors of permuted dyadic
products (the pivots must undo the permutation), and against the Wilkinson
growth matrix (a magnitude tie in every column).  GMRES-IR is pinned by the
finite termination of GMRES: from x0 = b on A = I + U V^T of rank r it ends
after exactly r Arnoldi steps, on a diagonal matrix with k distinct entries
other than 1 after k.
The last tests record what the pivoted variant does on the plain HPL system."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from tests import inputs


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
@pytest.mark.parametrize("n,nb", [(300, 128), (257, 64)])
def test_pivoted_equals_unpivoted_without_interchanges(prec, n, nb):
    A, _ = O.generate(n, 5 + n, dd=True)
    W0, info0 = O.mxp_getrf(A, nb, prec)
    W, ipiv, info = O.mxp_getrf_piv(A, nb, prec)
    assert info == info0 == 0
    assert np.array_equal(ipiv, np.arange(1, n + 1))
    assert np.array_equal(W, W0)


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
@pytest.mark.parametrize("n,nb", [(64, 16), (300, 128), (260, 256)])
def test_pivoted_exact_on_permuted_dyadic_factors(prec, n, nb):
    L0, U0, A0 = inputs.dyadic_factors(n, seed=3 * n + prec)
    P, _ = inputs.permutation_matrix(n, seed=n)
    A = np.asfortranarray(P @ A0)
    W, ipiv, info = O.mxp_getrf_piv(A, nb, prec)
    assert info == 0
    # every multiplier of L0 is at most 1/2 in magnitude, so the pivot search
    # finds the permuted row of A0 each time and the factors are L0, U0
    assert np.array_equal(np.tril(W, -1) + np.eye(n), L0.astype(np.float32))
    assert np.array_equal(np.triu(W), U0.astype(np.float32))
    PA = O.laswp(A.copy(order="F"), 0, n, ipiv)
    assert np.array_equal(PA, A0)


@pytest.mark.parametrize("prec", [O.BF16, O.E4M3], ids=["bf16", "e4m3"])
def test_pivoted_wilkinson_ties_and_growth(prec):
    n = 20
    A = inputs.wilkinson_growth(n)
    W, ipiv, info = O.mxp_getrf_piv(A, 8, prec)
    assert info == 0
    assert np.array_equal(ipiv, np.arange(1, n + 1))  # +-1 ties go to the first row
    assert np.array_equal(W[:, n - 1], (2.0 ** np.arange(n)).astype(np.float32))


def test_pivoted_backward_error_bound_and_a_planted_mistake():
    """With BF16 operands every quantized L21 and U12 entry is within u = 2^-9
    (relative) of its FP32 value, so each product of the trailing updates is
    off by at most (2u + u^2) |l||u|, and the FP32 arithmetic of the panels,
    substitutions and updates adds gamma_n = n 2^-24 / (1 - n 2^-24):
    |P A - L U| <= (2u + u^2 + gamma_n) |L||U| elementwise.  The same factors
    with the later panels' interchanges taken back out of the first panel's
    L columns (the slip of applying interchanges only to the right of the
    panel) break the bound."""
    n, nb = 200, 64
    u, gam = 2.0 ** -9, n * 2.0 ** -24 / (1 - n * 2.0 ** -24)
    A = inputs.uniform((n, n), seed=11)
    W, ipiv, info = O.mxp_getrf_piv(A, nb, O.BF16)
    assert info == 0
    L = np.tril(W.astype(np.float64), -1) + np.eye(n)
    U = np.triu(W.astype(np.float64))
    PA = O.laswp(A.copy(order="F"), 0, n, ipiv)
    c = 2 * u + u * u + gam
    assert np.all(np.abs(PA - L @ U) <= c * (np.abs(L) @ np.abs(U)))
    Lb = L.copy()
    for j in range(n - 1, nb - 1, -1):  # the later interchanges, undone in reverse order
        p = ipiv[j] - 1
        if p != j:
            Lb[[j, p], :nb] = Lb[[p, j], :nb]
    assert not np.array_equal(Lb, L)
    assert not np.all(np.abs(PA - Lb @ U) <= c * (np.abs(Lb) @ np.abs(U)))


@pytest.mark.parametrize("r", [1, 3, 6])
def test_gmres_terminates_after_rank_steps(r):
    """A = I + U V^T with M = I: x0 = b, so r0 = -U V^T b lies in range(U),
    which A maps into itself; the Krylov space is range(U) after r steps and
    GMRES ends there, not one step earlier or later."""
    n = 80
    g = np.random.default_rng(r)
    A = np.eye(n) + g.standard_normal((n, r)) @ g.standard_normal((r, n)) / np.sqrt(n)
    b = g.standard_normal(n)
    x, outer, inner = O.gmres_ir(A, b, lambda v: v, m=30)
    assert inner[0] == r
    assert O.residual_dense(A, x, b)[0] < 16 and outer <= 2


def test_gmres_terminates_after_distinct_eigenvalue_count():
    """A diagonal with k distinct entries, none equal to 1 (so that r0 = (I - A) b
    keeps a component in every eigenspace): GMRES ends after exactly k steps."""
    n, k = 90, 5
    d = np.repeat(np.array([2.0, 3.5, 5.0, 9.0, 12.0]), n // k)
    A = np.diag(d)
    b = np.random.default_rng(2).standard_normal(n)
    x, outer, inner = O.gmres_ir(A, b, lambda v: v, m=30)
    assert inner[0] == k
    assert np.max(np.abs(x - b / d)) <= 1e-12 * np.max(np.abs(b / d))


def test_gmres_ir_with_an_exact_preconditioner_takes_no_step():
    n = 120
    A, b = O.generate(n, 3)
    lu = sla.lu_factor(A)
    x, outer, inner = O.gmres_ir(A, b, lambda v: sla.lu_solve(lu, v))
    assert outer == 0 and inner == []


@pytest.mark.parametrize("n", [512, 1024])
def test_pivoted_bf16_gmres_ir_solves_the_plain_hpl_system(n):
    """On the plain HPL system (no diagonal dominance) the pivoted BF16 factors
    precondition GMRES well enough to reach the FP64 bound."""
    nb = 128
    A, b = O.generate(n, 42)
    W, ipiv, info = O.mxp_getrf_piv(A, nb, O.BF16)
    assert info == 0
    x, outer, inner = O.gmres_ir(A, b, lambda v: O.mxp_getrs_piv(W, ipiv, v))
    assert O.residual_dense(A, x, b)[0] < 16 and outer <= 3
    x64 = np.linalg.solve(A, b)
    assert np.max(np.abs(x - x64)) / np.max(np.abs(x64)) < 1e-10


def test_pivoted_e4m3_does_not_precondition_the_plain_hpl_system():
    """A recorded limit: with E4M3 factors (unit roundoff 2^-4 against a
    condition number near 1e5) GMRES(50) makes almost no progress, so the
    E4M3 variant stays on diagonally dominant systems."""
    n, nb = 512, 128
    A, b = O.generate(n, 42)
    W, ipiv, info = O.mxp_getrf_piv(A, nb, O.E4M3)
    x, outer, inner = O.gmres_ir(A, b, lambda v: O.mxp_getrs_piv(W, ipiv, v), outer_max=3)
    assert O.residual_dense(A, x, b)[0] > 16 and inner == [50, 50, 50]
