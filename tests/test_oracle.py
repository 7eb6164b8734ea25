"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: the
published LCG definition computed with Python integers, closed-form LU
factors, brute-force determinants, exact rational arithmetic, LAPACK (scipy /
numpy, run as libraries) and PyTorch autograd.  A plausible slip in the oracle
(a dropped term, a wrong sign or index, a transposed operand, a wrong tie
rule) breaks at least one of them.
"""
from __future__ import annotations

import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests import inputs

M64 = 2 ** 64


def py_lcg_values(seed, count):
    s = seed
    out = []
    for _ in range(count):
        s = (O.LCG_A * s + O.LCG_C) % M64
        out.append((s >> 11) * 2.0 ** -53 - 0.5)
    return out


def py_lcg_state(seed, t):
    """Closed form s_t = a^t s_0 + c (a^t - 1)/(a - 1) mod 2^64, the geometric
    sum taken modulo (a - 1) 2^64 and divided exactly."""
    a, c = O.LCG_A, O.LCG_C
    mod = (a - 1) * M64
    geo = (pow(a, t, mod) - 1) % mod // (a - 1)
    return (pow(a, t, M64) * seed + c * geo) % M64


# ------------------------------------------------------------------ generator

def test_generator_matches_python_lcg_sequence():
    n = 23
    A, b = O.generate(n, seed=42)
    ref = py_lcg_values(42, n * n + n)
    got = list(A.reshape(-1, order="F")) + list(b)
    assert got == ref  # bit-exact


def _golden(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_generator_golden_seed42():
    """The frozen first values of the seed-42 system (tests/golden): the oracle
    still produces them bit for bit, and they are the definition's values
    (Python integers), so the fixture itself is checked too."""
    rows = _golden("generator_n4_seed42.txt")
    n = 4
    A, b = O.generate(n, seed=42)
    ref = py_lcg_values(42, n * n + n)
    seen = 0
    for kind, i, j, v in rows:
        if kind == "A":
            i, j = int(i), int(j)
            assert float.fromhex(v) == A[i, j] == ref[i + j * n]
        elif kind == "b":
            i = int(i)
            assert float.fromhex(v) == b[i] == ref[n * n + i]
        else:
            t = int(i)
            assert int(v) == O.lcg_skip(42, t) == py_lcg_state(42, t)
        seen += 1
    assert seen == n * n + n + 6


@pytest.mark.parametrize("t", [0, 1, 2, 1000, 2 ** 33 + 7, 131072 * 131072 + 5, 2 ** 63 + 12345])
def test_skip_matches_closed_form(t):
    assert O.lcg_skip(42, t) == py_lcg_state(42, t)
    assert O.lcg_skip(7, t) == py_lcg_state(7, t)


def test_generator_moments_and_range():
    A, b = O.generate(1024, seed=3)
    v = A.reshape(-1)
    assert v.min() >= -0.5 and v.max() < 0.5
    assert abs(v.mean()) < 2e-3
    assert abs(v.var() - 1.0 / 12.0) < 1e-3


def test_generator_lda_and_dd():
    n = 17
    A, b = O.generate(n, seed=5)
    Ad, bd = O.generate(n, seed=5, dd=True)
    assert np.array_equal(b, bd)
    off = ~np.eye(n, dtype=bool)
    assert np.array_equal(A[off], Ad[off])
    for i in range(n):
        # plain left-to-right sum in ascending j (an explicit loop: Python's
        # built-in sum() of floats is compensated since 3.12)
        d = 0.0
        for j in range(n):
            if j != i:
                d = d + abs(float(A[i, j]))
        assert Ad[i, i] == d


# ---------------------------------------------------------------------- getrf

def unpack(LU):
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    return L, U


def perm_from_ipiv(ipiv, n):
    p = list(range(n))
    for j, v in enumerate(ipiv):
        q = int(v) - 1
        p[j], p[q] = p[q], p[j]
    return p


def leibniz_det(A):
    n = A.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        prod = 1.0
        for i in range(n):
            prod *= A[i, perm[i]]
        tot += (-1) ** inv * prod
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_det_brute_force(n):
    A = inputs.uniform((n, n), seed=100 + n)
    LU, ipiv, info, st, _ = O.getrf(A)
    assert info == 0 and st == 0
    sign = (-1) ** sum(1 for j in range(n) if ipiv[j] != j + 1)
    det = sign * np.prod(np.diag(LU))
    ref = leibniz_det(A)
    assert abs(det - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("n", [1, 8, 64, 200])
def test_pa_equals_lu(n):
    A = inputs.uniform((n, n), seed=n)
    LU, ipiv, info, st, _ = O.getrf(A)
    L, U = unpack(LU)
    p = perm_from_ipiv(ipiv, n)
    E = A[p, :] - L @ U
    assert np.linalg.norm(E) <= 10 * np.linalg.norm(A) * n * O.EPS
    assert np.all(np.abs(np.tril(LU, -1)) <= 1.0)  # partial pivoting bound
    assert O.factor_error(A, LU, ipiv) <= 10


@pytest.mark.parametrize("n", [4, 31, 96])
def test_dyadic_factors_exact(n):
    L0, U0, A0 = inputs.dyadic_factors(n, seed=n)
    LU, ipiv, info, st, _ = O.getrf(A0)
    assert np.array_equal(ipiv, np.arange(1, n + 1, dtype=np.int32))
    L, U = unpack(LU)
    assert np.array_equal(L, L0)
    assert np.array_equal(U, U0)


@pytest.mark.parametrize("n", [2, 5, 33, 60])
def test_wilkinson_growth(n):
    A = inputs.wilkinson_growth(n)
    LU, ipiv, info, st, _ = O.getrf(A)
    # every column is a magnitude tie, so the smallest-index rule never swaps
    assert np.array_equal(ipiv, np.arange(1, n + 1, dtype=np.int32))
    L, U = unpack(LU)
    assert np.array_equal(L, np.tril(A, -1) + np.eye(n))
    Uref = np.eye(n)
    Uref[:, n - 1] = [2.0 ** i for i in range(n)]  # 2^(i-1), 1-based
    assert np.array_equal(U, Uref)


def test_permutation_matrix():
    n = 40
    P, p = inputs.permutation_matrix(n, seed=9)
    LU, ipiv, info, st, _ = O.getrf(P)
    assert np.array_equal(LU, np.eye(n))
    q = perm_from_ipiv(ipiv, n)
    assert np.array_equal(P[q, :], np.eye(n))


def test_matches_lapack_dgetrf():
    sl = pytest.importorskip("scipy.linalg")
    A, b = O.generate(300, seed=11)
    LU, ipiv, info, st, _ = O.getrf(A)
    lu, piv = sl.lu_factor(A)
    assert np.array_equal(piv + 1, ipiv)
    assert np.max(np.abs(lu - LU)) <= 1e-11


def test_singular_info():
    n = 12
    A = inputs.uniform((n, n), seed=4)
    A[:, 5] = 0.0
    LU, ipiv, info, st, _ = O.getrf(A)
    assert info == 6
    A = inputs.uniform((n, n), seed=4)
    A[:, 0] = 0.0
    A[:, 3] = 0.0
    assert O.getrf(A)[2] == 1


def test_pivot_replay_rule():
    A, b = O.generate(64, seed=42)
    LU, ipiv, info, st, mism = O.getrf(A)
    # identical replay: no mismatch, same factors
    LU2, ipiv2, _, st2, mism2 = O.getrf(A, replay=ipiv)
    assert st2 == 0 and len(mism2) == 0 and np.array_equal(LU, LU2)
    # a replayed pivot far from a tie is rejected at that column
    bad = ipiv.copy()
    j = 3
    alt = [r for r in range(j + 1, 65) if r != ipiv[j]][0]
    bad[j] = alt
    assert O.getrf(A, replay=bad)[3] == -(j + 1)
    # an exact magnitude tie: +x and -x in column 0 -> replaying either is fine
    T = inputs.uniform((8, 8), seed=2)
    T[:, 0] = 0.1
    T[2, 0] = 0.9
    T[6, 0] = -0.9
    LU, ipiv, info, st, mism = O.getrf(T)
    assert ipiv[0] == 3  # smallest index wins the tie
    rep = np.zeros_like(ipiv)  # 0 = no replay for that column
    rep[0] = 7
    LUr, ipr, _, str_, mr = O.getrf(T, replay=rep)
    assert str_ == 0 and list(mr) == [0] and ipr[0] == 7
    assert O.factor_error(T, LUr, ipr) <= 10


def test_nopiv_dyadic_and_dd():
    L0, U0, A0 = inputs.dyadic_factors(24, seed=3)
    LU, info = O.getrf_nopiv(A0)
    L, U = unpack(LU)
    assert info == 0 and np.array_equal(L, L0) and np.array_equal(U, U0)
    A, b = O.generate(150, seed=8, dd=True)
    LU, info = O.getrf_nopiv(A)
    assert info == 0 and O.factor_error(A, LU, None) <= 10


# ---------------------------------------------------------------------- getrs

@pytest.mark.parametrize("n,k", [(1, 1), (50, 1), (200, 3)])
def test_getrs_vs_numpy_solve(n, k):
    A = inputs.uniform((n, n), seed=n + 1)
    B = inputs.uniform((n, k), seed=n + 2)
    LU, ipiv, *_ = O.getrf(A)
    X = O.getrs("N", LU, ipiv, B)
    XT = O.getrs("T", LU, ipiv, B)
    cond = np.linalg.cond(A)
    tol = 50 * cond * n * O.EPS
    Xr = np.linalg.solve(A, B)
    XTr = np.linalg.solve(A.T, B)
    assert np.max(np.abs(X - Xr)) <= tol * np.max(np.abs(Xr))
    assert np.max(np.abs(XT - XTr)) <= tol * np.max(np.abs(XTr))


def test_getrs_adjoint_identity():
    n = 120
    A = inputs.uniform((n, n), seed=21)
    LU, ipiv, *_ = O.getrf(A)
    g = inputs.uniform((n,), seed=22)
    b = inputs.uniform((n,), seed=23)
    lhs = float(np.dot(O.getrs("T", LU, ipiv, g), b))
    rhs = float(np.dot(g, O.getrs("N", LU, ipiv, b)))
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1.0)


def test_getrs_roundtrip_exact_system():
    L0, U0, A0 = inputs.dyadic_factors(40, seed=5)
    xt = inputs.rng(6).integers(-4, 5, size=40).astype(np.float64)
    b = A0 @ xt  # exact
    LU, ipiv, *_ = O.getrf(A0)
    x = O.getrs("N", LU, ipiv, b)
    cond = np.linalg.cond(A0)
    assert np.max(np.abs(x - xt)) <= cond * 40 * O.EPS * 10 * np.max(np.abs(xt))


# ------------------------------------------------------------------- residual

def test_residual_identity_is_zero():
    n = 30
    A = np.asfortranarray(np.eye(n))
    b = inputs.uniform((n,), seed=1)
    out = O.residual_dense(A, b.copy(), b)
    assert out[0] == 0.0 and out[1] == 0.0 and out[2] == 1.0


def test_residual_exact_rational():
    n = 12
    A = inputs.uniform((n, n), seed=31)
    b = inputs.uniform((n,), seed=32)
    x = np.linalg.solve(A, b)  # tiny, nonzero residual
    out = O.residual_dense(A, x, b)
    rex = [sum(Fraction(float(A[i, j])) * Fraction(float(x[j])) for j in range(n)) - Fraction(float(b[i]))
           for i in range(n)]
    rinf = max(abs(r) for r in rex)
    assert rinf > 0
    assert abs(out[1] - float(rinf)) <= 1e-12 * float(rinf)
    anorm = max(sum(abs(Fraction(float(A[i, j]))) for j in range(n)) for i in range(n))
    assert abs(out[2] - float(anorm)) <= 1e-15 * float(anorm)
    scaled = float(rinf) / (O.EPS * (float(anorm) * np.max(np.abs(x)) + np.max(np.abs(b))) * n)
    assert abs(out[0] - scaled) <= 1e-12 * scaled


def test_residual_planted():
    n = 16
    A = inputs.uniform((n, n), seed=41)
    xt = inputs.uniform((n,), seed=42)
    b = A @ xt
    x = xt.copy()
    x[5] += 1e-9  # r = A e5 * 1e-9 up to rounding of b
    out = O.residual_dense(A, x, b)
    assert abs(out[1] - 1e-9 * np.max(np.abs(A[:, 5]))) <= 1e-14


@pytest.mark.parametrize("dd", [False, True])
def test_residual_seeded_equals_dense(dd):
    n = 257
    A, b = O.generate(n, seed=77, dd=dd)
    LU, ipiv, *_ = O.getrf(A)
    x = O.getrs("N", LU, ipiv, b)
    d = O.residual_dense(A, x, b)
    s = O.residual_seeded(n, 77, x, dd=dd)
    assert np.allclose(d, s, rtol=1e-12, atol=0)
    assert d[0] < 16


def test_hpl_residual_passes_n2048():
    n = 2048
    A, b = O.generate(n, seed=42)
    LU, ipiv, info, st, _ = O.getrf(A)
    x = O.getrs("N", LU, ipiv, b)
    out = O.residual_seeded(n, 42, x)
    assert info == 0 and out[0] < 16


def test_factor_error_planted():
    n = 64
    A = inputs.uniform((n, n), seed=51)
    LU, ipiv, *_ = O.getrf(A)
    base = O.factor_error(A, LU, ipiv)
    delta = 1e-6
    k, c = 10, 40
    LU2 = LU.copy()
    LU2[k, c] += delta  # U(k,c): LU changes by L[:,k] * delta in column c
    L, _ = unpack(LU)
    expect = delta * np.linalg.norm(L[:, k]) / (np.linalg.norm(A) * n * O.EPS)
    got = O.factor_error(A, LU2, ipiv)
    assert abs(got - expect) <= 1e-6 * expect + 2 * base


# -------------------------------------------------------------------- adjoint

def test_adjoint_central_fd():
    n, k, h = 64, 3, 1e-6
    A = inputs.uniform((n, n), seed=61) + np.eye(n)
    B = inputs.uniform((n, k), seed=62)
    W = inputs.uniform((n, k), seed=63)
    LU, ipiv, *_ = O.getrf(A)
    X = O.getrs("N", LU, ipiv, B)
    dA, dB = O.solve_adjoint(LU, ipiv, X, W)

    def loss(Am, Bm):
        return float(np.sum(W * np.linalg.solve(Am, Bm)))

    g = inputs.rng(64)
    for _ in range(6):
        i, j = g.integers(0, n, size=2)
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (loss(Ap, B) - loss(Am, B)) / (2 * h)
        assert abs(fd - dA[i, j]) <= 1e-7 * max(1.0, abs(fd))
        r, c = g.integers(0, n), g.integers(0, k)
        Bp, Bm = B.copy(), B.copy()
        Bp[r, c] += h
        Bm[r, c] -= h
        fd = (loss(A, Bp) - loss(A, Bm)) / (2 * h)
        assert abs(fd - dB[r, c]) <= 1e-7 * max(1.0, abs(fd))


def test_adjoint_vs_torch_autograd():
    torch = pytest.importorskip("torch")
    n, k = 100, 4
    A = inputs.uniform((n, n), seed=71)
    B = inputs.uniform((n, k), seed=72)
    W = inputs.uniform((n, k), seed=73)
    LU, ipiv, *_ = O.getrf(A)
    X = O.getrs("N", LU, ipiv, B)
    dA, dB = O.solve_adjoint(LU, ipiv, X, W)
    At = torch.tensor(A, dtype=torch.float64, requires_grad=True)
    Bt = torch.tensor(B, dtype=torch.float64, requires_grad=True)
    (torch.linalg.solve(At, Bt) * torch.tensor(W)).sum().backward()
    assert np.max(np.abs(At.grad.numpy() - dA)) <= 1e-10 * np.max(np.abs(dA))
    assert np.max(np.abs(Bt.grad.numpy() - dB)) <= 1e-10 * np.max(np.abs(dB))


def test_hpl_flops():
    assert O.hpl_flops(2048) == pytest.approx(2 / 3 * 2048 ** 3 + 1.5 * 2048 ** 2)
    assert math.isclose(O.hpl_flops(131072), 1.50122e15, rel_tol=1e-5)


# ----------------------------------------------------- panel / RS / UPDATE

@pytest.mark.parametrize("m,n", [(50, 16), (300, 7), (129, 129), (64, 1)])
def test_rectangular_getrf_vs_lapack(m, n):
    sl = pytest.importorskip("scipy.linalg")
    A = inputs.uniform((m, n), seed=m + n)
    LU, ipiv, info, st, _ = O.getrf(A)
    assert info == 0 and st == 0 and len(ipiv) == min(m, n)
    P, Lr, Ur = sl.lu(A)  # A = P L U
    p = perm_from_ipiv(ipiv, m)
    assert np.array_equal(np.argmax(P, axis=0), np.array(p))  # row i of PA is row p[i] of A
    L = np.tril(LU[:, :n], -1) + np.eye(m, n)
    U = np.triu(LU[:n, :])
    assert np.max(np.abs(L - Lr)) <= 1e-12 and np.max(np.abs(U - Ur)) <= 1e-12


def test_laswp_is_the_interchange_product():
    n = 30
    g = inputs.rng(3)
    ipiv = np.array([g.integers(k, n) + 1 for k in range(n)], dtype=np.int32)
    P = O.laswp(np.eye(n), 0, n, ipiv)
    p = perm_from_ipiv(ipiv, n)
    assert np.array_equal(P, np.eye(n)[p, :])
    A = inputs.uniform((n, 5), seed=4)
    assert np.array_equal(O.laswp(A, 0, n, ipiv), A[p, :])
    # a sub-range k1..k2 leaves the other interchanges out
    q = list(range(n))
    for k in range(4, 11):
        j = ipiv[k] - 1
        q[k], q[j] = q[j], q[k]
    assert np.array_equal(O.laswp(A, 4, 11, ipiv), A[q, :])


def test_trsm_vs_lapack():
    sl = pytest.importorskip("scipy.linalg")
    m, n = 77, 9
    A = inputs.uniform((m, m), seed=5)
    B = inputs.uniform((m, n), seed=6)
    X = O.trsm_llnu(A, B)
    ref = sl.solve_triangular(A, B, lower=True, unit_diagonal=True)
    assert np.max(np.abs(X - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
def test_gemm_exact_integers(ta, tb):
    g = inputs.rng(7)
    m, n, k = 13, 11, 17
    A = g.integers(-9, 10, size=(k, m) if ta == "T" else (m, k)).astype(np.float64)
    B = g.integers(-9, 10, size=(n, k) if tb == "T" else (k, n)).astype(np.float64)
    Cm = g.integers(-9, 10, size=(m, n)).astype(np.float64)
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    got = O.gemm(ta, tb, -1.0, A, B, 1.0, Cm)
    assert np.array_equal(got, Cm - opA @ opB)
    got0 = O.gemm(ta, tb, 2.0, A, B, 0.0, np.full((m, n), np.nan))
    assert np.array_equal(got0, 2.0 * (opA @ opB))


def test_factor_probe_estimates_frobenius_error():
    n, seed = 300, 19
    A, b = O.generate(n, seed=seed)
    LU, ipiv, *_ = O.getrf(A)
    # planted error well above rounding: U(20, 200) += 1e-9
    LU2 = LU.copy()
    LU2[20, 200] += 1e-9
    exact = O.factor_error(A, LU2, ipiv)
    est = np.sqrt(np.mean([O.factor_probe(n, seed, LU2, ipiv, inputs.rng(100 + r).standard_normal(n)) ** 2
                           for r in range(16)]))
    assert 0.5 * exact <= est <= 2.0 * exact
    # an unperturbed factorization reads as tiny
    base = O.factor_probe(n, seed, LU, ipiv, inputs.rng(5).standard_normal(n))
    assert base < 1.0


def test_getrf_steps_is_a_prefix_of_getrf():
    n, s = 120, 37
    A, b = O.generate(n, seed=8)
    LU, ipiv, *_ = O.getrf(A)
    P = np.asfortranarray(A.copy())
    ip = O.getrf_steps_inplace(P, s)
    assert np.array_equal(ip, ipiv[:s])
    assert np.array_equal(P[:s, :], LU[:s, :])  # finished rows of U
    # finished columns of L, once the later interchanges (rows >= s) are applied
    assert np.array_equal(O.laswp(P, s, n, ipiv)[:, :s], LU[:, :s])
    # flop count: step j divides n-1-j entries and does (n-1-j)^2 multiply-subtracts
    brute = 0
    for j in range(s):
        r = n - 1 - j
        brute += r + 2 * r * r
    assert O.getrf_steps_flops(n, s) == brute
    assert O.getrf_steps_flops(n, n) == pytest.approx(2 / 3 * n ** 3, rel=0.03)
