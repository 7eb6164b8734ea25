"""GPU parity tests: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (derivations are in the design notes):
  - generator, interchanges: bit-exact;
  - pivots: identical, except a column where the two candidate rows differ in
    magnitude by less than 1e-13 relative (replayed by the oracle and logged);
  - factorization: ||PA - LU||_F / (||A||_F N eps) <= 10, HPL scaled residual < 16;
  - products and substitutions: the standard componentwise error bound
    |fl(x) - x| <= gamma_k (|A||B|) with gamma_k = k eps / (1 - k eps), applied to
    the difference of two computations (so 2 gamma_k).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from tests import inputs

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53
RTOL_PIV = 1e-13


@pytest.fixture(scope="module")
def H():
    import __graft_entry__ as g
    g.build()
    import paper_2304_10397_gb300 as H
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    H.load_library()
    return H


def dev(M, ld=None):
    """numpy (Fortran) -> column-major CUDA tensor."""
    import paper_2304_10397_gb300 as H
    M = np.asarray(M, dtype=np.float64)
    if M.ndim == 1:
        return torch.from_numpy(M.copy()).cuda()
    T = H.colmajor(M.shape[0], M.shape[1], ld=ld)
    T.copy_(torch.from_numpy(np.ascontiguousarray(M)))
    return T


def host(T):
    torch.cuda.synchronize()
    return np.asfortranarray(T.cpu().numpy())


def gamma(k):
    return k * EPS / (1 - k * EPS)


# ------------------------------------------------------------------ a1 generate

@pytest.mark.parametrize("n,ld", [(1, 1), (257, 300), (1024, 1024)])
@pytest.mark.parametrize("dd", [False, True])
def test_generate_bitwise(H, n, ld, dd):
    A = H.colmajor(n, n, ld=ld)
    b = torch.empty(n, device="cuda", dtype=torch.float64)
    H.generate(n, 42, dd=dd, A=A, b=b)
    Ao, bo = O.generate(n, 42, dd=dd)
    assert np.array_equal(host(A), Ao)
    assert np.array_equal(b.cpu().numpy(), bo)


# -------------------------------------------------------------------- a6 gemm

@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(131, 77, 45), (64, 64, 16), (1, 1, 1), (200, 3, 384), (65, 130, 0),
                                   (1000, 24, 24), (777, 8, 16), (300, 32, 32), (513, 33, 24), (513, 24, 33)])
def test_dgemm_parity(H, ta, tb, m, n, k):
    # n, k <= 32 without transposes takes the skinny kernel of the panel
    # recursion's narrow updates; 33 on either side the tiled one
    A = inputs.uniform((k, m) if ta == "T" else (m, k), seed=m + 1)
    B = inputs.uniform((n, k) if tb == "T" else (k, n), seed=n + 2)
    Cm = inputs.uniform((m, n), seed=k + 3)
    ref = O.gemm(ta, tb, -1.0, A, B, 1.0, Cm)
    Cd = dev(Cm, ld=m + 3)
    H.dgemm(ta, tb, -1.0, dev(A) if A.size else H.colmajor(*A.shape), dev(B) if B.size else H.colmajor(*B.shape),
            1.0, Cd)
    got = host(Cd)
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    bound = 2 * gamma(k + 1) * (np.abs(opA) @ np.abs(opB) + np.abs(Cm))
    assert np.all(np.abs(got - ref) <= bound + 1e-300)


def test_dgemm_skinny_alpha_beta(H):
    # C = alpha A B + beta C on the skinny path: beta = 0 (C not read) and a general alpha, beta
    m, n, k = 2049, 17, 9
    A = inputs.uniform((m, k), seed=5)
    B = inputs.uniform((k, n), seed=6)
    for alpha, beta in ((0.75, 0.0), (-1.5, 0.25)):
        Cm = inputs.uniform((m, n), seed=7) if beta != 0.0 else np.full((m, n), np.nan)
        ref = O.gemm("N", "N", alpha, A, B, beta, np.nan_to_num(Cm))
        Cd = dev(Cm)
        H.dgemm("N", "N", alpha, dev(A), dev(B), beta, Cd)
        bound = 2 * gamma(k + 1) * (abs(alpha) * (np.abs(A) @ np.abs(B)) + abs(beta) * np.abs(np.nan_to_num(Cm)))
        assert np.all(np.abs(host(Cd) - ref) <= bound + 1e-300)


def test_outer_update_parity(H):
    m, n, k = 300, 200, 64
    U = inputs.uniform((m, k), seed=1)
    V = inputs.uniform((n, k), seed=2)
    Cd = dev(np.full((m, n), np.nan))  # not read
    H.outer_update(-1.0, dev(U), dev(V), Cd)
    ref = O.gemm("N", "T", -1.0, U, V, 0.0, np.zeros((m, n)))
    assert np.all(np.abs(host(Cd) - ref) <= 2 * gamma(k) * (np.abs(U) @ np.abs(V).T))


# ------------------------------------------------------------------- a4 laswp

def random_ipiv(n, seed, k1=0, k2=None, rows=None):
    g = inputs.rng(seed)
    rows = n if rows is None else rows
    k2 = n if k2 is None else k2
    ipiv = np.arange(1, n + 1, dtype=np.int32)
    for k in range(k1, k2):
        r = g.random()
        if r < 0.1:
            ipiv[k] = k + 1                     # no interchange
        elif r < 0.3:
            ipiv[k] = min(rows, k2) if k2 <= rows else rows  # repeated target
        else:
            ipiv[k] = g.integers(k, rows) + 1
    return ipiv


@pytest.mark.parametrize("k1,k2", [(0, 512), (100, 612), (900, 1000), (5, 6), (0, 1000)])
def test_laswp_bitwise(H, k1, k2):
    n, ncols = 1000, 37
    ipiv = random_ipiv(n, seed=k1 + k2, k1=k1, k2=k2)
    A = inputs.uniform((n, ncols), seed=3)
    ref = O.laswp(A, k1, k2, ipiv)
    Ad = dev(A, ld=1003)
    H.laswp(Ad, k1, k2, torch.from_numpy(ipiv).cuda())
    assert np.array_equal(host(Ad), ref)


# -------------------------------------------------------------------- a5 trsm

@pytest.mark.parametrize("m", [1, 16, 24, 31, 32, 33, 64, 65, 100, 128, 256, 384, 512, 1000])
@pytest.mark.parametrize("n", [1, 17, 300, 2000])
def test_trsm_parity(H, m, n):
    # a warp per column for m <= 32, for m <= 64 on up to 4096 columns and for
    # m <= 128 on up to 1024; otherwise the strip kernel up to 256 rows, then
    # blocked by 128 rows (each block by one of the two)
    Lsrc, *_ = O.getrf(inputs.uniform((m, m), seed=m))  # a pivoted L: |l_ij| <= 1
    B = inputs.uniform((m, n), seed=n)
    ref = O.trsm_llnu(Lsrc, B)
    Bd = dev(B)
    H.trsm_llnu(dev(Lsrc, ld=m + 1), Bd)
    got = host(Bd)
    L = np.tril(Lsrc, -1) + np.eye(m)
    # substitution: (L + dL) X^ = B, |dL| <= gamma_m |L|, so
    # |X^ - X| <= gamma_m |L^-1| |L| |X|; twice that for two computations
    bound = 2 * gamma(m) * (np.abs(np.linalg.inv(L)) @ (np.abs(L) @ np.abs(ref))) + 1e-300
    assert np.all(np.abs(got - ref) <= bound)


# ------------------------------------------------------------- a2/a3 panel FACT

def compare_pivots(gpu_ipiv, A, rows_label=""):
    """Oracle factorization replaying the GPU pivots under the 1e-13 rule."""
    LU, ipiv, info, st, mism = O.getrf(A, replay=gpu_ipiv, rtol=RTOL_PIV)
    assert st == 0, "pivot of column %d differs beyond the tie tolerance %s" % (-st - 1, rows_label)
    assert np.array_equal(ipiv, gpu_ipiv)
    return LU, info, mism


@pytest.mark.parametrize("m,w", [(1000, 16), (1000, 64), (4096, 256), (3000, 384), (517, 100), (33, 33),
                                  (20000, 512), (7, 1)])
def test_panel_parity(H, m, w):
    A = inputs.uniform((m, w), seed=m * 7 + w)
    Ad = dev(A, ld=m + 1)
    ipiv, info = H.panel_getrf(Ad)
    H.sync_check()
    gp = ipiv.cpu().numpy()[:w]
    LU, oinfo, mism = compare_pivots(gp, A, "(panel %dx%d)" % (m, w))
    got = host(Ad)
    assert int(info.item()) == oinfo == 0
    # same pivots: both are backward-stable eliminations of the same PA
    assert np.max(np.abs(got - LU)) <= 1e-11 * max(1.0, np.max(np.abs(LU)))


# ----------------------------------------------------------------- full getrf

def factor_and_check(H, n, nb, ld=None, seed=42, lookahead=True):
    A_d = H.colmajor(n, n, ld=ld or n)
    b_d = torch.empty(n, device="cuda", dtype=torch.float64)
    H.generate(n, seed, A=A_d, b=b_d)
    ipiv, info = H.getrf(A_d, nb, lookahead=lookahead)
    x = b_d.clone()
    H.getrs("N", A_d, ipiv, x)
    H.sync_check()
    res_gpu = H.residual(n, seed, x)
    A, b = O.generate(n, seed)
    gp = ipiv.cpu().numpy()[:n]
    LU, oinfo, mism = compare_pivots(gp, A, "(getrf n=%d nb=%d)" % (n, nb))
    LUg = host(A_d)
    ferr = O.factor_error(A, LUg, gp)
    res_orc = O.residual_dense(A, x.cpu().numpy(), b)
    return dict(info=int(info.item()), oinfo=oinfo, mism=mism, ferr=ferr, res_gpu=res_gpu,
                res_orc=res_orc, LUg=LUg, LU=LU, x=x.cpu().numpy(), A=A, b=b, ipiv=gp)


def test_getrf_n2048_nb256(H):
    r = factor_and_check(H, 2048, 256)
    assert r["info"] == 0 and r["oinfo"] == 0
    assert r["ferr"] <= 10
    assert r["res_orc"][0] < 16 and r["res_gpu"][0] < 16
    # the GPU residual kernel against the oracle's (both Dot2-accurate)
    assert np.allclose(r["res_gpu"], r["res_orc"], rtol=1e-6, atol=0)
    assert np.max(np.abs(r["LUg"] - r["LU"])) <= 1e-10 * np.max(np.abs(r["LU"]))
    print("n=2048 ferr=%.3g res=%.3g mism=%d maxdiff=%.3g" % (
        r["ferr"], r["res_orc"][0], len(r["mism"]), np.max(np.abs(r["LUg"] - r["LU"]))))


@pytest.mark.parametrize("n,nb,ld,la", [(1000, 96, 1000, True), (333, 64, 400, True), (1, 1, 1, True),
                                         (17, 16, 17, True), (300, 512, 300, True), (1500, 256, 1501, False),
                                         (640, 128, 640, True), (2000, 384, 2000, True)])
def test_getrf_ragged(H, n, nb, ld, la):
    r = factor_and_check(H, n, nb, ld=ld, seed=n + nb, lookahead=la)
    assert r["info"] == 0 and r["ferr"] <= 10 and r["res_orc"][0] < 16
    assert np.max(np.abs(r["LUg"] - r["LU"])) <= 1e-10 * max(1.0, np.max(np.abs(r["LU"])))


def test_getrf_zero_size(H):
    A = H.colmajor(0, 0)
    ipiv, info = H.getrf(A, 64)
    torch.cuda.synchronize()
    assert int(info.item()) == 0


def test_getrf_singular_info(H):
    n = 700
    A = inputs.uniform((n, n), seed=9)
    A[:, 401] = 0.0
    Ad = dev(A)
    ipiv, info = H.getrf(Ad, 128)
    H.sync_check()
    _, _, oinfo, st, _ = O.getrf(A, replay=ipiv.cpu().numpy()[:n])
    assert st == 0 and int(info.item()) == oinfo == 402


@pytest.mark.parametrize("n,nb", [(60, 16), (60, 32)])
def test_getrf_wilkinson_exact(H, n, nb):
    A = inputs.wilkinson_growth(n)
    Ad = dev(A)
    ipiv, info = H.getrf(Ad, nb)
    LU = host(Ad)
    assert np.array_equal(ipiv.cpu().numpy()[:n], np.arange(1, n + 1))
    U = np.triu(LU)
    Uref = np.eye(n)
    Uref[:, n - 1] = [2.0 ** i for i in range(n)]
    assert np.array_equal(U, Uref)
    assert np.array_equal(np.tril(LU, -1), np.tril(A, -1))


@pytest.mark.parametrize("n,nb", [(96, 32), (200, 64)])
def test_getrf_dyadic_exact(H, n, nb):
    L0, U0, A0 = inputs.dyadic_factors(n, seed=n)
    Ad = dev(A0)
    ipiv, info = H.getrf(Ad, nb)
    LU = host(Ad)
    assert np.array_equal(ipiv.cpu().numpy()[:n], np.arange(1, n + 1))
    assert np.array_equal(np.tril(LU, -1) + np.eye(n), L0)
    assert np.array_equal(np.triu(LU), U0)


def test_getrf_permutation_matrix(H):
    n = 300
    P, p = inputs.permutation_matrix(n, seed=3)
    Ad = dev(P)
    ipiv, info = H.getrf(Ad, 64)
    assert np.array_equal(host(Ad), np.eye(n))
    LU, oipiv, *_ = O.getrf(P)
    assert np.array_equal(ipiv.cpu().numpy()[:n], oipiv)


# -------------------------------------------------------------------- a8 getrs

@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("nrhs", [1, 3, 64])
def test_getrs_parity(H, trans, nrhs):
    n = 1000
    A = inputs.uniform((n, n), seed=11)
    Ad = dev(A)
    ipiv, info = H.getrf(Ad, 128)
    LU = host(Ad)
    gp = ipiv.cpu().numpy()[:n]
    B = inputs.uniform((n, nrhs), seed=12)
    ref = O.getrs(trans, LU, gp, B)
    Bd = dev(B)
    H.getrs(trans, Ad, ipiv, Bd)
    got = host(Bd)
    cond = np.linalg.cond(A, 1)
    assert np.max(np.abs(got - ref)) <= 10 * cond * n * EPS * np.max(np.abs(ref))


def test_getrs_vector_and_unpivoted(H):
    n = 700
    A, b = O.generate(n, 5, dd=True)
    LU, info = O.getrf_nopiv(A)
    ref = O.getrs("N", LU, None, b)
    x = torch.from_numpy(b.copy()).cuda()
    H.getrs("N", dev(LU), None, x)
    assert np.max(np.abs(x.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))


# ----------------------------------------------------------------- a9 residual

@pytest.mark.parametrize("dd", [False, True])
def test_residual_parity(H, dd):
    n = 1100
    A, b = O.generate(n, 77, dd=dd)
    LU, ipiv, *_ = O.getrf(A)
    x = O.getrs("N", LU, ipiv, b)
    ref = O.residual_dense(A, x, b)
    xd = torch.from_numpy(x).cuda()
    got_regen = H.residual(n, 77, xd, dd=dd)
    got_stored = H.residual(n, 77, xd, b=torch.from_numpy(b).cuda(), A=dev(A, ld=n + 5))
    assert np.allclose(got_regen, ref, rtol=1e-9, atol=0)
    assert np.allclose(got_stored, ref, rtol=1e-9, atol=0)


def test_residual_identity(H):
    n = 64
    b = inputs.uniform((n,), seed=1)
    out = H.residual(n, 0, torch.from_numpy(b).cuda(), b=torch.from_numpy(b).cuda(), A=dev(np.eye(n)))
    assert out[0] == 0.0 and out[2] == 1.0


# --------------------------------------------------------- full-size (bench) case

def test_getrf_full_size_n32768_nb384(H):
    """The benchmarked configuration: residual by the oracle (regenerated A) and
    a Freivalds probe of ||PA - LU||_F (the oracle cannot factor this size)."""
    n, nb, seed = 32768, 384, 42
    A_d = H.colmajor(n, n)
    b_d = torch.empty(n, device="cuda", dtype=torch.float64)
    H.generate(n, seed, A=A_d, b=b_d)
    ipiv, info = H.getrf(A_d, nb, lookahead=True)
    x = b_d.clone()
    H.getrs("N", A_d, ipiv, x)
    H.sync_check()
    assert int(info.item()) == 0
    xh = x.cpu().numpy()
    res_orc = O.residual_seeded(n, seed, xh)
    res_gpu = H.residual(n, seed, x)
    assert res_orc[0] < 16
    assert np.allclose(res_gpu, res_orc, rtol=1e-6, atol=0)
    gp = ipiv.cpu().numpy()[:n]
    assert np.all(gp >= np.arange(1, n + 1)) and np.all(gp <= n)
    LUh = host(A_d)
    del A_d
    probe = O.factor_probe(n, seed, LUh, gp, inputs.rng(1).standard_normal(n))
    assert probe <= 10
    print("n=32768 res=%.4g probe=%.4g" % (res_orc[0], probe))
