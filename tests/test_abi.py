"""CPU-side checks of the C ABI (no GPU): the library builds, exports every
entry point that include/hplgb.h declares, validates arguments before touching
the GPU, and reports host-side injected faults."""
from __future__ import annotations

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2304_10397_gb300 import build as B
    B.build()
    import paper_2304_10397_gb300 as H
    return H.load_library()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(hpl_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("hpl_generate", "hpl_getrf", "hpl_getrs", "hpl_residual", "hpl_outer_update"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2304_10397_gb300 as H
    assert sorted(set(H.EXPORTS)) == declared_functions()


def test_argument_checks(L):
    vp = C.c_void_p
    assert L.hpl_getrf(C.c_int64(-1), C.c_int64(64), None, C.c_int64(1), None, None, 1, None) == -1
    assert L.hpl_getrf(C.c_int64(10), C.c_int64(0), vp(8), C.c_int64(10), vp(8), None, 1, None) == -2
    assert L.hpl_getrf(C.c_int64(10), C.c_int64(4), None, C.c_int64(10), vp(8), None, 1, None) == -3
    assert L.hpl_getrf(C.c_int64(10), C.c_int64(4), vp(8), C.c_int64(9), vp(8), None, 1, None) == -4
    assert L.hpl_getrf(C.c_int64(10), C.c_int64(4), vp(8), C.c_int64(10), None, None, 1, None) == -5
    assert L.hpl_getrs(b"X", C.c_int64(4), C.c_int64(1), vp(8), C.c_int64(4), None, vp(8), C.c_int64(4), None) == -1
    assert L.hpl_getrs(b"N", C.c_int64(4), C.c_int64(1), vp(8), C.c_int64(3), None, vp(8), C.c_int64(4), None) == -5
    assert L.hpl_dgemm(b"N", b"Q", C.c_int64(1), C.c_int64(1), C.c_int64(1), C.c_double(1), vp(8), C.c_int64(1),
                       vp(8), C.c_int64(1), C.c_double(0), vp(8), C.c_int64(1), None) == -2
    assert L.hpl_generate(C.c_int64(5), C.c_uint64(1), 0, vp(8), C.c_int64(4), None, None) == -5
    L.hpl_last_error.restype = C.c_char_p
    assert b"lda" in L.hpl_last_error()
    i64 = C.c_int64
    assert L.hpl_strsm_llnu(i64(-1), i64(4), vp(8), i64(1), vp(8), i64(1), None) == -1
    assert L.hpl_strsm_llnu(i64(4096), i64(4), vp(8), i64(4096), vp(8), i64(4096), None) == -1
    assert L.hpl_strsm_llnu(i64(8), i64(-4), vp(8), i64(8), vp(8), i64(8), None) == -2
    assert L.hpl_strsm_llnu(i64(8), i64(4), vp(8), i64(7), vp(8), i64(8), None) == -4
    assert L.hpl_strsm_llnu(i64(8), i64(4), vp(8), i64(8), vp(8), i64(7), None) == -6
    assert L.hpl_strsm_llnu(i64(0), i64(4), None, i64(1), None, i64(1), None) == 0
    assert b"ldb" in L.hpl_last_error()


def test_mxp_argument_checks(L):
    # every check runs before any device work, so no GPU is needed
    vp, i64, d = C.c_void_p, C.c_int64, C.c_double
    L.hpl_last_error.restype = C.c_char_p
    # hpl_mxp_getrf(n, nb, prec, A64, lda, LU32, ldl, info, stream)
    assert L.hpl_mxp_getrf(i64(-1), i64(256), 0, vp(8), i64(1), vp(8), i64(1), None, None) == -1
    for nb in (16, 100, 4096):  # below 32, not a multiple of 32, above 2048
        assert L.hpl_mxp_getrf(i64(64), i64(nb), 0, vp(8), i64(64), vp(8), i64(64), None, None) == -2
    assert L.hpl_mxp_getrf(i64(64), i64(64), 2, vp(8), i64(64), vp(8), i64(64), None, None) == -3
    assert L.hpl_mxp_getrf(i64(64), i64(64), 1, None, i64(64), vp(8), i64(64), None, None) == -4
    assert L.hpl_mxp_getrf(i64(64), i64(64), 1, vp(8), i64(63), vp(8), i64(64), None, None) == -5
    assert L.hpl_mxp_getrf(i64(64), i64(64), 1, vp(8), i64(64), None, i64(64), None, None) == -6
    assert L.hpl_mxp_getrf(i64(64), i64(64), 1, vp(8), i64(64), vp(8), i64(63), None, None) == -7
    assert b"ldl" in L.hpl_last_error()
    assert L.hpl_mxp_getrf(i64(0), i64(64), 1, None, i64(1), None, i64(1), None, None) == 0
    # hpl_mxp_getrs(n, LU32, ldl, x, stream)
    assert L.hpl_mxp_getrs(i64(-1), vp(8), i64(1), vp(8), None) == -1
    assert L.hpl_mxp_getrs(i64(8), None, i64(8), vp(8), None) == -2
    assert L.hpl_mxp_getrs(i64(8), vp(8), i64(7), vp(8), None) == -3
    # hpl_mxp_quantize(prec, m2, jb, L21, U12, ld, kp, eL, eU, qL, qU, stream)
    assert L.hpl_mxp_quantize(3, i64(8), i64(8), vp(8), vp(8), i64(8), i64(128), vp(8), vp(8), vp(8), vp(8), None) == -1
    assert L.hpl_mxp_quantize(1, i64(-8), i64(8), vp(8), vp(8), i64(8), i64(128), vp(8), vp(8), vp(8), vp(8),
                              None) == -2
    # kp below jb, or BF16 codes whose K pitch is not a multiple of 128 bytes
    assert L.hpl_mxp_quantize(1, i64(8), i64(200), vp(8), vp(8), i64(200), i64(128), vp(8), vp(8), vp(8), vp(8),
                              None) == -7
    assert L.hpl_mxp_quantize(0, i64(8), i64(8), vp(8), vp(8), i64(8), i64(32), vp(8), vp(8), vp(8), vp(8),
                              None) == -7
    # hpl_mxp_gemm(prec, m, n, kp, qL, qU, eL, eU, C, ldc, stream)
    assert L.hpl_mxp_gemm(2, i64(8), i64(8), i64(128), vp(8), vp(8), vp(8), vp(8), vp(8), i64(8), None) == -1
    assert L.hpl_mxp_gemm(1, i64(-8), i64(8), i64(128), vp(8), vp(8), vp(8), vp(8), vp(8), i64(8), None) == -2
    assert L.hpl_mxp_gemm(1, i64(8), i64(8), i64(128), vp(8), vp(8), vp(8), vp(8), vp(8), i64(7), None) == -10
    # hpl_gmres_ir(n, A, lda, LU32, ldl, b, x, restart, max_outer, inner_tol, target, stats, stream)
    args = lambda **k: [k.get("n", i64(8)), k.get("A", vp(8)), k.get("lda", i64(8)), vp(8), k.get("ldl", i64(8)),
                        vp(8), vp(8), k.get("restart", 50), k.get("outer", 5), d(1e-10), d(16.0), vp(8), None]
    assert L.hpl_gmres_ir(*args(n=i64(0))) == -1
    assert L.hpl_gmres_ir(*args(A=None)) == -2
    assert L.hpl_gmres_ir(*args(lda=i64(7))) == -3
    assert L.hpl_gmres_ir(*args(restart=0)) == -8
    assert L.hpl_gmres_ir(*args(restart=121)) == -8
    assert L.hpl_gmres_ir(*args(outer=0)) == -9
    assert b"max_outer" in L.hpl_last_error()


def test_injected_fault_is_reported_on_host(L, monkeypatch):
    monkeypatch.setenv("HPLGB_FAULT", "getrf")
    vp = C.c_void_p
    assert L.hpl_getrf(C.c_int64(10), C.c_int64(4), vp(8), C.c_int64(10), vp(8), None, 1, None) == -102
    L.hpl_last_error.restype = C.c_char_p
    assert b"HPLGB_FAULT" in L.hpl_last_error()
    monkeypatch.setenv("HPLGB_FAULT", "getrs")
    assert L.hpl_getrs(b"N", C.c_int64(4), C.c_int64(1), vp(8), C.c_int64(4), None, vp(8), C.c_int64(4), None) == -102


def test_zero_sizes_are_no_ops(L):
    # n = 0: nothing is launched, so no device is needed
    assert L.hpl_generate(C.c_int64(0), C.c_uint64(1), 0, None, C.c_int64(1), None, None) == 0
    assert L.hpl_getrs(b"N", C.c_int64(0), C.c_int64(1), None, C.c_int64(1), None, None, C.c_int64(1), None) == 0


def test_null_operands_are_refused_before_the_gpu(L):
    """A NULL operand that a call would read or write is an argument error
    (the argument's position, negated), not a launch; operands that a call
    does not touch (empty products, k = 0) may be NULL."""
    vp, i64, d = C.c_void_p, C.c_int64, C.c_double
    P = vp(64)
    L.hpl_last_error.restype = C.c_char_p
    # hpl_dgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream)
    dg = lambda A, B, Cm, k=4: L.hpl_dgemm(b"N", b"N", i64(4), i64(4), i64(k), d(1), A, i64(4), B, i64(4), d(0),
                                           Cm, i64(4), None)
    assert dg(None, P, P) == -7 and dg(P, None, P) == -9 and dg(P, P, None) == -12
    # hpl_outer_update(m, n, k, alpha, U, ldu, V, ldv, C, ldc, stream)
    ou = lambda U, V, Cm: L.hpl_outer_update(i64(4), i64(4), i64(1), d(1), U, i64(4), V, i64(4), Cm, i64(4), None)
    assert ou(None, P, P) == -5 and ou(P, None, P) == -7 and ou(P, P, None) == -9
    # hpl_laswp(ncols, A, lda, k1, k2, ipiv, stream)
    assert L.hpl_laswp(i64(4), None, i64(4), i64(0), i64(2), P, None) == -2
    assert L.hpl_laswp(i64(4), P, i64(4), i64(0), i64(2), None, None) == -6
    assert L.hpl_laswp(i64(4), None, i64(4), i64(1), i64(1), None, None) == 0  # no interchange: no-op
    # hpl_trsm_llnu(m, n, A, lda, B, ldb, stream)
    assert L.hpl_trsm_llnu(i64(4), i64(4), None, i64(4), P, i64(4), None) == -3
    assert L.hpl_trsm_llnu(i64(4), i64(4), P, i64(4), None, i64(4), None) == -5
    assert L.hpl_trsm_llnu(i64(4), i64(0), None, i64(4), None, i64(4), None) == 0
    # hpl_panel_getrf(m, w, A, lda, ipiv, info, stream)
    assert L.hpl_panel_getrf(i64(16), i64(8), None, i64(16), P, None, None) == -3
    assert L.hpl_panel_getrf(i64(16), i64(8), P, i64(16), None, None, None) == -5
    # hpl_strsm_llnu(m, n, L, ldl, B, ldb, stream)
    assert L.hpl_strsm_llnu(i64(8), i64(4), None, i64(8), P, i64(8), None) == -3
    assert L.hpl_strsm_llnu(i64(8), i64(4), P, i64(8), None, i64(8), None) == -5
    # hpl_mxp_quantize(prec, m2, jb, L21, U12, ld, kp, eL, eU, qL, qU, stream)
    q = [1, i64(8), i64(8), P, P, i64(8), i64(128), P, P, P, P, None]
    for pos, code in ((3, -4), (4, -5), (7, -8), (8, -9), (9, -10), (10, -11)):
        a = list(q)
        a[pos] = None
        assert L.hpl_mxp_quantize(*a) == code
    # hpl_mxp_gemm(prec, m, n, kp, qL, qU, eL, eU, C, ldc, stream)
    g = [1, i64(8), i64(8), i64(128), P, P, P, P, P, i64(8), None]
    for pos, code in ((4, -5), (5, -6), (6, -7), (7, -8), (8, -9)):
        a = list(g)
        a[pos] = None
        assert L.hpl_mxp_gemm(*a) == code
    assert b"C is NULL" in L.hpl_last_error()


def test_remaining_argument_checks(L):
    vp, i64, d = C.c_void_p, C.c_int64, C.c_double
    P = vp(64)
    # hpl_dgemm_emulated(m, n, k, A, lda, B, ldb, C, ldc, slices, stream)
    em = [i64(4), i64(4), i64(4), P, i64(4), P, i64(4), P, i64(4), 0, None]
    for pos, val, code in ((0, i64(-1), -1), (1, i64(-1), -2), (2, i64(-1), -3), (3, None, -4), (4, i64(3), -5),
                           (5, None, -6), (6, i64(3), -7), (7, None, -8), (8, i64(3), -9), (9, -1, -10),
                           (9, 40, -10)):
        a = list(em)
        a[pos] = val
        assert L.hpl_dgemm_emulated(*a) == code, (pos, code)
    # hpl_getrf_emulated(n, nb, A, lda, ipiv, info, lookahead, slices, stream)
    ge = [i64(10), i64(4), P, i64(10), P, None, 1, 0, None]
    for pos, val, code in ((0, i64(-1), -1), (1, i64(0), -2), (2, None, -3), (3, i64(9), -4), (4, None, -5)):
        a = list(ge)
        a[pos] = val
        assert L.hpl_getrf_emulated(*a) == code, (pos, code)
    # hpl_outer_update, hpl_laswp, hpl_trsm_llnu, hpl_panel_getrf: sizes and leading dimensions
    assert L.hpl_outer_update(i64(-1), i64(4), i64(1), d(1), P, i64(4), P, i64(4), P, i64(4), None) == -1
    assert L.hpl_outer_update(i64(4), i64(4), i64(1), d(1), P, i64(4), P, i64(4), P, i64(3), None) == -10
    assert L.hpl_laswp(i64(-1), P, i64(4), i64(0), i64(2), P, None) == -1
    assert L.hpl_laswp(i64(4), P, i64(4), i64(2), i64(1), P, None) == -4
    assert L.hpl_laswp(i64(4), P, i64(1), i64(0), i64(2), P, None) == -3
    assert L.hpl_trsm_llnu(i64(-1), i64(4), P, i64(1), P, i64(1), None) == -1
    assert L.hpl_trsm_llnu(i64(4), i64(4), P, i64(3), P, i64(4), None) == -4
    assert L.hpl_panel_getrf(i64(4), i64(8), P, i64(4), P, None, None) == -2
    assert L.hpl_panel_getrf(i64(4096), i64(2048), P, i64(4096), P, None, None) == -2
    assert L.hpl_panel_getrf(i64(16), i64(8), P, i64(15), P, None, None) == -4
    # hpl_panel_getrf_noalloc: the fixed scratch caps w; info is required
    assert L.hpl_panel_getrf_noalloc(i64(4096), i64(2048), P, i64(4096), P, P, None) == -2
    assert L.hpl_panel_getrf_noalloc(i64(64), i64(8), P, i64(64), P, None, None) == -6
    # hpl_residual(n, seed, dd, A, lda, x, b, out5, stream)
    assert L.hpl_residual(i64(-1), C.c_uint64(1), 0, None, i64(1), P, None, P, None) == -1
    assert L.hpl_residual(i64(4), C.c_uint64(1), 0, P, i64(3), P, None, P, None) == -5
    assert L.hpl_residual(i64(4), C.c_uint64(1), 0, None, i64(4), None, None, P, None) == -6
    assert L.hpl_residual(i64(4), C.c_uint64(1), 0, None, i64(4), P, None, None, None) == -8

