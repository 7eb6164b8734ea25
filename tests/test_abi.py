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
