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
