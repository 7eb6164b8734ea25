"""GB300-native High-Performance Linpack hot path: Python binding of libhplgb.

Thin ctypes marshalling over the C ABI of ``include/hplgb.h``; every step of
the computation runs in the library's CUDA kernels.  PyTorch provides device
memory and streams only.  There is no CPU fallback: if the library is not
built, or there is no CUDA device, every call raises.

Matrix convention (as in the C ABI): column-major FP64.  A torch tensor ``M``
of shape (rows, cols) qualifies when ``M.stride(0) == 1`` and
``M.stride(1) >= rows`` (its leading dimension); :func:`colmajor` makes one.
Pivots are int32, 1-based.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "libhplgb.so")
_lock = threading.Lock()
_lib = None

HPL_OK = 0
HPL_ERR_CUDA = -100
HPL_ERR_ALLOC = -101
HPL_ERR_FAULT = -102
HPL_ERR_TIMEOUT = -103
HPL_ERR_NOTSUP = -104

EXPORTS = [
    "hpl_generate", "hpl_getrf", "hpl_getrs", "hpl_residual", "hpl_dgemm", "hpl_outer_update",
    "hpl_laswp", "hpl_trsm_llnu", "hpl_panel_getrf", "hpl_phase_times", "hpl_sync_check",
    "hpl_fp64_peak", "hpl_fp64_dmma_peak", "hpl_kernel_launches", "hpl_last_error", "hpl_finalize",
    "hpl_set_gemm_timing", "hpl_gemm_timing", "hpl_panel_getrf_noalloc", "hpl_fp64_mixed_peak",
    "hpl_workspace_bytes", "hpl_dgemm_emulated", "hpl_getrf_emulated",
    "hpl_mxp_getrf", "hpl_mxp_getrs", "hpl_gmres_ir", "hpl_mxp_quantize", "hpl_mxp_gemm", "hpl_strsm_llnu",
]


class HplError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("hplgb error %d: %s" % (code, msg))
        self.code = code


def load_library(path: str = SO_PATH):
    """Load libhplgb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libhplgb.so is not built (run __graft_entry__.build() or "
                               "python paper_2304_10397_gb300/build.py)")
        L = C.CDLL(path)
        i64, u64, vp, dbl, i32 = C.c_int64, C.c_uint64, C.c_void_p, C.c_double, C.c_int
        L.hpl_generate.argtypes = [i64, u64, i32, vp, i64, vp, vp]
        L.hpl_getrf.argtypes = [i64, i64, vp, i64, vp, vp, i32, vp]
        L.hpl_getrs.argtypes = [C.c_char, i64, i64, vp, i64, vp, vp, i64, vp]
        L.hpl_residual.argtypes = [i64, u64, i32, vp, i64, vp, vp, vp, vp]
        L.hpl_dgemm.argtypes = [C.c_char, C.c_char, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp]
        L.hpl_outer_update.argtypes = [i64, i64, i64, dbl, vp, i64, vp, i64, vp, i64, vp]
        L.hpl_laswp.argtypes = [i64, vp, i64, i64, i64, vp, vp]
        L.hpl_trsm_llnu.argtypes = [i64, i64, vp, i64, vp, i64, vp]
        L.hpl_panel_getrf.argtypes = [i64, i64, vp, i64, vp, vp, vp]
        L.hpl_panel_getrf_noalloc.argtypes = [i64, i64, vp, i64, vp, vp, vp]
        L.hpl_phase_times.argtypes = [vp, i64]
        L.hpl_sync_check.argtypes = [vp]
        L.hpl_fp64_peak.argtypes = [i64, vp, vp]
        L.hpl_fp64_dmma_peak.argtypes = [i64, vp, vp]
        L.hpl_fp64_mixed_peak.argtypes = [i64, i32, i32, vp, vp]
        L.hpl_workspace_bytes.restype = C.c_int64
        L.hpl_dgemm_emulated.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, i32, vp]
        L.hpl_getrf_emulated.argtypes = [i64, i64, vp, i64, vp, vp, i32, i32, vp]
        L.hpl_mxp_getrf.argtypes = [i64, i64, i32, vp, i64, vp, i64, vp, vp]
        L.hpl_mxp_getrs.argtypes = [i64, vp, i64, vp, vp]
        L.hpl_gmres_ir.argtypes = [i64, vp, i64, vp, i64, vp, vp, i32, i32, dbl, dbl, vp, vp]
        L.hpl_mxp_quantize.argtypes = [i32, i64, i64, vp, vp, i64, i64, vp, vp, vp, vp, vp]
        L.hpl_mxp_gemm.argtypes = [i32, i64, i64, i64, vp, vp, vp, vp, vp, i64, vp]
        L.hpl_strsm_llnu.argtypes = [i64, i64, vp, i64, vp, i64, vp]
        L.hpl_set_gemm_timing.argtypes = [i32]
        L.hpl_gemm_timing.argtypes = [vp]
        L.hpl_kernel_launches.restype = C.c_int64
        L.hpl_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def lib():
    return load_library()


def _check(code: int):
    if code != HPL_OK:
        raise HplError(code, lib().hpl_last_error().decode(errors="replace"))


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _mat(M, name, rows=None, cols=None):
    """Validate a column-major FP64 CUDA matrix and return its leading dimension."""
    if not (isinstance(M, torch.Tensor) and M.is_cuda and M.dtype == torch.float64 and M.dim() == 2):
        raise TypeError("%s must be a 2-D float64 CUDA tensor" % name)
    r, c = M.shape
    if (rows is not None and r != rows) or (cols is not None and c != cols):
        raise ValueError("%s has shape %s, expected (%s, %s)" % (name, tuple(M.shape), rows, cols))
    if r > 1 and M.stride(0) != 1:
        raise ValueError("%s must be column-major (stride(0) == 1)" % name)
    ld = M.stride(1) if c > 1 else max(1, r)
    if ld < max(1, r):
        raise ValueError("%s: leading dimension %d < rows %d" % (name, ld, r))
    return ld


def _vec(v, name, n, dtype=torch.float64):
    if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == dtype and v.is_contiguous()
            and v.numel() >= n):
        raise TypeError("%s must be a contiguous %s CUDA tensor with >= %d elements" % (name, dtype, n))


def colmajor(rows: int, cols: int, device="cuda", dtype=torch.float64, ld: int | None = None):
    """Empty column-major (rows x cols) tensor with leading dimension ld."""
    ld = max(1, rows) if ld is None else ld
    base = torch.empty((cols, ld), device=device, dtype=dtype)
    return base.t()[:rows, :]


def to_colmajor(M: torch.Tensor) -> torch.Tensor:
    out = colmajor(M.shape[0], M.shape[1], device=M.device, dtype=M.dtype)
    out.copy_(M)
    return out


# ----------------------------------------------------------------- API

def generate(n: int, seed: int = 42, dd: bool = False, A=None, b=None, with_b: bool = True,
             stream=None):
    """Random system of Sec. II (hpl_generate).  Returns (A, b)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    if A is None:
        A = colmajor(n, n, device=dev)
    if b is None and with_b:
        b = torch.empty(n, device=dev, dtype=torch.float64)
    lda = _mat(A, "A", n, n)
    if b is not None:
        _vec(b, "b", n)
    _check(lib().hpl_generate(n, seed, 1 if dd else 0, _ptr(A), lda, _ptr(b), _stream(stream)))
    return A, b


def getrf(A, nb: int, ipiv=None, info=None, lookahead: bool = True, stream=None):
    """In-place LU with partial pivoting of the square column-major A."""
    n = A.shape[0]
    lda = _mat(A, "A", n, n)
    if ipiv is None:
        ipiv = torch.empty(max(1, n), device=A.device, dtype=torch.int32)
    if info is None:
        info = torch.zeros(1, device=A.device, dtype=torch.int32)
    _vec(ipiv, "ipiv", n, torch.int32)
    _vec(info, "info", 1, torch.int32)
    _check(lib().hpl_getrf(n, nb, _ptr(A), lda, _ptr(ipiv), _ptr(info), 1 if lookahead else 0,
                           _stream(stream)))
    return ipiv, info


def getrf_emulated(A, nb: int, slices: int = 0, ipiv=None, info=None, lookahead: bool = True, stream=None):
    """hpl_getrf with the trailing updates in emulated FP64 (BF16 slice products)."""
    n = A.shape[0]
    lda = _mat(A, "A", n, n)
    if ipiv is None:
        ipiv = torch.empty(max(1, n), device=A.device, dtype=torch.int32)
    if info is None:
        info = torch.zeros(1, device=A.device, dtype=torch.int32)
    _vec(ipiv, "ipiv", n, torch.int32)
    _vec(info, "info", 1, torch.int32)
    _check(lib().hpl_getrf_emulated(n, nb, _ptr(A), lda, _ptr(ipiv), _ptr(info), 1 if lookahead else 0, slices,
                                    _stream(stream)))
    return ipiv, info


def dgemm_emulated(A, B, C_, slices: int = 0, stream=None):
    """C_ <- C_ - A B in FP64 accuracy from BF16 slice products (hpl_dgemm_emulated)."""
    m, k = A.shape
    n = B.shape[1]
    lda, ldb, ldc = _mat(A, "A", m, k), _mat(B, "B", k, n), _mat(C_, "C", m, n)
    _check(lib().hpl_dgemm_emulated(m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(C_), ldc, slices, _stream(stream)))
    return C_


def getrs(trans: str, LU, ipiv, B, stream=None):
    """In-place solve B <- A^-1 B ('N') or A^-T B ('T'); B is (n,) or column-major (n, k)."""
    n = LU.shape[0]
    lda = _mat(LU, "LU", n, n)
    if ipiv is not None:
        _vec(ipiv, "ipiv", n, torch.int32)
    if B.dim() == 1:
        _vec(B, "B", n)
        nrhs, ldb = 1, max(1, n)
    else:
        ldb = _mat(B, "B", n)
        nrhs = B.shape[1]
    _check(lib().hpl_getrs(trans.encode()[:1], n, nrhs, _ptr(LU), lda, _ptr(ipiv), _ptr(B), ldb,
                           _stream(stream)))
    return B


def residual(n: int, seed: int, x, b=None, A=None, dd: bool = False, stream=None) -> np.ndarray:
    """HPL scaled residual and its norms (synchronizes); A/b regenerated when None."""
    _vec(x, "x", n)
    lda = 1
    if A is not None:
        lda = _mat(A, "A", n, n)
    if b is not None:
        _vec(b, "b", n)
    out = np.zeros(5, dtype=np.float64)
    _check(lib().hpl_residual(n, seed, 1 if dd else 0, _ptr(A), lda, _ptr(x), _ptr(b),
                              out.ctypes.data_as(C.c_void_p), _stream(stream)))
    return out


def dgemm(ta: str, tb: str, alpha: float, A, B, beta: float, C_, stream=None):
    m, n = C_.shape
    k = A.shape[0] if ta.upper() == "T" else A.shape[1]
    lda, ldb, ldc = _mat(A, "A"), _mat(B, "B"), _mat(C_, "C")
    _check(lib().hpl_dgemm(ta.encode()[:1], tb.encode()[:1], m, n, k, alpha, _ptr(A), lda, _ptr(B),
                           ldb, beta, _ptr(C_), ldc, _stream(stream)))
    return C_


def outer_update(alpha: float, U, V, C_, stream=None):
    """C = alpha U V^T (rank-k, C not read)."""
    m, k = U.shape
    n = V.shape[0]
    ldu, ldv, ldc = _mat(U, "U", m, k), _mat(V, "V", n, k), _mat(C_, "C", m, n)
    _check(lib().hpl_outer_update(m, n, k, alpha, _ptr(U), ldu, _ptr(V), ldv, _ptr(C_), ldc,
                                  _stream(stream)))
    return C_


def laswp(A, k1: int, k2: int, ipiv, stream=None):
    lda = _mat(A, "A")
    _check(lib().hpl_laswp(A.shape[1], _ptr(A), lda, k1, k2, _ptr(ipiv), _stream(stream)))
    return A


def trsm_llnu(A, B, stream=None):
    m = A.shape[0]
    lda, ldb = _mat(A, "A"), _mat(B, "B", m)
    _check(lib().hpl_trsm_llnu(m, B.shape[1], _ptr(A), lda, _ptr(B), ldb, _stream(stream)))
    return B


def panel_getrf(A, ipiv=None, info=None, stream=None):
    m, w = A.shape
    lda = _mat(A, "A")
    if ipiv is None:
        ipiv = torch.empty(max(1, w), device=A.device, dtype=torch.int32)
    if info is None:
        info = torch.zeros(1, device=A.device, dtype=torch.int32)
    _check(lib().hpl_panel_getrf(m, w, _ptr(A), lda, _ptr(ipiv), _ptr(info), _stream(stream)))
    return ipiv, info


def panel_getrf_noalloc(A, ipiv, info, stream=None):
    """hpl_panel_getrf without device allocations (caller passes ipiv and info)."""
    m, w = A.shape
    lda = _mat(A, "A")
    _vec(ipiv, "ipiv", w, torch.int32)
    _vec(info, "info", 1, torch.int32)
    _check(lib().hpl_panel_getrf_noalloc(m, w, _ptr(A), lda, _ptr(ipiv), _ptr(info), _stream(stream)))
    return ipiv, info


# ------------------------------------------------------- mixed precision

BF16, E4M3 = 0, 1


def _fmat32(M, name, rows=None, cols=None):
    if not (isinstance(M, torch.Tensor) and M.is_cuda and M.dtype == torch.float32 and M.dim() == 2):
        raise TypeError("%s must be a 2-D float32 CUDA tensor" % name)
    r, c = M.shape
    if (rows is not None and r != rows) or (cols is not None and c != cols):
        raise ValueError("%s has shape %s" % (name, tuple(M.shape)))
    if r > 1 and M.stride(0) != 1:
        raise ValueError("%s must be column-major" % name)
    ld = M.stride(1) if c > 1 else max(1, r)
    return ld


def strsm_llnu(L32, B32, stream=None):
    """B32 <- L^-1 B32 in FP32 (L = unit-lower part of the square L32, <= 2048 rows)."""
    m = L32.shape[0]
    ldl = _fmat32(L32, "L32", m, m)
    ldb = _fmat32(B32, "B32", m)
    _check(lib().hpl_strsm_llnu(m, B32.shape[1], _ptr(L32), ldl, _ptr(B32), ldb, _stream(stream)))
    return B32


def mxp_getrf(A64, nb: int, prec: int, LU32=None, info=None, stream=None):
    """FP32 unpivoted mixed-precision LU of the FP64 matrix A64 (not modified)."""
    n = A64.shape[0]
    lda = _mat(A64, "A64", n, n)
    if LU32 is None:
        LU32 = colmajor(n, n, device=A64.device, dtype=torch.float32)
    ldl = _fmat32(LU32, "LU32", n, n)
    if info is None:
        info = torch.zeros(1, device=A64.device, dtype=torch.int32)
    _check(lib().hpl_mxp_getrf(n, nb, prec, _ptr(A64), lda, _ptr(LU32), ldl, _ptr(info), _stream(stream)))
    return LU32, info


def mxp_getrs(LU32, x, stream=None):
    n = LU32.shape[0]
    ldl = _fmat32(LU32, "LU32", n, n)
    _vec(x, "x", n)
    _check(lib().hpl_mxp_getrs(n, _ptr(LU32), ldl, _ptr(x), _stream(stream)))
    return x


def gmres_ir(A64, LU32, b, x=None, restart: int = 50, max_outer: int = 50, inner_tol: float = 1e-10,
             target: float = 16.0, stream=None):
    """FP64 GMRES iterative refinement with the mixed-precision factors."""
    n = A64.shape[0]
    lda = _mat(A64, "A64", n, n)
    ldl = _fmat32(LU32, "LU32", n, n)
    _vec(b, "b", n)
    if x is None:
        x = torch.empty(n, device=A64.device, dtype=torch.float64)
    stats = np.zeros(6, dtype=np.float64)
    _check(lib().hpl_gmres_ir(n, _ptr(A64), lda, _ptr(LU32), ldl, _ptr(b), _ptr(x), restart, max_outer,
                              inner_tol, target, stats.ctypes.data_as(C.c_void_p), _stream(stream)))
    keys = ["outer", "inner", "scaled_residual", "r_inf", "A_inf", "x_inf"]
    return x, dict(zip(keys, stats.tolist()))


def mxp_quantize(prec: int, L21, U12, kp: int, stream=None):
    """Codes and tile exponents of L21 (m2 x jb) and U12 (jb x m2), as in the LU."""
    m2, jb = L21.shape
    ld = _fmat32(L21, "L21")
    if _fmat32(U12, "U12", jb, m2) != ld:
        raise ValueError("L21 and U12 must share the leading dimension")
    nt = max(1, (m2 + 127) // 128)
    eL = torch.zeros(nt, device=L21.device, dtype=torch.int32)
    eU = torch.zeros(nt, device=L21.device, dtype=torch.int32)
    dt = torch.int16 if prec == BF16 else torch.uint8
    qL = torch.zeros((m2, kp), device=L21.device, dtype=dt)
    qU = torch.zeros((m2, kp), device=L21.device, dtype=dt)
    _check(lib().hpl_mxp_quantize(prec, m2, jb, _ptr(L21), _ptr(U12), ld, kp, _ptr(eL), _ptr(eU), _ptr(qL),
                                  _ptr(qU), _stream(stream)))
    return eL, eU, qL, qU


def mxp_gemm(prec: int, qL, qU, eL, eU, C32, stream=None):
    """C32 -= 2^-(eL+eU) qL qU^T on the tensor cores (qL, qU: row-major codes)."""
    m, kp = qL.shape
    n = qU.shape[0]
    for q, name in ((qL, "qL"), (qU, "qU")):
        if not (q.is_cuda and q.is_contiguous() and q.dim() == 2 and q.shape[1] == kp):
            raise ValueError("%s must be a row-major (contiguous) CUDA array of codes with %d columns" % (name, kp))
    ldc = _fmat32(C32, "C", m, n)
    _check(lib().hpl_mxp_gemm(prec, m, n, kp, _ptr(qL), _ptr(qU), _ptr(eL), _ptr(eU), _ptr(C32), ldc,
                              _stream(stream)))
    return C32


def sync_check(stream=None):
    _check(lib().hpl_sync_check(_stream(stream)))


def fp64_peak(iters: int = 20000, stream=None) -> float:
    g = C.c_double(0.0)
    _check(lib().hpl_fp64_peak(iters, C.byref(g), _stream(stream)))
    return g.value


def fp64_dmma_peak(iters: int = 4096, stream=None) -> float:
    g = C.c_double(0.0)
    _check(lib().hpl_fp64_dmma_peak(iters, C.byref(g), _stream(stream)))
    return g.value


def fp64_mixed_peak(iters: int = 4096, dfma_tiles: int = 1, split_warps: bool = False, stream=None) -> float:
    """Total FP64 GFLOP/s of DMMA and DFMA issued together (hpl_fp64_mixed_peak)."""
    g = C.c_double(0.0)
    _check(lib().hpl_fp64_mixed_peak(iters, dfma_tiles, 1 if split_warps else 0, C.byref(g), _stream(stream)))
    return g.value


def workspace_bytes() -> int:
    """Device bytes the library holds as workspace on the current device."""
    return int(lib().hpl_workspace_bytes())


PHASES = ["total", "panel", "laswp", "trsm", "gemm", "quantize", "matvec", "precond", "orth"]


def phase_times() -> dict:
    """Per-phase device ms of the last timed call (HPLGB_TIMERS=1)."""
    out = np.zeros(len(PHASES), dtype=np.float64)
    k = lib().hpl_phase_times(out.ctypes.data_as(C.c_void_p), len(PHASES))
    return dict(zip(PHASES[:k], out[:k].tolist()))


def set_gemm_timing(on: bool):
    _check(lib().hpl_set_gemm_timing(1 if on else 0))


def gemm_timing() -> dict:
    """{launches, ms, flops, bytes} of the trailing updates since set_gemm_timing()."""
    out = np.zeros(4, dtype=np.float64)
    _check(lib().hpl_gemm_timing(out.ctypes.data_as(C.c_void_p)))
    return {"launches": int(out[0]), "ms": float(out[1]), "flops": float(out[2]), "bytes": float(out[3])}


def kernel_launches() -> int:
    return int(lib().hpl_kernel_launches())


def hpl_flops(n: int) -> float:
    """HPL operation count (2/3) N^3 + (3/2) N^2."""
    return (2.0 / 3.0) * n ** 3 + 1.5 * n ** 2
