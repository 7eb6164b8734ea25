"""CPU oracle for the HPL hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct FP64 implementation of what the CUDA library
computes (random system of Sec. II, LU with partial pivoting and the
triangular solves of Sec. I/II, the HPL scaled residual, the adjoint of the
solve).  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library and never calls it.

The arithmetic lives in ``hpl_oracle.c`` (plain C, ``-ffp-contract=off``);
this module only marshals numpy arrays through ctypes.  Matrices are numpy
arrays in Fortran (column-major) order; ``lda`` is their leading dimension.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libhpl_oracle.so")
_lock = threading.Lock()
_lib = None

EPS = 2.0 ** -53  # unit roundoff used by the HPL residual (reading of Sec. II)
LCG_A = 6364136223846793005
LCG_C = 1442695040888963407


def build(force: bool = False) -> str:
    """Compile hpl_oracle.c into a shared library next to it (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            i64, u64, dp, ip = C.c_int64, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_int32)
            L.orc_value.restype = C.c_double
            L.orc_value.argtypes = [u64]
            L.orc_lcg_skip.restype = u64
            L.orc_lcg_skip.argtypes = [u64, u64]
            L.orc_generate.argtypes = [i64, u64, dp, i64, dp]
            L.orc_generate_dd.argtypes = [i64, u64, dp, i64, dp]
            L.orc_getrf.restype = C.c_int
            L.orc_getrf.argtypes = [i64, dp, i64, ip, ip, ip, C.c_double,
                                    C.POINTER(C.c_int64), i64, C.POINTER(C.c_int64)]
            L.orc_getrf_mn.restype = C.c_int
            L.orc_getrf_mn.argtypes = [i64, i64, dp, i64, ip, ip, ip, C.c_double,
                                       C.POINTER(C.c_int64), i64, C.POINTER(C.c_int64)]
            L.orc_getrf_steps.restype = C.c_int
            L.orc_getrf_steps.argtypes = [i64, i64, i64, dp, i64, ip, ip]
            L.orc_laswp.argtypes = [i64, dp, i64, i64, i64, ip]
            L.orc_trsm_llnu.argtypes = [i64, i64, dp, i64, dp, i64]
            L.orc_gemm.argtypes = [C.c_char, C.c_char, i64, i64, i64, C.c_double, dp, i64, dp, i64,
                                   C.c_double, dp, i64]
            L.orc_factor_probe.restype = C.c_double
            L.orc_factor_probe.argtypes = [i64, u64, dp, i64, ip, dp]
            L.orc_getrf_nopiv.argtypes = [i64, dp, i64, ip]
            L.orc_getrs.argtypes = [C.c_char, i64, i64, dp, i64, ip, dp, i64]
            L.orc_residual_dense.argtypes = [i64, dp, i64, dp, dp, dp]
            L.orc_residual_seeded.argtypes = [i64, u64, C.c_int, dp, dp, dp]
            L.orc_factor_error.restype = C.c_double
            L.orc_factor_error.argtypes = [i64, dp, i64, dp, i64, ip]
            L.orc_solve_adjoint.argtypes = [i64, i64, dp, i64, ip, dp, i64, dp, i64, dp, i64, dp, i64]
            L.orc_f32_to_bf16.restype = C.c_uint16
            L.orc_f32_to_bf16.argtypes = [C.c_float]
            L.orc_bf16_to_f32.restype = C.c_float
            L.orc_bf16_to_f32.argtypes = [C.c_uint16]
            L.orc_f32_to_e4m3.restype = C.c_uint8
            L.orc_f32_to_e4m3.argtypes = [C.c_float]
            L.orc_e4m3_to_f32.restype = C.c_float
            L.orc_e4m3_to_f32.argtypes = [C.c_uint8]
            L.orc_scale_exp.restype = C.c_int
            L.orc_scale_exp.argtypes = [C.c_double, C.c_double]
            L.orc_qmax.restype = C.c_double
            L.orc_qmax.argtypes = [C.c_int]
            fp = C.POINTER(C.c_float)
            L.orc_tile_exps.argtypes = [i64, i64, fp, i64, C.c_int, C.c_int, ip]
            L.orc_quantize.argtypes = [i64, i64, fp, i64, C.c_int, C.c_int, ip, C.POINTER(C.c_uint16)]
            L.orc_mxp_getrf.argtypes = [i64, i64, C.c_int, dp, i64, fp, i64, ip]
            L.orc_mxp_getrf_ex.argtypes = [i64, i64, C.c_int, dp, i64, fp, i64, ip, fp, i64, i64, C.c_double]
            L.orc_mxp_getrs.argtypes = [i64, fp, i64, dp]
            L.orc_mxp_getrf_piv.argtypes = [i64, i64, C.c_int, dp, i64, fp, i64, ip, ip]
            L.orc_mxp_getrs_piv.argtypes = [i64, fp, i64, ip, dp]
            L.orc_ozaki_gemm.argtypes = [i64, i64, i64, C.c_int, C.c_int, dp, i64, dp, i64, dp, i64]
            L.orc_ozaki_gemm.restype = C.c_int
            L.orc_ozaki_split_rows.argtypes = [i64, i64, dp, i64, C.c_int, C.c_int, ip, dp]
            L.orc_ozaki_split_cols.argtypes = [i64, i64, dp, i64, C.c_int, C.c_int, ip, dp]
            L.orc_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


def _fmat(a):
    a = np.asarray(a, dtype=np.float64)
    if not a.flags.f_contiguous:
        a = np.asfortranarray(a)
    return a


def _ld(a):
    return max(1, a.shape[0])


def num_threads() -> int:
    return int(lib().orc_num_threads())


def value(state: int) -> float:
    return float(lib().orc_value(state & (2 ** 64 - 1)))


def lcg_skip(seed: int, t: int) -> int:
    return int(lib().orc_lcg_skip(seed, t))


def generate(n: int, seed: int = 42, dd: bool = False):
    """Random system of Sec. II: (A, b), A Fortran-ordered n x n."""
    A = np.zeros((n, n), dtype=np.float64, order="F")
    b = np.zeros(n, dtype=np.float64)
    f = lib().orc_generate_dd if dd else lib().orc_generate
    f(n, seed, _dp(A), _ld(A), _dp(b))
    return A, b


def getrf(A, replay=None, rtol: float = 1e-13, mism_cap: int = 4096):
    """LU with partial pivoting (unblocked right-looking) of an m x n matrix.

    Returns (LU, ipiv[int32, 1-based], info, status, mismatch_columns).
    status = 0, or -(j+1) if the replayed pivot of column j breaks the
    tolerance rule (factorization stopped there)."""
    LU = _fmat(np.array(A, dtype=np.float64, order="F", copy=True))
    m, n = LU.shape
    ipiv = np.zeros(max(1, min(m, n)), dtype=np.int32)
    info = np.zeros(1, dtype=np.int32)
    mism = np.zeros(max(1, mism_cap), dtype=np.int64)
    nm = C.c_int64(0)
    rp = None
    if replay is not None:
        rp = np.ascontiguousarray(replay, dtype=np.int32)
        assert rp.shape[0] >= min(m, n)
    st = lib().orc_getrf_mn(m, n, _dp(LU), _ld(LU), _ip(ipiv), _ip(info), _ip(rp), rtol,
                            mism.ctypes.data_as(C.POINTER(C.c_int64)), mism_cap, C.byref(nm))
    return LU, ipiv[: min(m, n)], int(info[0]), int(st), mism[: min(nm.value, mism_cap)].copy()


def getrf_steps_inplace(A, steps: int):
    """Run the first `steps` elimination steps of getrf in place on the Fortran
    array A (a bounded sample of the factorization, for timing)."""
    assert A.flags.f_contiguous and A.dtype == np.float64
    m, n = A.shape
    ipiv = np.zeros(max(1, min(m, n)), dtype=np.int32)
    info = np.zeros(1, dtype=np.int32)
    lib().orc_getrf_steps(m, n, steps, _dp(A), _ld(A), _ip(ipiv), _ip(info))
    return ipiv[:steps]


def getrf_steps_flops(n: int, steps: int) -> float:
    """Algorithmic flops of the first `steps` steps of an n x n elimination:
    step j divides n-1-j entries and updates (n-1-j)^2 of them (2 flops each)."""
    return float(sum(2 * (n - 1 - j) ** 2 + (n - 1 - j) for j in range(min(steps, n))))


def laswp(A, k1: int, k2: int, ipiv):
    """Apply interchanges k1..k2-1 (1-based values) to the rows of a copy of A."""
    X = np.array(A, dtype=np.float64, order="F", copy=True)
    ip = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib().orc_laswp(X.shape[1], _dp(X), _ld(X), k1, k2, _ip(ip))
    return X


def trsm_llnu(A, B):
    """L^-1 B with L the unit-lower triangle of the square A."""
    A = _fmat(A)
    X = np.array(B, dtype=np.float64, order="F", copy=True)
    lib().orc_trsm_llnu(X.shape[0], X.shape[1], _dp(A), _ld(A), _dp(X), _ld(X))
    return X


def gemm(ta: str, tb: str, alpha: float, A, B, beta: float, Cm):
    A = _fmat(A)
    B = _fmat(B)
    X = np.array(Cm, dtype=np.float64, order="F", copy=True)
    m, n = X.shape
    k = A.shape[0] if ta.upper() == "T" else A.shape[1]
    lib().orc_gemm(ta.encode()[:1], tb.encode()[:1], m, n, k, alpha, _dp(A), _ld(A), _dp(B), _ld(B),
                   beta, _dp(X), _ld(X))
    return X


def factor_probe(n: int, seed: int, LU, ipiv, v):
    """Freivalds estimate of ||PA - LU||_F / (||A||_F n eps), A regenerated."""
    LU = _fmat(LU)
    v = np.ascontiguousarray(v, dtype=np.float64)
    ip = np.ascontiguousarray(ipiv, dtype=np.int32)
    return float(lib().orc_factor_probe(n, seed, _dp(LU), _ld(LU), _ip(ip), _dp(v)))


def getrf_nopiv(A):
    LU = _fmat(np.array(A, dtype=np.float64, order="F", copy=True))
    info = np.zeros(1, dtype=np.int32)
    lib().orc_getrf_nopiv(LU.shape[1], _dp(LU), _ld(LU), _ip(info))
    return LU, int(info[0])


def getrs(trans: str, LU, ipiv, B):
    """Solve A X = B ('N') or A^T X = B ('T') with packed factors; returns X."""
    LU = _fmat(LU)
    X = np.array(B, dtype=np.float64, order="F", copy=True)
    vec = X.ndim == 1
    if vec:
        X = X.reshape(-1, 1, order="F")
    n, nrhs = X.shape
    ip = None if ipiv is None else np.ascontiguousarray(ipiv, dtype=np.int32)
    lib().orc_getrs(trans.encode()[:1], n, nrhs, _dp(LU), _ld(LU), _ip(ip), _dp(X), max(1, n))
    return X.reshape(-1) if vec else X


def residual_dense(A, x, b):
    """HPL scaled residual and its four norms from a stored matrix."""
    A = _fmat(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(5, dtype=np.float64)
    lib().orc_residual_dense(A.shape[1], _dp(A), _ld(A), _dp(x), _dp(b), _dp(out))
    return out


def residual_seeded(n: int, seed: int, x, dd: bool = False):
    """HPL scaled residual with A, b regenerated from the seed (no n x n copy)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(5, dtype=np.float64)
    lib().orc_residual_seeded(n, seed, 1 if dd else 0, _dp(x), None, _dp(out))
    return out


def factor_error(A0, LU, ipiv):
    """||PA - LU||_F / (||A||_F n eps)."""
    A0 = _fmat(A0)
    LU = _fmat(LU)
    ip = None if ipiv is None else np.ascontiguousarray(ipiv, dtype=np.int32)
    return float(lib().orc_factor_error(LU.shape[1], _dp(A0), _ld(A0), _dp(LU), _ld(LU), _ip(ip)))


def solve_adjoint(LU, ipiv, X, W):
    """Closed-form adjoint of X = A^-1 B under loss sum(W*X): (dA, dB)."""
    LU = _fmat(LU)
    X = _fmat(X)
    W = _fmat(W)
    n, k = X.shape
    dB = np.zeros((n, k), dtype=np.float64, order="F")
    dA = np.zeros((n, n), dtype=np.float64, order="F")
    ip = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib().orc_solve_adjoint(n, k, _dp(LU), _ld(LU), _ip(ip), _dp(X), _ld(X), _dp(W), _ld(W),
                            _dp(dB), _ld(dB), _dp(dA), _ld(dA))
    return dA, dB


# ------------------------------------------------------ mixed precision

BF16, E4M3 = 0, 1


def f32_to_bf16(x: float) -> int:
    return int(lib().orc_f32_to_bf16(x))


def bf16_to_f32(h: int) -> float:
    return float(lib().orc_bf16_to_f32(h))


def f32_to_e4m3(x: float) -> int:
    return int(lib().orc_f32_to_e4m3(x))


def e4m3_to_f32(c: int) -> float:
    return float(lib().orc_e4m3_to_f32(c))


def scale_exp(amax: float, qmax: float) -> int:
    return int(lib().orc_scale_exp(amax, qmax))


def qmax(prec: int) -> float:
    return float(lib().orc_qmax(prec))


def _f32(a):
    a = np.asarray(a, dtype=np.float32)
    return a if a.flags.f_contiguous else np.asfortranarray(a)


def tile_exps(X, by_rows: bool, prec: int):
    X = _f32(X)
    rows, cols = X.shape
    ext = rows if by_rows else cols
    ex = np.zeros(max(1, (ext + 127) // 128), dtype=np.int32)
    lib().orc_tile_exps(rows, cols, X.ctypes.data_as(C.POINTER(C.c_float)), max(1, rows), 1 if by_rows else 0,
                        prec, _ip(ex))
    return ex[: (ext + 127) // 128]


def quantize(X, by_rows: bool, prec: int, exps):
    X = _f32(X)
    rows, cols = X.shape
    out = np.zeros((rows, cols), dtype=np.uint16, order="F")
    ex = np.ascontiguousarray(exps, dtype=np.int32)
    lib().orc_quantize(rows, cols, X.ctypes.data_as(C.POINTER(C.c_float)), max(1, rows), 1 if by_rows else 0,
                       prec, _ip(ex), out.ctypes.data_as(C.POINTER(C.c_uint16)))
    return out


def mxp_getrf(A64, nb: int, prec: int, replay=None, plant=None):
    """Mixed-precision unpivoted LU (FP32 factors) of the FP64 matrix A64.

    replay: FP32 factors of another implementation whose panels' L21 and U12
    are quantized in step 3 instead of the oracle's own (see
    orc_mxp_getrf_ex).  plant: (panel, rel) multiplies that panel's L21 by
    (1 + rel) after its factorization (a planted error, for tests)."""
    A64 = _fmat(A64)
    n = A64.shape[0]
    W = np.zeros((n, n), dtype=np.float32, order="F")
    info = np.zeros(1, dtype=np.int32)
    fptr = C.POINTER(C.c_float)
    if replay is None and plant is None:
        lib().orc_mxp_getrf(n, nb, prec, _dp(A64), _ld(A64), W.ctypes.data_as(fptr), max(1, n), _ip(info))
        return W, int(info[0])
    R = None if replay is None else np.asfortranarray(replay, dtype=np.float32)
    if R is not None and R.shape != (n, n):
        raise ValueError("replay factors must be %d x %d" % (n, n))
    pp, pr = (-1, 0.0) if plant is None else (int(plant[0]), float(plant[1]))
    lib().orc_mxp_getrf_ex(n, nb, prec, _dp(A64), _ld(A64), W.ctypes.data_as(fptr), max(1, n), _ip(info),
                           None if R is None else R.ctypes.data_as(fptr), max(1, n), pp, pr)
    return W, int(info[0])


def mxp_getrs(LU32, x):
    LU32 = _f32(LU32)
    y = np.array(x, dtype=np.float64, copy=True)
    lib().orc_mxp_getrs(LU32.shape[0], LU32.ctypes.data_as(C.POINTER(C.c_float)), max(1, LU32.shape[0]), _dp(y))
    return y


def mxp_getrf_piv(A64, nb: int, prec: int):
    """Mixed-precision LU with partial pivoting (FP32 factors, 1-based pivots)
    of the FP64 matrix A64: (W, ipiv, info), see orc_mxp_getrf_piv."""
    A64 = _fmat(A64)
    n = A64.shape[0]
    W = np.zeros((n, n), dtype=np.float32, order="F")
    ipiv = np.zeros(n, dtype=np.int32)
    info = np.zeros(1, dtype=np.int32)
    lib().orc_mxp_getrf_piv(n, nb, prec, _dp(A64), _ld(A64), W.ctypes.data_as(C.POINTER(C.c_float)), max(1, n),
                            _ip(ipiv), _ip(info))
    return W, ipiv, int(info[0])


def mxp_getrs_piv(LU32, ipiv, x):
    """x <- U^-1 L^-1 P x with FP32 pivoted factors, arithmetic in FP64."""
    LU32 = _f32(LU32)
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    y = np.array(x, dtype=np.float64, copy=True)
    lib().orc_mxp_getrs_piv(LU32.shape[0], LU32.ctypes.data_as(C.POINTER(C.c_float)), max(1, LU32.shape[0]),
                            _ip(ipiv), _dp(y))
    return y


def gmres_ir(A, b, solve_m, m: int = 50, inner_tol: float = 1e-10, outer_max: int = 50):
    """Iterative refinement with GMRES as the correction solver (Carson and
    Higham 2018), in FP64, with the preconditioner applied by solve_m(v) ~ A^-1 v:
      x0 = M^-1 b;
      outer step: r = b - A x; stop once the HPL scaled residual of x is below
      16; else solve M^-1 A d = M^-1 r by one cycle of GMRES of at most m
      steps (Arnoldi with classical Gram-Schmidt applied twice, the small
      least-squares problem solved directly), stopping once the preconditioned
      residual has fallen by the factor inner_tol; x += d.
    Returns (x, outer steps taken, inner steps of each outer step)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    x = solve_m(b)
    inner = []
    for outer in range(outer_max + 1):
        if residual_dense(A, x, b)[0] < 16:
            return x, outer, inner
        if outer == outer_max:
            break
        z = solve_m(b - A @ x)
        beta = float(np.linalg.norm(z))
        if beta == 0.0:
            break
        V = np.zeros((len(b), m + 1))
        H = np.zeros((m + 1, m))
        V[:, 0] = z / beta
        for j in range(m):
            w = solve_m(A @ V[:, j])
            for _ in range(2):
                h = V[:, :j + 1].T @ w
                w = w - V[:, :j + 1] @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            rhs = np.zeros(j + 2)
            rhs[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], rhs, rcond=None)[0]
            rel = np.linalg.norm(H[:j + 2, :j + 1] @ y - rhs) / beta
            if rel <= inner_tol or H[j + 1, j] == 0.0:
                break
            V[:, j + 1] = w / H[j + 1, j]
        x = x + V[:, :j + 1] @ y
        inner.append(j + 1)
    return x, outer, inner


def ozaki_gemm(A, B, Cm, s: int, beta: int):
    """C - A B by the slice products of the emulated FP64 update (a new array).

    Raises ValueError where a level sum could exceed 2^24 (see orc_ozaki_gemm)."""
    A, B = _fmat(A), _fmat(B)
    out = np.array(Cm, dtype=np.float64, order="F", copy=True)
    m, k = A.shape
    n = B.shape[1]
    rc = lib().orc_ozaki_gemm(m, n, k, s, beta, _dp(A), _ld(A), _dp(B), _ld(B), _dp(out), _ld(out))
    if rc != 0:
        raise ValueError("slice parameters s=%d beta=%d leave exact FP32 accumulation at k=%d" % (s, beta, k))
    return out


def ozaki_split_rows(A, s: int, beta: int):
    """(exponents E (m,), slices Q (s, m, k)) of the rows of A."""
    A = _fmat(A)
    m, k = A.shape
    E = np.zeros(m, dtype=np.int32)
    Q = np.zeros((s, m, k), dtype=np.float64)
    lib().orc_ozaki_split_rows(m, k, _dp(A), _ld(A), s, beta, _ip(E), _dp(Q))
    return E, Q


def ozaki_split_cols(B, s: int, beta: int):
    """(exponents F (n,), slices Q (s, n, k)) of the columns of B."""
    B = _fmat(B)
    k, n = B.shape
    F = np.zeros(n, dtype=np.int32)
    Q = np.zeros((s, n, k), dtype=np.float64)
    lib().orc_ozaki_split_cols(k, n, _dp(B), _ld(B), s, beta, _ip(F), _dp(Q))
    return F, Q


def hpl_flops(n: int) -> float:
    """HPL operation count (2/3) N^3 + (3/2) N^2."""
    return (2.0 / 3.0) * n ** 3 + 1.5 * n ** 2
