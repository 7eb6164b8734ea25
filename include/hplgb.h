/*
 * hplgb.h -- C ABI of the GB300 (sm_103a) High-Performance Linpack hot path.
 *
 * The method is the one of "Optimizing High-Performance Linpack for Exascale
 * Accelerated Architectures" (rocHPL): a random dense FP64 system A x = b
 * (Sec. II) is solved by right-looking blocked LU with partial pivoting, each
 * step being FACT (panel factorization), RS (row swapping) and UPDATE (DTRSM
 * of the U block row and the rank-NB DGEMM Schur update) (Sec. I, Fig. 2),
 * with a look-ahead that factors the next panel while the rest of the update
 * runs (Sec. III), then the triangular solves (Sec. II).
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major FP64 (element (i,j) at ptr[i + j*ld]) and
 *     ld >= max(1, rows).  Pivot vectors are int32, 1-based global row indices
 *     (LAPACK convention).
 *   - Every pointer argument is a DEVICE pointer owned by the caller, unless
 *     its comment says "host".  The library never frees caller memory.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *     is the legacy default stream) unless stated otherwise.  Internal streams
 *     fork from and join back to `stream` through events; nothing synchronizes
 *     the host except where stated.
 *   - The library allocates internal workspace on first use (cached per device
 *     and grown on demand) and releases it in hpl_finalize().
 *   - Return value: HPL_OK (0), or -i when argument i (1-based) is illegal, or
 *     one of the HPL_ERR_* codes below.  hpl_last_error() gives a message.
 *   - Concurrent calls that share the library's workspace (two getrf calls in
 *     flight on different streams of the same device) are not supported: the
 *     caller orders them on one stream or synchronizes between them.
 */
#ifndef HPLGB_H_
#define HPLGB_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HPL_OK 0
#define HPL_ERR_CUDA (-100)     /* a CUDA runtime call or launch failed          */
#define HPL_ERR_ALLOC (-101)    /* workspace allocation failed                   */
#define HPL_ERR_FAULT (-102)    /* host-side fault injection (HPLGB_FAULT=name)  */
#define HPL_ERR_TIMEOUT (-103)  /* a bounded device-side wait gave up            */
#define HPL_ERR_NOTSUP (-104)   /* feature not supported on this device          */

/* Fill A (n x n, lda) and b (n) with the random system of Sec. II: element
 * t = i + j*n of A and t = n*n + i of b take the (t+1)-th state s of the 64-bit
 * LCG s' = 6364136223846793005 s + 1442695040888963407 (mod 2^64), s_0 = seed,
 * mapped to (s >> 11) * 2^-53 - 0.5, i.e. uniform in [-0.5, 0.5).  (The paper
 * does not name HPL's generator; this LCG is this library's choice.)
 * dd != 0 makes A diagonally dominant for the mixed-precision solve:
 * A(i,i) = sum over j != i of |A(i,j)|, summed in ascending j in FP64.
 * b may be NULL.  Bit-identical to a sequential host implementation. */
int hpl_generate(int64_t n, uint64_t seed, int dd, double* A, int64_t lda, double* b,
                 void* stream);

/* LU factorization with partial pivoting, A = P L U (Sec. II), by the
 * right-looking blocked algorithm of Sec. I: for each panel of nb columns,
 * FACT (recursive panel LU on the GPU; per-column pivot = largest magnitude,
 * ties to the smallest row), RS (the panel's interchanges applied to the
 * columns left and right of it), UPDATE (U12 = L11^-1 A12, then
 * A22 -= L21 U12), with a depth-1 look-ahead (Sec. III: the next panel is
 * updated and factored on a second stream while the rest of the update runs).
 *   n >= 0; nb >= 1 (clamped to n); lda >= max(1,n).
 *   A (in/out): overwritten by the unit-lower L (strictly below the diagonal)
 *     and U (on and above it).
 *   ipiv (out, n int32): row i was interchanged with row ipiv[i]-1 (1-based).
 *   info (out, device int32, may be NULL): 0, or k > 0 if U(k-1,k-1) is
 *     exactly zero (first such k); the factorization is completed anyway.
 *   lookahead: 0 = single stream, 1 = depth-1 look-ahead on two streams.
 * n = 0 returns HPL_OK and does nothing.  Not checked: non-finite entries
 * (they propagate, as in LAPACK).  A bounded device wait that expires (it
 * can only happen if the GPU cannot co-schedule the panel kernel's blocks)
 * is reported by hpl_sync_check(). */
int hpl_getrf(int64_t n, int64_t nb, double* A, int64_t lda, int32_t* ipiv, int32_t* info,
              int lookahead, void* stream);

/* Solve with the factors of hpl_getrf (Sec. II: U x = L^-1 P^-1 b, then U^-1).
 *   trans 'N': B <- A^-1 B (interchanges, unit-lower L, then U).
 *   trans 'T': B <- A^-T B (U^T, unit-lower L^T, then the interchanges in
 *              reverse order) -- the adjoint solve of the differentiable solve.
 *   LU (n x n, lda), ipiv (n, 1-based; NULL = no interchanges, for factors of
 *   hpl_mxp-style unpivoted LU), B (in/out, n x nrhs, ldb >= max(1,n)). */
int hpl_getrs(char trans, int64_t n, int64_t nrhs, const double* LU, int64_t lda,
              const int32_t* ipiv, double* B, int64_t ldb, void* stream);

/* HPL scaled residual (the paper states none; this is the standard HPL
 * acceptance test):
 *   out5 (HOST, 5 doubles) = { ||Ax-b||_inf / (eps (||A||_inf ||x||_inf +
 *   ||b||_inf) n), ||Ax-b||_inf, ||A||_inf, ||x||_inf, ||b||_inf }, eps = 2^-53.
 * A is regenerated from `seed` (and `dd`, as in hpl_generate) when A == NULL,
 * otherwise read from A (n x n, lda).  b may be NULL, in which case b is
 * regenerated from the seed too.  r = Ax - b is accumulated with error-free
 * transformations (Dot2, Ogita-Rump-Oishi 2005) so that it is accurate even
 * though it is of the order of rounding errors.  Synchronizes `stream`
 * (the 5 doubles are copied to the host); NaN entries propagate to out5. */
int hpl_residual(int64_t n, uint64_t seed, int dd, const double* A, int64_t lda,
                 const double* x, const double* b, double* out5, void* stream);

/* The trailing update of Sec. I, C <- C - A B (C m x n, ldc; A m x k, lda;
 * B k x n, ldb; all FP64 column-major), in FP64 accuracy from BF16 tensor-core
 * products: not the paper's method (rocHPL runs an FP64 DGEMM), an emulation
 * after Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012).  Every row
 * of A and column of B is split exactly into `slices` integer slices of beta
 * bits under one power-of-two exponent per row (column); the s (s + 1) / 2
 * slice products whose levels i + j <= s + 1 are computed exactly (integer
 * sums below 2^24 in FP32 accumulators) and summed, the lowest levels exactly
 * in 64-bit integers and the top ones in FP64.  slices = 0 chooses 8 slices of
 * 7 bits for k <= 409 and 9 of 6 bits up to k = 1489 (k is taken in passes of
 * at most 1024); slices > 0 takes the widest beta <= 8 with exact level sums
 * and slices * beta <= 60.  The error is of the order of an FP64 DGEMM's
 * rounding error for slices * beta >= 54.  Results are bitwise those of the
 * library's CPU oracle of the scheme.  Workspace: the slices (2 s k bytes per
 * row of A and column of B).
 * Errors: -1..-3 negative size, -4/-6/-8 NULL operand, -5/-7/-9 leading
 * dimension, -10 slices < 0 or no exact slice width for that many slices. */
int hpl_dgemm_emulated(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                       const double* B, int64_t ldb, double* C, int64_t ldc, int slices,
                       void* stream);

/* hpl_getrf with every trailing-update DGEMM (A22 -= L21 U12) replaced by
 * hpl_dgemm_emulated with the given slices; the U12 solve done as
 * U12 <- U12 - M U12 with M = I - L11^-1 (L11^-1 by FP64 substitution once
 * per panel) by the same emulated product; and the panel recursion's Schur
 * updates at least 32 wide emulated too.  The pivot search, the base
 * elimination, the interchanges and the small solves stay FP64.  Arguments
 * and results as hpl_getrf; -8 for an unusable `slices`. */
int hpl_getrf_emulated(int64_t n, int64_t nb, double* A, int64_t lda, int32_t* ipiv,
                       int32_t* info, int lookahead, int slices, void* stream);

/* General FP64 product C = alpha op(A) op(B) + beta C (op = identity or
 * transpose, ta/tb in {'N','T'}), C m x n.  The trailing update of Sec. I
 * (DGEMM, A22 -= L21 U12) is this with alpha = -1, beta = 1; beta = 0 does
 * not read C.  Errors: -1 / -2 ta / tb not 'N' or 'T', -3..-5 negative size,
 * -7 / -9 A / B NULL (when m, n, k > 0), -8 / -10 / -13 leading dimension
 * too small, -12 C NULL (when m, n > 0). */
int hpl_dgemm(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha,
              const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
              double* C, int64_t ldc, void* stream);

/* Rank-k outer product C = alpha U V^T (U m x k, V n x k, C m x n, C is not
 * read): the gradient dA = -lambda x^T of the differentiable solve (not in
 * the paper; it is the adjoint of X = A^-1 B under a loss sum(W .* X)).
 * Errors: -1..-3 negative size, -5 / -7 U / V NULL (when m, n, k > 0),
 * -6 / -8 / -10 leading dimension too small, -9 C NULL (when m, n > 0). */
int hpl_outer_update(int64_t m, int64_t n, int64_t k, double alpha, const double* U,
                     int64_t ldu, const double* V, int64_t ldv, double* C, int64_t ldc,
                     void* stream);

/* Apply the interchanges ipiv[k1..k2) (0-based positions, 1-based values, in
 * increasing order) to the rows of the n-column matrix A (lda): the RS phase
 * of Sec. I, done as one gather/scatter per column of the composed
 * permutation.  Errors: -1 ncols < 0, -2 A NULL, -6 ipiv NULL (both when
 * ncols > 0 and k2 > k1), -3 lda < k2, -4 k1 < 0 or k2 < k1; an interchange
 * row outside [1, lda] is reported by hpl_sync_check (-100) and moves nothing. */
int hpl_laswp(int64_t ncols, double* A, int64_t lda, int64_t k1, int64_t k2,
              const int32_t* ipiv, void* stream);

/* B <- L^-1 B with L the unit-lower m x m triangle of A (lda), B m x n (ldb):
 * the DTRSM of the UPDATE phase (Sec. I, U12 = L11^-1 A12).  Errors: -1 / -2
 * negative size, -3 / -5 A / B NULL (when m, n > 0), -4 / -6 leading
 * dimension too small. */
int hpl_trsm_llnu(int64_t m, int64_t n, const double* A, int64_t lda, double* B,
                  int64_t ldb, void* stream);

/* Factor only the m x w panel A (lda) with partial pivoting (FACT of Sec. I;
 * recursive, two subdivisions, right-looking base of width <= 16, Sec. III-A).
 * Interchanges are applied to the panel's own columns only; ipiv (w entries)
 * gets 1-based row indices relative to the panel's first row; info (device,
 * may be NULL) as in hpl_getrf.  Errors: -1 m < 0, -2 w < 0, w > m or
 * w > 1024, -3 / -5 A / ipiv NULL (when m, w > 0), -4 lda < max(1, m). */
int hpl_panel_getrf(int64_t m, int64_t w, double* A, int64_t lda, int32_t* ipiv,
                    int32_t* info, void* stream);

/* The panel factorization of hpl_panel_getrf without any device allocation:
 * for callers that cannot allocate device memory when they call the library
 * (a process whose memory is all handed to its own pool at start-up, a loop
 * that must never enter the driver's allocator).  The paper has no
 * counterpart; this is a deployment variant of FACT.  Its scratch (64 KiB:
 * pivot candidates, barrier counter, error word, one composed permutation)
 * is a static device array of the library that every GPU loading the library
 * holds until exit; the first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current, so make the first
 * call outside any stream capture.  Limits: w <= 1024 (larger w returns -2).
 * info is REQUIRED (device int32): 0, k > 0 for a zero pivot as in
 * hpl_getrf, -1 if a bounded device wait expired, or -2 if an interchange
 * named a row outside the panel (the panel was changed under the call).
 * Uses the same launch shape as hpl_panel_getrf (HPLGB_PANEL_ROWS,
 * HPLGB_PANEL_CTAS), and its first call on a device also checks that the
 * base kernel's CTAs can all be resident (HPL_ERR_NOTSUP otherwise).  Every call reuses the
 * same array and clears its counter and error word on `stream` first; calls
 * whose work overlaps on the GPU race on the array, so order them (one stream,
 * or synchronize).  Arguments and results as hpl_panel_getrf. */
int hpl_panel_getrf_noalloc(int64_t m, int64_t w, double* A, int64_t lda, int32_t* ipiv,
                            int32_t* info, void* stream);

/* ---------------------------------------------------------------------------
 * Mixed-precision variant (not in the paper, which only names HPL-MxP in
 * Sec. I): LU without interchanges of a diagonally dominant system (see
 * hpl_generate, dd = 1) whose trailing update runs on the tensor cores with
 * BF16 (prec 0) or FP8-E4M3 (prec 1) operands scaled per tile by powers of two,
 * FP32 accumulation and FP32 factors; FP64 accuracy is won back by GMRES
 * iterative refinement.
 * ------------------------------------------------------------------------- */

/* LU32 (n x n FP32, ldl) <- unpivoted LU of A64 (n x n FP64, lda; not
 * modified), panels of nb columns (32 <= nb <= 2048, nb % 32 == 0).  Per
 * panel: FP32 panel LU, U12 = L11^-1 A12 in FP32, tile exponents
 * e = max{e : amax 2^e <= qmax} (qmax = 1 for BF16, 448 for E4M3) for 128-row
 * tiles of L21 and 128-column tiles of U12, codes of L21 2^eL and U12 2^eU
 * (round to nearest even, E4M3 saturating), and
 * A22 -= 2^-(eL+eU) qL qU^T accumulated in FP32 on tcgen05.  info (device,
 * may be NULL): first exactly zero pivot (1-based) or 0.  With nb % 128 == 0
 * the next panel's diagonal-block LU runs on the library's look-ahead stream
 * beside the rest of each update (Sec. III, Fig. 3), joined back into
 * `stream` before the call returns; the factors are bitwise those without it
 * (HPLGB_MXP_LOOKAHEAD=0 turns it off, and so does HPLGB_TIMERS=1). */
int hpl_mxp_getrf(int64_t n, int64_t nb, int prec, const double* A64, int64_t lda, float* LU32,
                  int64_t ldl, int32_t* info, void* stream);

/* x (FP64, n) <- U^-1 L^-1 x with the FP32 factors of hpl_mxp_getrf (the
 * preconditioner of the refinement): computed in FP32 on x / max|x|, then
 * rescaled; max|x| is reduced on the device, so the call is asynchronous on
 * `stream` (a call that has to grow the library's workspace, the first one
 * for a larger n, synchronizes the device before it frees the old buffers).
 * Each call inverts the 128 x 128 diagonal blocks of L and U again, so the
 * factors may change between calls. */
int hpl_mxp_getrs(int64_t n, const float* LU32, int64_t ldl, double* x, void* stream);

/* GMRES-IR (Carson and Higham 2018): x (out, FP64) solves A x = b (A FP64,
 * lda) starting from x0 = M^-1 b with M = L U from hpl_mxp_getrf; each outer
 * step computes r = b - A x in FP64 (FMA within 1024-column chunks, the chunks
 * combined with TwoSum), solves A d = r by left-preconditioned restarted
 * GMRES(restart) in FP64 (classical Gram-Schmidt applied twice) to a relative
 * preconditioned residual inner_tol, and sets x += d, until the HPL scaled
 * residual of x is below `target` or max_outer steps.  stats (HOST, 6
 * doubles): {outer steps, total inner steps, scaled residual, ||b - Ax||_inf,
 * ||A||_inf, ||x||_inf}.  Synchronizes `stream`.  Errors: -1 n <= 0, -2 a
 * NULL pointer, -3 lda or ldl < n, -8 restart outside [1, 120], -9
 * max_outer < 1. */
int hpl_gmres_ir(int64_t n, const double* A, int64_t lda, const float* LU32, int64_t ldl,
                 const double* b, double* x, int restart, int max_outer, double inner_tol,
                 double target, double* stats, void* stream);

/* Step 3 of hpl_mxp_getrf alone: exponents eL (ceil(m2/128) ints) and eU
 * (ceil(m2/128)) of L21 (m2 x jb) and U12 (jb x m2) (both FP32 in one
 * column-major array with leading dimension ld), and the codes qL[i*kp + k] =
 * code(L21(i,k) 2^eL[i/128]), qU[j*kp + k] = code(U12(k,j) 2^eU[j/128])
 * (zero for jb <= k < kp; kp >= jb and kp * element size a multiple of 128). */
int hpl_mxp_quantize(int prec, int64_t m2, int64_t jb, const float* L21, const float* U12,
                     int64_t ld, int64_t kp, int* eL, int* eU, void* qL, void* qU, void* stream);

/* Step 2 of hpl_mxp_getrf alone: B <- L^-1 B in FP32 with L the unit-lower
 * m x m triangle of L (ldl), m <= 2048, and B m x n (ldb), both FP32
 * column-major (the U12 = L11^-1 A12 of the UPDATE phase, Sec. I, for the
 * mixed-precision factors).  L^-1 is formed by substitution and applied as a
 * tensor-core product of three BF16 pieces per FP32 operand with FP32
 * accumulation, accurate to a small multiple of the FP32 unit roundoff times
 * |L^-1| |B|.  Errors: -1 m out of range, -2 n < 0, -3 / -5 L / B NULL
 * (when m, n > 0), -4 / -6 leading dimension too small; -101 if its
 * workspace cannot be allocated. */
int hpl_strsm_llnu(int64_t m, int64_t n, const float* L, int64_t ldl, float* B, int64_t ldb,
                   void* stream);

/* Step 4 of hpl_mxp_getrf alone, on tcgen05:
 * C (m x n FP32, ldc) -= 2^-(eL[i/128] + eU[j/128]) sum_k qL[i*kp+k] qU[j*kp+k].
 * Errors: -1 prec not 0 or 1, -2 negative size, -5..-9 qL, qU, eL, eU or C
 * NULL (when m, n, kp > 0), -10 ldc < max(1, m). */
int hpl_mxp_gemm(int prec, int64_t m, int64_t n, int64_t kp, const void* qL, const void* qU,
                 const int* eL, const int* eU, float* C, int64_t ldc, void* stream);

/* Per-phase device times (ms) of the last timed call (hpl_getrf,
 * hpl_mxp_getrf, hpl_mxp_getrs or hpl_gmres_ir) made while the environment
 * variable HPLGB_TIMERS=1 was set, recorded with CUDA events on the caller's
 * stream: out[0..8] = {total, panel (FACT), laswp (RS), trsm, gemm, quantize,
 * matvec, preconditioner solve, orthogonalization and vector work}.
 * hpl_getrf with timers runs without look-ahead so the phases do not overlap.
 * Synchronizes with the last recorded event.  Returns the number written. */
int hpl_phase_times(double* out_host, int64_t cap);

/* Trailing-update timing: while enabled (on != 0), hpl_getrf brackets each of
 * its trailing-update DGEMM launches, and hpl_mxp_getrf each of its tcgen05
 * trailing updates, with two CUDA events on the stream the launch is made on.
 * hpl_set_gemm_timing also resets the record.  hpl_gemm_timing writes
 * {launches, total device ms, total algorithmic flops (2 m n k per launch),
 * total algorithmic bytes (DGEMM: 8 (m k + k n + 2 m n); tcgen05 update: the
 * FP32 C read and written, 8 m n, plus both code blocks once)} to out4 (HOST)
 * and synchronizes with the events. */
int hpl_set_gemm_timing(int on);
int hpl_gemm_timing(double* out4_host);

/* Synchronize `stream` and report a device-side error recorded by the
 * library's kernels since the last check (HPL_ERR_TIMEOUT if a bounded
 * grid-wide wait expired), then clear it. */
int hpl_sync_check(void* stream);

/* Measured FP64 FMA throughput: every thread of one full wave of 256-thread
 * CTAs (as many per SM as fit) updates a 4x4 register tile
 * acc[i][j] += a[i] b[j] (the inner step of the trailing-update DGEMM)
 * `iters` times; returns GFLOP/s in *gflops (host), best of 5 timed launches
 * after 4 warm-up launches.  Synchronizes. */
int hpl_fp64_peak(int64_t iters, double* gflops_host, void* stream);

/* The same measurement for the FP64 tensor path sm_103a exposes to PTX
 * (mma.sync.aligned.m8n8k4.f64, four independent chains per warp): GFLOP/s
 * in *gflops (host).  Synchronizes. */
int hpl_fp64_dmma_peak(int64_t iters, double* gflops_host, void* stream);

/* Both FP64 paths at once, to test whether they share one pipe: with
 * split_warps == 0 every warp does one DMMA step and dfma_tiles DFMA tile
 * steps per iteration; with split_warps != 0 even warps run the DFMA loop
 * (dfma_tiles steps per iteration) and odd warps the DMMA loop.  *gflops
 * (host) is the total FP64 flop rate of both.  dfma_tiles in [0, 64].
 * Synchronizes. */
int hpl_fp64_mixed_peak(int64_t iters, int dfma_tiles, int split_warps, double* gflops_host,
                        void* stream);

/* Bytes of device memory the library currently holds on the current device
 * as its own workspace (everything it obtained from cudaMalloc and has not
 * freed; the static array of hpl_panel_getrf_noalloc is not counted, since
 * it is part of the loaded module).  -1 if there is no current device. */
int64_t hpl_workspace_bytes(void);

/* Number of CUDA kernels this library has launched in this process. */
int64_t hpl_kernel_launches(void);

const char* hpl_last_error(void);
void hpl_finalize(void);

#ifdef __cplusplus
}
#endif

#endif /* HPLGB_H_ */
