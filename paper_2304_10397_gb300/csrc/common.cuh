// common.cuh -- internal declarations shared by the CUDA sources of libhplgb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hplgb.h"

namespace hplgb {

// ------------------------------------------------------------------ errors
// Records a message for hpl_last_error() and returns the code.
int set_error(int code, const char* fmt, ...);
// Returns HPL_ERR_FAULT if HPLGB_FAULT names `site` (host-side fault injection).
int fault_point(const char* site);
// Counts kernel launches made by the library (the number is a public claim).
void count_launch(int n = 1);
// Checks cudaGetLastError() after a launch; returns HPL_OK or HPL_ERR_CUDA.
int check_launch(const char* what);
// Raises the dynamic shared-memory limit of kernel `fn` to `bytes` on the
// current device.  cudaFuncSetAttribute applies to the current device only, so
// the call is made once per (device, kernel) pair, under a lock.
int set_smem_attr(const void* fn, int bytes);
// Every device allocation of the library goes through these two, which keep
// a per-device count of the bytes held (hpl_workspace_bytes).  dev_free must
// be called with the allocating device current.
int dev_alloc(void** p, size_t bytes);
void dev_free(void* p, size_t bytes);

#define HPL_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::hplgb::set_error(HPL_ERR_CUDA, "%s: %s (%s:%d)", #call,              \
                                cudaGetErrorString(e_), __FILE__, __LINE__);        \
  } while (0)

#define HPL_TRY(expr)           \
  do {                          \
    int r_ = (expr);            \
    if (r_ != HPL_OK) return r_; \
  } while (0)

// Device error word values (written by kernels, read by hpl_sync_check).
enum DevErr : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BADPIV = 2 };

// ------------------------------------------------------ per-device context
struct Workspace {
  int device = -1;
  int num_sms = 0;
  int* dev_err = nullptr;                 // device error word
  unsigned long long* bar = nullptr;      // grid-barrier counter (panel kernel)
  unsigned long long bar_next = 0;        // host copy of the counter's next base
  double* panel_slots = nullptr;          // published pivot candidates
  size_t panel_slots_bytes = 0;
  int32_t* perm = nullptr;                // composed permutations (laswp)
  size_t perm_ints = 0;
  double* scratch = nullptr;              // residual partials etc.
  size_t scratch_bytes = 0;
  double* minv = nullptr;                 // I - L11^-1 of the emulated path's U12 solve
  size_t minv_bytes = 0;
  int* tile_ctr = nullptr;                // per-panel tile counters of the emulated look-ahead
  size_t tile_ctr_bytes = 0;
  cudaStream_t la_stream = nullptr;       // look-ahead stream (high priority)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev[8] = {};
  bool events_ready = false;
};
// Returns the context of the current device, creating it on first use.
// Growing a buffer synchronizes the device before the old one is freed, so
// buffers must be sized before the launches that use them are queued.
int get_workspace(Workspace** ws);
int ensure_perm(Workspace* ws, size_t ints);
int ensure_scratch(Workspace* ws, size_t bytes);

// ------------------------------------------------------- phase timers
// With HPLGB_TIMERS=1, entry points record CUDA events between phases on the
// caller's stream; hpl_phase_times() sums them per phase.
enum PhaseId { PH_TOTAL = 0, PH_PANEL = 1, PH_LASWP = 2, PH_TRSM = 3, PH_GEMM = 4, PH_QUANT = 5,
               PH_MATVEC = 6, PH_PRECOND = 7, PH_ORTH = 8, kNumPhases = 9 };
void phase_timing_begin(cudaStream_t s);
// Trailing-update event timing (hpl_set_gemm_timing): brackets one launch.
int gemm_timing_begin(cudaStream_t s);
int gemm_timing_end(cudaStream_t s, double flops, double bytes);
void phase_mark(int phase_of_previous);
bool phase_timing_on();

// ------------------------------------------------------------- launchers
// All launchers are asynchronous on `s` and return HPL_OK or an error code.
int launch_generate(int64_t n, uint64_t seed, double* A, int64_t lda, double* b, cudaStream_t s);
int launch_dd_diag(int64_t n, double* A, int64_t lda, cudaStream_t s);
int launch_residual(Workspace* ws, int64_t n, uint64_t seed, int dd, const double* A, int64_t lda,
                    const double* x, const double* b, double* out5_host, cudaStream_t s);

// C = alpha op(A) op(B) + beta C
int launch_dgemm(bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                 int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                 cudaStream_t s);

// Composed permutation of the interchanges k = k1..k2-1: row k <-> row
// ipiv[k] - 1 - val_shift (rows local to the matrix the permutation is applied
// to), written to perm (layout documented in laswp.cu).  reverse = apply in
// decreasing k (for the transposed solve).  nrows bounds the rows; an
// out-of-range pivot moves nothing and sets DEV_BADPIV in dev_err.
int launch_laswp_compose(const int32_t* ipiv, int64_t k1, int64_t k2, int64_t val_shift,
                         int64_t nrows, bool reverse, int32_t* perm, int* dev_err, cudaStream_t s);
int launch_laswp_apply(const int32_t* perm, int64_t jb, int64_t ncols, double* A, int64_t lda,
                       cudaStream_t s);
// The same interchanges composed and applied to ncols columns of A in one
// launch (each CTA composes them itself; for few columns).
int launch_laswp_fused(const int32_t* ipiv, int64_t k1, int64_t k2, int64_t val_shift, int64_t nrows,
                       bool reverse, int64_t ncols, double* A, int64_t lda, int* dev_err, cudaStream_t s);
inline size_t perm_ints_for(int64_t jb) { return (size_t)(4 * jb + 4); }

// A (n x n, lda) <- I; and A <- I - A restricted to the strictly lower part
// (the diagonal and upper part set to zero), for a unit-lower A.
int launch_identity_f64(int64_t n, double* A, int64_t lda, cudaStream_t s);
int launch_i_minus_lower(int64_t n, double* A, int64_t lda, cudaStream_t s);
// B <- L^-1 B, L unit lower m x m; the strip solve alone (m <= 1024).
int launch_trsm_llnu_strip(int64_t m, int64_t n, const double* L, int64_t ldl, double* B, int64_t ldb,
                           cudaStream_t s);
// B <- L^-1 B, L unit lower m x m.
int launch_trsm_llnu(int64_t m, int64_t n, const double* L, int64_t ldl, double* B, int64_t ldb,
                     cudaStream_t s);

size_t panel_slots_bytes_for(int num_sms);
// Panel FACT (recursive) of the m x w block at A, interchanges within the
// block's columns, ipiv gets (row index relative to A's first row) + 1 + ipiv_shift.
// slices >= 0: the recursion's wide Schur updates use the emulated FP64 product.
// max_ctas > 0: the base kernel and the emulated products on at most max_ctas
// CTAs each.
int panel_factor(Workspace* ws, int64_t m, int64_t w, double* A, int64_t lda, int32_t* ipiv,
                 int64_t ipiv_shift, int32_t* info, int64_t info_shift, cudaStream_t s, int slices = -1,
                 int max_ctas = 0);

// Triangular solves for getrs.
int launch_getrs(Workspace* ws, char trans, int64_t n, int64_t nrhs, const double* LU, int64_t lda,
                 const int32_t* ipiv, double* B, int64_t ldb, cudaStream_t s);

// Frees the mixed-precision buffers of every device (hpl_finalize).
void mxp_finalize();

// A second launch of one emulated update on another stream: once `js`
// reaches this point (after the work queued on it before), js_ctas more CTAs
// of the fused kernel join the ones on the caller's stream, and both take
// their tiles from the zeroed counter *ctr.  `ev` (no timing) orders the
// splits before the joining launch.
struct OzakiJoin {
  cudaStream_t js;
  cudaEvent_t ev;
  int js_ctas;
  int* ctr;
};
// C <- C - A B in FP64 accuracy from BF16 slice products on the tensor cores
// (ozaki.cu); slices = 0 picks the slice count for k.
// max_ctas > 0 caps the fused kernel's persistent grid (leaving SMs to
// kernels that run beside it).  join (may be null) adds the second launch;
// it applies to the fused path with k <= 1024 (one pass), and is ignored
// otherwise.
int launch_ozaki_gemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                      double* C, int64_t ldc, int slices, int* err, cudaStream_t s, int max_ctas = 0,
                      const OzakiJoin* join = nullptr);
bool ozaki_params(int64_t k, int slices, int* s_out, int* beta_out);
void ozaki_finalize();
// Per-CTA shared memory (static + dynamic), registers per thread and threads
// of the fused emulated kernel, and of the first base-kernel launch of a FACT
// of m rows (w columns; ctas = its grid): whether the two fit on one SM.
int ozaki_fused_footprint(int* smem, int* regs, int* threads);
int panel_base_max_width();
int panel_base_footprint(int num_sms, int64_t m, int w, int64_t* ctas, int* smem, int* regs, int* threads);

int launch_fp64_peak(int64_t iters, double* gflops, cudaStream_t s);
int launch_fp64_dmma_peak(int64_t iters, double* gflops, cudaStream_t s);
int launch_fp64_mixed_peak(int64_t iters, int dfma_tiles, int split_warps, double* gflops, cudaStream_t s);

}  // namespace hplgb
