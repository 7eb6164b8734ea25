// getrs.cu -- the solves after the factorization (Sec. II: U x = L^-1 P^-1 b,
// then U^-1), and their transposes for the adjoint of the solve.
//
// Blocked substitution with row blocks of kBs: solve the kBs x kBs diagonal
// triangle (one CTA per right-hand side, column sweep through shared memory),
// then subtract the block's contribution from the remaining rows -- a GEMV
// (memory-bound, coalesced along the factor's columns) for few right-hand
// sides, the FP64 GEMM otherwise.  Interchanges are applied in blocks of up
// to 512 with the composed-permutation gather/scatter of laswp.cu.
#include "common.cuh"

namespace hplgb {

namespace {

constexpr int kBs = 128;  // diagonal block size

// op(T)(i,k) for the kBs x kBs diagonal block at D (ldd): trans ? T(k,i) : T(i,k).
// lower: forward sweep; else backward.  unit: no division.
template <bool LOWER, bool UNIT, bool TRANS>
__global__ void __launch_bounds__(kBs)
diag_solve_kernel(int nb, const double* __restrict__ D, int64_t ldd, double* __restrict__ B,
                  int64_t ldb) {
  __shared__ double xk;
  const int i = threadIdx.x;
  double* x = B + (int64_t)blockIdx.x * ldb;
  double xi = i < nb ? x[i] : 0.0;
  for (int s = 0; s < nb; ++s) {
    const int k = LOWER ? s : nb - 1 - s;
    if (i == k) {
      if (!UNIT) xi = xi / D[k + k * ldd];
      xk = xi;
    }
    __syncthreads();
    const bool below = LOWER ? (i > k) : (i < k);
    if (below && i < nb) {
      double t = TRANS ? D[k + (int64_t)i * ldd] : D[i + (int64_t)k * ldd];
      xi = fma(-t, xk, xi);
    }
    __syncthreads();
  }
  if (i < nb) x[i] = xi;
}

// y[0..rows) -= op(M) x for one right-hand side per blockIdx.y.
// !TRANS: op(M)(r,k) = M[r + k ldm] (thread per row, loop over k).
// TRANS:  op(M)(r,k) = M[k + r ldm] (warp per row, lanes over k).
template <bool TRANS>
__global__ void __launch_bounds__(256)
gemv_update_kernel(int64_t rows, int kcols, const double* __restrict__ M, int64_t ldm,
                   const double* __restrict__ xb, int64_t ldx, double* __restrict__ y, int64_t ldy) {
  __shared__ double xs[kBs];
  const double* xv = xb + blockIdx.y * ldx;
  double* yv = y + blockIdx.y * ldy;
  for (int k = threadIdx.x; k < kcols; k += blockDim.x) xs[k] = xv[k];
  __syncthreads();
  if (!TRANS) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
      double acc = 0.0;
      for (int k = 0; k < kcols; ++k) acc = fma(M[r + k * ldm], xs[k], acc);
      yv[r] -= acc;
    }
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
      double acc = 0.0;
      const double* col = M + r * ldm;
      for (int k = lane; k < kcols; k += 32) acc = fma(col[k], xs[k], acc);
#pragma unroll
      for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) yv[r] -= acc;
    }
  }
}

template <bool LOWER, bool UNIT, bool TRANS>
int diag_solve(int nb, const double* D, int64_t ldd, double* B, int64_t ldb, int64_t nrhs, cudaStream_t s) {
  diag_solve_kernel<LOWER, UNIT, TRANS><<<(unsigned)nrhs, kBs, 0, s>>>(nb, D, ldd, B, ldb);
  count_launch();
  return check_launch("diag_solve_kernel");
}

// y(rows x nrhs) -= op(M)(rows x kcols) xb(kcols x nrhs)
int block_update(bool trans, int64_t rows, int kcols, const double* M, int64_t ldm, const double* xb,
                 double* y, int64_t ldb, int64_t nrhs, cudaStream_t s) {
  if (rows <= 0) return HPL_OK;
  if (nrhs <= 4) {
    int64_t per_block = trans ? 8 : 256;
    int64_t bx = (rows + per_block - 1) / per_block;
    if (bx > 152 * 16) bx = 152 * 16;
    dim3 grid((unsigned)bx, (unsigned)nrhs);
    if (trans) gemv_update_kernel<true><<<grid, 256, 0, s>>>(rows, kcols, M, ldm, xb, ldb, y, ldb);
    else gemv_update_kernel<false><<<grid, 256, 0, s>>>(rows, kcols, M, ldm, xb, ldb, y, ldb);
    count_launch();
    return check_launch("gemv_update_kernel");
  }
  return launch_dgemm(trans, false, rows, nrhs, kcols, -1.0, M, ldm, xb, ldb, 1.0, y, ldb, s);
}

int apply_pivots(Workspace* ws, int64_t n, int64_t nrhs, const int32_t* ipiv, double* B, int64_t ldb,
                 bool reverse, cudaStream_t s) {
  const int64_t pb = 512;
  int32_t* perm = ws->perm + perm_ints_for(1024);  // second slot
  int64_t nblk = (n + pb - 1) / pb;
  for (int64_t q = 0; q < nblk; ++q) {
    int64_t b = reverse ? nblk - 1 - q : q;
    int64_t k1 = b * pb, k2 = k1 + pb < n ? k1 + pb : n;
    HPL_TRY(launch_laswp_compose(ipiv, k1, k2, 0, n, reverse, perm, ws->dev_err, s));
    HPL_TRY(launch_laswp_apply(perm, k2 - k1, nrhs, B, ldb, s));
  }
  return HPL_OK;
}

}  // namespace

int launch_getrs(Workspace* ws, char trans, int64_t n, int64_t nrhs, const double* LU, int64_t lda,
                 const int32_t* ipiv, double* B, int64_t ldb, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return HPL_OK;
  if (nrhs > 65535) return set_error(HPL_ERR_NOTSUP, "getrs: at most 65535 right-hand sides");
  if (ws->perm_ints < 2 * perm_ints_for(1024)) return set_error(HPL_ERR_NOTSUP, "getrs: perm buffer");
  const int64_t nblk = (n + kBs - 1) / kBs;
  if (trans == 'N' || trans == 'n') {
    if (ipiv) HPL_TRY(apply_pivots(ws, n, nrhs, ipiv, B, ldb, false, s));
    // L y = P b, unit lower, forward
    for (int64_t b = 0; b < nblk; ++b) {
      int64_t b0 = b * kBs, be = b0 + kBs < n ? b0 + kBs : n;
      int nb = (int)(be - b0);
      HPL_TRY((diag_solve<true, true, false>(nb, LU + b0 + b0 * lda, lda, B + b0, ldb, nrhs, s)));
      HPL_TRY(block_update(false, n - be, nb, LU + be + b0 * lda, lda, B + b0, B + be, ldb, nrhs, s));
    }
    // U x = y, backward
    for (int64_t b = nblk - 1; b >= 0; --b) {
      int64_t b0 = b * kBs, be = b0 + kBs < n ? b0 + kBs : n;
      int nb = (int)(be - b0);
      HPL_TRY((diag_solve<false, false, false>(nb, LU + b0 + b0 * lda, lda, B + b0, ldb, nrhs, s)));
      HPL_TRY(block_update(false, b0, nb, LU + b0 * lda, lda, B + b0, B, ldb, nrhs, s));
    }
  } else {
    // U^T y = g, forward (op = U^T is lower, non-unit)
    for (int64_t b = 0; b < nblk; ++b) {
      int64_t b0 = b * kBs, be = b0 + kBs < n ? b0 + kBs : n;
      int nb = (int)(be - b0);
      HPL_TRY((diag_solve<true, false, true>(nb, LU + b0 + b0 * lda, lda, B + b0, ldb, nrhs, s)));
      // rows r >= be: y_r -= sum_k U(k, r) y_k, k in block
      HPL_TRY(block_update(true, n - be, nb, LU + b0 + be * lda, lda, B + b0, B + be, ldb, nrhs, s));
    }
    // L^T z = y, backward, unit
    for (int64_t b = nblk - 1; b >= 0; --b) {
      int64_t b0 = b * kBs, be = b0 + kBs < n ? b0 + kBs : n;
      int nb = (int)(be - b0);
      HPL_TRY((diag_solve<false, true, true>(nb, LU + b0 + b0 * lda, lda, B + b0, ldb, nrhs, s)));
      // rows r < b0: z_r -= sum_k L(k, r) z_k, k in block
      HPL_TRY(block_update(true, b0, nb, LU + b0, lda, B + b0, B, ldb, nrhs, s));
    }
    if (ipiv) HPL_TRY(apply_pivots(ws, n, nrhs, ipiv, B, ldb, true, s));
  }
  return HPL_OK;
}

}  // namespace hplgb
