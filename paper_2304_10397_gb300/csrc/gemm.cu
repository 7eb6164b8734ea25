// gemm.cu -- FP64 GEMM, C = alpha op(A) op(B) + beta C, for the trailing
// update of Sec. I (A22 -= L21 U12, "rank-NB update ... DGEMM").
//
// On GB300 FP64 runs on the DFMA pipe at 2 FMA/clk/SM (measured: 1.20
// TFLOP/s at 2.0 GHz); the FP64 mma.sync (DMMA) path measured slower (1.06
// TFLOP/s), so this kernel issues DFMA from a register tile.  The kernel is
// compute-bound by a wide margin (a 64x64 tile with K=384 does 16 flop per
// byte it stages), so the design goal is to keep every SM's DFMA pipe fed:
// 256 threads, a 4x4 register tile per thread, 16-deep K slices staged in
// shared memory and double-buffered through registers.
#include "common.cuh"

namespace hplgb {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;
constexpr int kGemmThreads = 256;

template <bool TA, bool TB>
__global__ void __launch_bounds__(kGemmThreads, 2)
dgemm_kernel(int64_t m, int64_t n, int64_t k, double alpha, const double* __restrict__ A, int64_t lda,
             const double* __restrict__ B, int64_t ldb, double beta, double* __restrict__ C,
             int64_t ldc, int64_t tiles_m) {
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int64_t tile = blockIdx.x;
  const int64_t m0 = (tile % tiles_m) * BM;
  const int64_t n0 = (tile / tiles_m) * BN;

  // Global -> register staging: 4 values of A and 4 of B per thread per slice.
  double ra[4], rb[4];
  auto load_slice = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!TA) {  // A(i, kk) at A[i + kk lda]: 64 consecutive rows per kk
        int i = t & 63, kk = (t >> 6) + 4 * q;
        int64_t gi = m0 + i, gk = k0 + kk;
        ra[q] = (gi < m && gk < k) ? A[gi + gk * lda] : 0.0;
      } else {    // op(A)(i, kk) = A[kk + i lda]: 16 consecutive kk per row
        int kk = t & 15, i = (t >> 4) + 16 * q;
        int64_t gi = m0 + i, gk = k0 + kk;
        ra[q] = (gi < m && gk < k) ? A[gk + gi * lda] : 0.0;
      }
      if (!TB) {  // op(B)(kk, j) = B[kk + j ldb]
        int kk = t & 15, j = (t >> 4) + 16 * q;
        int64_t gj = n0 + j, gk = k0 + kk;
        rb[q] = (gj < n && gk < k) ? B[gk + gj * ldb] : 0.0;
      } else {    // op(B)(kk, j) = B[j + kk ldb]
        int j = t & 63, kk = (t >> 6) + 4 * q;
        int64_t gj = n0 + j, gk = k0 + kk;
        rb[q] = (gj < n && gk < k) ? B[gj + gk * ldb] : 0.0;
      }
    }
  };
  auto store_slice = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!TA) As[buf][(t >> 6) + 4 * q][t & 63] = ra[q];
      else As[buf][t & 15][(t >> 4) + 16 * q] = ra[q];
      if (!TB) Bs[buf][t & 15][(t >> 4) + 16 * q] = rb[q];
      else Bs[buf][(t >> 6) + 4 * q][t & 63] = rb[q];
    }
  };

  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  const int64_t nslices = (k + BK - 1) / BK;
  load_slice(0);
  store_slice(0);
  __syncthreads();
  for (int64_t sl = 0; sl < nslices; ++sl) {
    const int buf = (int)(sl & 1);
    if (sl + 1 < nslices) load_slice((sl + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[buf][kk][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[buf][kk][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    if (sl + 1 < nslices) store_slice(buf ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int64_t gj = n0 + ty + 16 * c;
    if (gj >= n) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int64_t gi = m0 + tx + 16 * r;
      if (gi >= m) continue;
      double* p = C + gi + gj * ldc;
      *p = (beta == 0.0) ? alpha * acc[r][c] : fma(alpha, acc[r][c], beta * *p);
    }
  }
}

// Skinny C = alpha A B + beta C for n, k <= 32 (no transposes): the panel
// recursion's narrow Schur updates, where a 64 x 64 tile would compute mostly
// padding.  B lives in shared memory; a thread takes one row and kSkinnyCols
// columns.  Each entry is summed as in dgemm_kernel (FMAs over k in order
// from 0, then fma(alpha, acc, beta c)), so the results are the same.
constexpr int kSkinnyCols = 8;
__global__ void __launch_bounds__(256)
dgemm_skinny_kernel(int64_t m, int n, int k, double alpha, const double* __restrict__ A, int64_t lda,
                    const double* __restrict__ B, int64_t ldb, double beta, double* __restrict__ C, int64_t ldc) {
  __shared__ double Bs[32][32 + 1];
  for (int t = threadIdx.x; t < k * n; t += blockDim.x) {
    const int kk = t % k, j = t / k;
    Bs[kk][j] = B[kk + (int64_t)j * ldb];
  }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * kSkinnyCols;
  if (i >= m) return;
  double acc[kSkinnyCols];
#pragma unroll
  for (int c = 0; c < kSkinnyCols; ++c) acc[c] = 0.0;
#pragma unroll 4
  for (int kk = 0; kk < k; ++kk) {
    const double a = A[i + kk * lda];
#pragma unroll
    for (int c = 0; c < kSkinnyCols; ++c) acc[c] = fma(a, Bs[kk][min(j0 + c, 32)], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < kSkinnyCols; ++c) {
    const int j = j0 + c;
    if (j >= n) break;
    double* p = C + i + (int64_t)j * ldc;
    *p = (beta == 0.0) ? alpha * acc[c] : fma(alpha, acc[c], beta * *p);
  }
}

template <bool TA, bool TB>
int launch_t(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
             const double* B, int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t s) {
  int64_t tm = (m + BM - 1) / BM, tn = (n + BN - 1) / BN;
  int64_t tiles = tm * tn;
  if (tiles > 0x7fffffffLL) return set_error(HPL_ERR_NOTSUP, "dgemm: too many tiles");
  dgemm_kernel<TA, TB><<<(unsigned)tiles, kGemmThreads, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta,
                                                                 C, ldc, tm);
  count_launch();
  return check_launch("dgemm_kernel");
}

}  // namespace

int launch_dgemm(bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                 int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                 cudaStream_t s) {
  if (m <= 0 || n <= 0) return HPL_OK;
  if (k <= 0 && beta == 1.0) return HPL_OK;
  if (!ta && !tb && n <= 32 && k >= 1 && k <= 32) {
    if ((m + 255) / 256 > 0x7fffffffLL) return set_error(HPL_ERR_NOTSUP, "dgemm: too many rows");
    dim3 grid((unsigned)((m + 255) / 256), (unsigned)((n + kSkinnyCols - 1) / kSkinnyCols));
    dgemm_skinny_kernel<<<grid, 256, 0, s>>>(m, (int)n, (int)k, alpha, A, lda, B, ldb, beta, C, ldc);
    count_launch();
    return check_launch("dgemm_skinny_kernel");
  }
  if (!ta && !tb) return launch_t<false, false>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
  if (!ta && tb) return launch_t<false, true>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
  if (ta && !tb) return launch_t<true, false>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
  return launch_t<true, true>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
}

}  // namespace hplgb
