// trsm.cu -- the DTRSM of the UPDATE phase (Sec. I): U12 <- L11^-1 A12 with
// L11 the unit-lower diagonal block of the factored panel.
//
// Blocked by column strips: each CTA owns a strip of SW columns of B, keeps it
// in registers (rows distributed over the CTA's threads, R rows per thread),
// and runs forward substitution down the rows.  At step k the owner of row k
// publishes its SW values through shared memory (double-buffered, one barrier
// per step) and every thread with a row i > k subtracts L(i,k) * x_k, with
// L(i,k) prefetched one step ahead (coalesced loads along the column of L).
#include "common.cuh"

namespace hplgb {

namespace {

constexpr int kTrsmThreads = 256;

template <typename T, int R, int SW>
__global__ void __launch_bounds__(kTrsmThreads)
trsm_llnu_kernel(int m, int64_t n, const T* __restrict__ L, int64_t ldl, T* __restrict__ B,
                 int64_t ldb) {
  __shared__ T xs[2][SW];
  const int t = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * SW;
  const int ncols = (int)((n - c0) < SW ? (n - c0) : SW);
  T x[R][SW];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int i = t + r * kTrsmThreads;
#pragma unroll
    for (int c = 0; c < SW; ++c)
      x[r][c] = (i < m && c < ncols) ? B[i + (c0 + c) * ldb] : T(0);
  }
  T lnext[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int i = t + r * kTrsmThreads;
    lnext[r] = (i < m) ? L[i] : T(0);  // column 0
  }
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int kbeg = rr * kTrsmThreads;
    const int kend = min(m, kbeg + kTrsmThreads);
    for (int k = kbeg; k < kend; ++k) {
      const int buf = k & 1;
      if (t == k - kbeg) {
#pragma unroll
        for (int c = 0; c < SW; ++c) xs[buf][c] = x[rr][c];
      }
      T lcur[R];
#pragma unroll
      for (int r = 0; r < R; ++r) lcur[r] = lnext[r];
      if (k + 1 < m) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          int i = t + r * kTrsmThreads;
          lnext[r] = (i < m) ? L[i + (int64_t)(k + 1) * ldl] : T(0);
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int i = t + r * kTrsmThreads;
        if (r >= rr && i > k && i < m) {
          T l = lcur[r];
#pragma unroll
          for (int c = 0; c < SW; ++c) x[r][c] = fma(-l, xs[buf][c], x[r][c]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int i = t + r * kTrsmThreads;
    if (i < m)
#pragma unroll
      for (int c = 0; c < SW; ++c)
        if (c < ncols) B[i + (c0 + c) * ldb] = x[r][c];
  }
}

// m <= 32 R (the panel recursion's triangles, and the 128-row blocks of the
// blocked solve on few columns): a warp per column, lane l holding x_i for
// rows i = l + 32 r; at step k the owner of x_k passes it to the others by a
// shuffle and every row i > k subtracts L(i,k) x_k, L staged once in shared
// memory.  The same FMAs in the same order as the strip kernel, without its
// CTA barrier per step (and without its wait on the next column of L).
template <int R>
__global__ void __launch_bounds__(256)
trsm_llnu_warp_kernel(int m, int64_t n, const double* __restrict__ L, int64_t ldl, double* __restrict__ B,
                      int64_t ldb) {
  extern __shared__ double Ls[];  // Ls[i * (m + 1) + k] = L(i, k)
  const int lp = m + 1;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t % m, k = t / m;
    Ls[i * lp + k] = L[i + (int64_t)k * ldl];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t c = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= n) return;
  double* col = B + c * ldb;
  double x[R];
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = lane + 32 * r < m ? col[lane + 32 * r] : 0.0;
  for (int k = 0; k < m; ++k) {
    const int kr = k >> 5;
    double own = x[0];
#pragma unroll
    for (int r = 1; r < R; ++r)
      if (kr == r) own = x[r];
    const double xk = __shfl_sync(0xffffffffu, own, k & 31);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      if (i > k && i < m) x[r] = fma(-Ls[i * lp + k], xk, x[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (lane + 32 * r < m) col[lane + 32 * r] = x[r];
}

template <int R>
int launch_trsm_warp(int64_t m, int64_t n, const double* L, int64_t ldl, double* B, int64_t ldb, cudaStream_t s) {
  const int64_t blocks = (n + 7) / 8;
  if (blocks > 0x7fffffff) return set_error(HPL_ERR_NOTSUP, "trsm: too many columns");
  const size_t smem = (size_t)m * (m + 1) * sizeof(double);
  HPL_TRY(set_smem_attr((const void*)trsm_llnu_warp_kernel<R>, (int)((size_t)(32 * R) * (32 * R + 1) * sizeof(double))));
  trsm_llnu_warp_kernel<R><<<(unsigned)blocks, 256, smem, s>>>((int)m, n, L, ldl, B, ldb);
  count_launch();
  return check_launch("trsm_llnu_warp_kernel");
}

template <typename T, int R, int SW>
int launch_trsm_t(int64_t m, int64_t n, const T* L, int64_t ldl, T* B, int64_t ldb, cudaStream_t s) {
  int64_t blocks = (n + SW - 1) / SW;
  if (blocks > 0x7fffffff) return set_error(HPL_ERR_NOTSUP, "trsm: too many columns");
  trsm_llnu_kernel<T, R, SW><<<(unsigned)blocks, kTrsmThreads, 0, s>>>((int)m, n, L, ldl, B, ldb);
  count_launch();
  return check_launch("trsm_llnu_kernel");
}

}  // namespace

int launch_trsm_llnu_strip(int64_t m, int64_t n, const double* L, int64_t ldl, double* B, int64_t ldb,
                           cudaStream_t s) {
  if (m <= 0 || n <= 0) return HPL_OK;
  // a warp per column while L fits in shared memory and the columns are few
  // (each CTA stages all of L for 8 columns)
  if (m <= 32) return launch_trsm_warp<1>(m, n, L, ldl, B, ldb, s);
  if (m <= 64 && n <= 4096) return launch_trsm_warp<2>(m, n, L, ldl, B, ldb, s);
  if (m <= 128 && n <= 1024) return launch_trsm_warp<4>(m, n, L, ldl, B, ldb, s);
  if (m <= 256) return launch_trsm_t<double, 1, 16>(m, n, L, ldl, B, ldb, s);
  if (m <= 512) return launch_trsm_t<double, 2, 16>(m, n, L, ldl, B, ldb, s);
  if (m <= 1024) return launch_trsm_t<double, 4, 8>(m, n, L, ldl, B, ldb, s);
  return set_error(HPL_ERR_NOTSUP, "trsm: triangle larger than 1024 rows");
}

// Blocked over 128-row diagonal blocks (as LAPACK's blocked TRSM): each
// block is solved by the strip kernel and the rows below it are updated by
// the FP64 GEMM, so that 7/8 of the flops of a 1024-row triangle (2/3 of a
// 384-row one) run at the GEMM's rate instead of the substitution's.
int launch_trsm_llnu(int64_t m, int64_t n, const double* L, int64_t ldl, double* B, int64_t ldb,
                     cudaStream_t s) {
  if (m <= 0 || n <= 0) return HPL_OK;
  const int64_t bs = 128;
  if (m <= bs) return launch_trsm_llnu_strip(m, n, L, ldl, B, ldb, s);
  for (int64_t b0 = 0; b0 < m; b0 += bs) {
    const int64_t nb = bs < m - b0 ? bs : m - b0;
    HPL_TRY(launch_trsm_llnu_strip(nb, n, L + b0 + b0 * ldl, ldl, B + b0, ldb, s));
    if (b0 + nb < m)
      HPL_TRY(launch_dgemm(false, false, m - b0 - nb, n, nb, -1.0, L + (b0 + nb) + b0 * ldl, ldl, B + b0, ldb, 1.0,
                           B + b0 + nb, ldb, s));
  }
  return HPL_OK;
}

namespace {

__global__ void identity_f64_kernel(int64_t n, double* __restrict__ A, int64_t lda) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, j = t / n;
    A[i + j * lda] = i == j ? 1.0 : 0.0;
  }
}

__global__ void i_minus_lower_kernel(int64_t n, double* __restrict__ A, int64_t lda) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, j = t / n;
    A[i + j * lda] = i > j ? -A[i + j * lda] : 0.0;
  }
}

}  // namespace

int launch_identity_f64(int64_t n, double* A, int64_t lda, cudaStream_t s) {
  if (n <= 0) return HPL_OK;
  int64_t g = (n * n + 255) / 256;
  if (g > 4096) g = 4096;
  identity_f64_kernel<<<(unsigned)g, 256, 0, s>>>(n, A, lda);
  count_launch();
  return check_launch("identity_f64_kernel");
}

int launch_i_minus_lower(int64_t n, double* A, int64_t lda, cudaStream_t s) {
  if (n <= 0) return HPL_OK;
  int64_t g = (n * n + 255) / 256;
  if (g > 4096) g = 4096;
  i_minus_lower_kernel<<<(unsigned)g, 256, 0, s>>>(n, A, lda);
  count_launch();
  return check_launch("i_minus_lower_kernel");
}

// FP32 variant (the U12 solve of the mixed-precision LU).
int launch_strsm_llnu_strip(int64_t m, int64_t n, const float* L, int64_t ldl, float* B, int64_t ldb,
                            cudaStream_t s) {
  if (m <= 0 || n <= 0) return HPL_OK;
  if (m <= 256) return launch_trsm_t<float, 1, 16>(m, n, L, ldl, B, ldb, s);
  if (m <= 512) return launch_trsm_t<float, 2, 16>(m, n, L, ldl, B, ldb, s);
  if (m <= 1024) return launch_trsm_t<float, 4, 16>(m, n, L, ldl, B, ldb, s);
  if (m <= 2048) return launch_trsm_t<float, 8, 8>(m, n, L, ldl, B, ldb, s);
  return set_error(HPL_ERR_NOTSUP, "strsm: triangle larger than 2048 rows");
}

}  // namespace hplgb
