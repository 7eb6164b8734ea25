// ozaki.cu -- the trailing update C <- C - A B of Sec. I (the DGEMM that takes
// nearly all of HPL's time) emulated in FP64 accuracy on the BF16 tensor
// cores, by the error-free slice products of Ozaki, Ogita, Oishi and Rump
// (Numer. Algorithms 59, 2012).  Not the paper's method: rocHPL runs this
// update as an FP64 DGEMM on the MI250X matrix cores.  On GB300 the FP64 pipe
// delivers 1.26 TFLOP/s while the BF16 tensor cores deliver about 1.9 PFLOP/s,
// so s (s + 1) / 2 BF16 products of integer slices still finish an order of
// magnitude sooner than one FP64 product.
//
//   split   every row r of A gets E_r with max_c |A(r,c)| < 2^E_r and every
//           column c of B gets F_c likewise; each entry, scaled into (-1, 1),
//           is peeled into s integer slices of beta bits (q_1 in
//           [-2^beta, 2^beta], the rest in [-2^(beta-1), 2^(beta-1)]), exactly,
//           and stored as BF16 (integers of <= 8 significant bits are exact in
//           BF16).  The peeling runs in 64-bit integer arithmetic on a fixed
//           point image of the entry (below).  A's slices go K-major in order
//           1..s along each row, B's in order s..1 along each column, so that
//           level d = i + j takes the first (d - 1) kp elements of A's rows and
//           the last (d - 1) kp of B's columns.
//   levels  P_d = sum_{i+j=d} Q_i Q'_j for d = 2 .. s+1 on tcgen05 (kind::f16,
//           FP32 accumulation in TMEM).  The host picks (s, beta) so that
//           K sum_{i+j=d} max|q_i| max|q'_j| <= 2^24: every partial sum is an
//           integer below 2^24, so the FP32 accumulation is exact and P_d is the
//           exact integer product, whatever the order of accumulation.
//   sum     the levels d >= d0 = max(2, s + 1 - floor(37 / beta)) exactly as a
//           64-bit integer T = sum P_d 2^((s+1-d) beta) (|T| < 2^63), rounded
//           once to FP64; then S = P_d + 2^-beta S in FP64 for d = d0-1 .. 2;
//           then C(r,c) <- C(r,c) - 2^(E_r + F_c - 2 beta) S: the oracle's
//           operations in the oracle's order, so the result is bitwise the
//           oracle's.
// The levels and the sum run fused in one persistent kernel (mxp_gemm.cu,
// ozaki_fused_kernel): per 128 x 128 tile of C the levels are made one after
// the other in TMEM and folded into an FP64 level sum kept in TMEM, and C is
// read and written once.  HPLGB_OZAKI_UNFUSED=1 runs the same arithmetic
// unfused instead: one product per level into an FP32 buffer in HBM, then a
// separate sum kernel.
// The pairs i + j > s + 1 are dropped; with s beta >= 54 the error is of the
// order of an FP64 DGEMM's rounding error (the bound is in the oracle's tests).
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace hplgb {

int launch_level_product(int64_t m, int64_t n, int64_t kext, int64_t pitch, const void* qa, const void* qb,
                         const int* ezero, float* P, int64_t ldp, int* err, cudaStream_t s);
int launch_ozaki_fused(int64_t m, int64_t n, int64_t kp, int s, int beta, int d0, const void* qa, const void* qb,
                       const int* E, const int* F, double* C, int64_t ldc, int* err, cudaStream_t st, int max_ctas,
                       int* tile_ctr = nullptr);

namespace {

constexpr int kMaxSlices = 12;
constexpr int kSplitRows = 32;     // rows of A per CTA of the row splitter
constexpr int kSplitCols = 32;     // columns of A per chunk of the row splitter

// The splitting in integer arithmetic (the FP64 pipe of GB300 runs 1/64 of
// the FP32 rate, the integer pipes do not): |x| < 2^E and
// X = x 2^(62 - E) is an integer below 2^62 in magnitude, exact for every x
// whose bits lie above 2^(E - 62); the bits below are folded into bit 0 (a
// sticky bit), which leaves every round-to-nearest-even decision at bit
// positions >= 2 as it would be with all bits (the host keeps s beta <= 60,
// so every slice boundary 62 - i beta is >= 2).  Slice i is
// q_i = rne(X_(i-1) / 2^(62 - i beta)), X_i = X_(i-1) - q_i 2^(62 - i beta):
// the same integers as t = a 2^beta, q = rint(t), a = t - q in FP64.

// Magnitude bits of x as an unsigned integer (orders like |x| for finite x).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}

// E with mu < 2^E <= 2 mu (the exponent of frexp) from mu's magnitude bits; 0
// for mu == 0 or a non-finite mu.
__device__ __forceinline__ int slice_exp_bits(unsigned long long b) {
  const int ex = (int)(b >> 52);
  if (b == 0 || ex == 0x7ff) return 0;
  if (ex == 0) return (63 - __clzll((long long)b)) + 1 - 1074;  // subnormal
  return ex - 1022;
}

// X = x 2^(62 - E) with the sticky bit (see above), as a signed integer.
__device__ __forceinline__ long long fixed62(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  unsigned long long M = b & 0xfffffffffffffULL;
  int e2;
  if (ex == 0) {
    e2 = -1074;
  } else {
    M |= 1ULL << 52;
    e2 = ex - 1075;
  }
  const int shift = e2 - E + 62;  // x 2^(62 - E) = M 2^shift
  unsigned long long X;
  if (M == 0) {
    X = 0;
  } else if (shift >= 0) {
    X = M << shift;  // < 2^62 because |x| < 2^E
  } else if (shift > -64) {
    const int r = -shift;
    X = (M >> r) | ((M & ((1ULL << r) - 1)) != 0 ? 1ULL : 0ULL);
  } else {
    X = 1;  // every bit is below 2^(E - 62): the sticky bit alone
  }
  return (b >> 63) ? -(long long)X : (long long)X;
}

// q = nearest integer to X / 2^p, ties to even (p >= 2), from the floor.
__device__ __forceinline__ long long rne_shift(long long X, int p) {
  const long long q0 = X >> p;  // arithmetic shift: floor
  const unsigned long long frac = (unsigned long long)(X - (q0 << p));
  const unsigned long long half = 1ULL << (p - 1);
  return (frac > half || (frac == half && (q0 & 1))) ? q0 + 1 : q0;
}

// Rows of A (m x k, column-major) -> E[r] and slices qa[(r * s + i) * kp + c]
// (BF16), zero for k <= c < kp.  CTA: 32 rows; phase 1 reduces the row maxima
// (8 warps over the columns), phase 2 peels 32 x 32 chunks and writes them
// out through shared memory, 64 contiguous bytes per (row, slice).
__global__ void __launch_bounds__(256)
ozaki_split_rows_kernel(int64_t m, int64_t k, int64_t kp, const double* __restrict__ A, int64_t lda, int s, int beta,
                        int* __restrict__ E, __nv_bfloat16* __restrict__ qa) {
  __shared__ unsigned long long red[8][kSplitRows];
  __shared__ int sE[kSplitRows];
  __shared__ __nv_bfloat16 sq[kMaxSlices][kSplitRows][kSplitCols + 4];  // rows 72 B apart: 8-byte aligned
  const int tr = threadIdx.x & 31, tc = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * kSplitRows;
  const int64_t r = r0 + tr;
  unsigned long long mu = 0;
  if (r < m)
    for (int64_t c = tc; c < k; c += 8) mu = max(mu, abs_bits(A[r + c * lda]));
  red[tc][tr] = mu;
  __syncthreads();
  if (tc == 0) {
    unsigned long long v = red[0][tr];
#pragma unroll
    for (int q = 1; q < 8; ++q) v = max(v, red[q][tr]);
    const int e = slice_exp_bits(v);
    sE[tr] = e;
    if (r < m) E[r] = e;
  }
  __syncthreads();
  const int e = sE[tr];
  for (int64_t c0 = 0; c0 < kp; c0 += kSplitCols) {
    // peel: thread (tr, tc) takes columns c0 + tc + 8 j of row tr
#pragma unroll 1
    for (int j = 0; j < kSplitCols / 8; ++j) {
      const int cc = tc + 8 * j;
      const int64_t c = c0 + cc;
      long long X = (r < m && c < k) ? fixed62(A[r + c * lda], e) : 0;
      int p = 62;
#pragma unroll 1
      for (int i = 0; i < s; ++i) {
        p -= beta;
        const long long q = rne_shift(X, p);
        X -= q << p;
        sq[i][tr][cc] = __float2bfloat16_rn((float)q);  // |q| <= 2^beta <= 256: exact
      }
    }
    __syncthreads();
    // write out: (row, slice) segments of 32 BF16 = 64 bytes, 8 bytes per thread
    const int segs = kSplitRows * s;
    for (int idx = threadIdx.x; idx < segs * (kSplitCols / 4); idx += 256) {
      const int seg = idx / (kSplitCols / 4), part = idx % (kSplitCols / 4);
      const int rr = seg / s, i = seg - rr * s;
      const int64_t row = r0 + rr;
      if (row >= m) continue;
      const uint2 v = *reinterpret_cast<const uint2*>(&sq[i][rr][part * 4]);
      *reinterpret_cast<uint2*>(qa + ((row * s + i) * kp + c0 + part * 4)) = v;
    }
    __syncthreads();
  }
}

// Columns of B (k x n, column-major) -> F[c] and slices in reverse order:
// qb[(c * s + (s - 1 - j)) * kp + r] = slice j + 1 of B(r, c) (BF16), zero for
// k <= r < kp.  One warp per column: the column is contiguous.
__global__ void __launch_bounds__(256)
ozaki_split_cols_kernel(int64_t k, int64_t n, int64_t kp, const double* __restrict__ B, int64_t ldb, int s, int beta,
                        int* __restrict__ F, __nv_bfloat16* __restrict__ qb) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= n) return;
  const double* col = B + c * ldb;
  unsigned long long mu = 0;
  for (int64_t r = lane; r < k; r += 32) mu = max(mu, abs_bits(col[r]));
#pragma unroll
  for (int o = 16; o; o >>= 1) mu = max(mu, (unsigned long long)__shfl_xor_sync(0xffffffffu, mu, o));
  const int e = slice_exp_bits(mu);
  if (lane == 0) F[c] = e;
  __nv_bfloat16* out = qb + c * s * kp;
  for (int64_t r = lane; r < kp; r += 32) {
    long long X = r < k ? fixed62(col[r], e) : 0;
    int p = 62;
#pragma unroll 1
    for (int j = 0; j < s; ++j) {
      p -= beta;
      const long long q = rne_shift(X, p);
      X -= q << p;
      out[(int64_t)(s - 1 - j) * kp + r] = __float2bfloat16_rn((float)q);
    }
  }
}

// The lowest level of the exact integer part of the level sum: the levels
// d >= d0 sum to |T| < 2^63 (|P_d| <= 2^24, weights 2^((s+1-d) beta)).
__host__ __device__ inline int int_level(int s, int beta) {
  const int d0 = s + 1 - 37 / beta;
  return d0 < 2 ? 2 : d0;
}

// C(r, c) <- C(r, c) - 2^(E_r + F_c - 2 beta) S(r, c), S the level sum of
// the levels P_d at P + (d - 2) * lvl_stride (column stride ldp): the levels
// d >= d0 exactly as a 64-bit integer T = sum P_d 2^((s+1-d) beta), rounded
// once, then S = P_d + 2^-beta S in FP64 for d = d0 - 1 .. 2.  All s levels of
// an element are loaded before the sum, so their loads are in flight together.
__global__ void __launch_bounds__(256)
ozaki_combine_kernel(int64_t m, int64_t n, int s, int beta, const float* __restrict__ P, int64_t ldp,
                     int64_t lvl_stride, const int* __restrict__ E, const int* __restrict__ F, double* __restrict__ C,
                     int64_t ldc) {
  const int d0 = int_level(s, beta);
  const double down = ldexp(1.0, -beta);
  for (int64_t c = blockIdx.y; c < n; c += gridDim.y) {
    const int fc = F[c];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
      const float* p = P + r + c * ldp;
      float lv[kMaxSlices];
#pragma unroll
      for (int i = 0; i < kMaxSlices; ++i) lv[i] = i < s ? p[(int64_t)i * lvl_stride] : 0.0f;  // level i + 2
      long long T = 0;
#pragma unroll
      for (int i = 0; i < kMaxSlices; ++i) {
        const int d = i + 2;
        if (d >= d0 && d <= s + 1)
          T += (long long)((unsigned long long)(long long)__float2int_rn(lv[i]) << ((s + 1 - d) * beta));
      }
      double S = ldexp(__ll2double_rn(T), -(s + 1 - d0) * beta);
#pragma unroll
      for (int i = kMaxSlices - 1; i >= 0; --i) {
        const int d = i + 2;
        if (d < d0) S = fma(S, down, (double)lv[i]);
      }
      const double scale = ldexp(1.0, E[r] + fc - 2 * beta);
      double* cp = C + r + c * ldc;
      *cp = fma(-scale, S, *cp);
    }
  }
}

__global__ void fill_zero_int_kernel(int n, int* __restrict__ p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0;
}

// Per-device buffers (grown on demand; growing synchronizes the device).
struct OzakiWork {
  void* qa = nullptr;
  void* qb = nullptr;
  int* E = nullptr;
  int* F = nullptr;
  int* ezero = nullptr;
  float* P = nullptr;
  size_t qa_bytes = 0, qb_bytes = 0, e_bytes = 0, f_bytes = 0, ezero_bytes = 0, p_bytes = 0;
};
// One set of buffers per (device, stream): the look-ahead panel factorization
// runs its emulated products on the library's second stream while the
// trailing update runs on the caller's, so the two must not share slices.
struct OzakiSlot {
  int dev;
  cudaStream_t stream;
  OzakiWork* w;
};
std::mutex g_oz_mutex;
std::vector<OzakiSlot> g_oz;

OzakiWork* oz_state(cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_oz_mutex);
  for (auto& e : g_oz)
    if (e.dev == dev && e.stream == st) return e.w;
  g_oz.push_back(OzakiSlot{dev, st, new OzakiWork()});
  return g_oz.back().w;
}

int oz_grow(void** p, size_t* have, size_t want) {
  if (*have >= want) return HPL_OK;
  if (*p) {
    HPL_CUDA(cudaDeviceSynchronize());
    dev_free(*p, *have);
    *p = nullptr;
    *have = 0;
  }
  HPL_TRY(dev_alloc(p, want));
  *have = want;
  return HPL_OK;
}

// Level sums stay exact in FP32 when k sum_{i+j=d} max|q_i| max|q_j| <= 2^24
// for every kept level d (max|q_1| = 2^beta, max|q_i| = 2^(beta-1) else).
bool levels_exact(int64_t k, int s, int beta) {
  for (int d = 2; d <= s + 1; ++d) {
    double bound = 0.0;
    for (int i = 1; i < d; ++i) {
      const int j = d - i;
      if (i > s || j > s) continue;
      bound += ldexp(1.0, i == 1 ? beta : beta - 1) * ldexp(1.0, j == 1 ? beta : beta - 1);
    }
    if ((double)k * bound > 16777216.0) return false;
  }
  return true;
}

}  // namespace

// Slice parameters for inner dimension k: s slices of beta bits with
// s beta >= 54 (as many bits as FP64 carries, plus one) and exact levels, the
// fewest slices first: (8, 7) up to k = 409, (9, 6) up to k = 1489.  With
// slices > 0 the caller fixes s; beta is then the largest width <= 8 that
// keeps the levels exact and s beta <= 60 (the integer splitter's range).
// Returns false if nothing fits.
bool ozaki_params(int64_t k, int slices, int* s_out, int* beta_out) {
  if (slices > 0) {
    if (slices > kMaxSlices) return false;
    for (int beta = 8; beta >= 1; --beta)
      if (slices * beta <= 60 && levels_exact(k, slices, beta)) {
        *s_out = slices;
        *beta_out = beta;
        return true;
      }
    return false;
  }
  const int cand[][2] = {{8, 7}, {9, 6}, {11, 5}};
  for (auto& c : cand)
    if (levels_exact(k, c[0], c[1])) {
      *s_out = c[0];
      *beta_out = c[1];
      return true;
    }
  return false;
}

// C (m x n, ldc) <- C - A B, A (m x k, lda), B (k x n, ldb), all FP64
// column-major, by slice products (see the top of the file).  k is taken in
// passes of at most 1024 (each pass a full update of its own); the unfused
// path takes C in column chunks that keep its level buffer within ~12 GB.
int launch_ozaki_gemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                      double* C, int64_t ldc, int slices, int* err, cudaStream_t st, int max_ctas,
                      const OzakiJoin* join) {
  if (m <= 0 || n <= 0 || k <= 0) return HPL_OK;
  const int64_t kc_max = 1024;
  if (k > kc_max) {
    for (int64_t k0 = 0; k0 < k; k0 += kc_max) {
      const int64_t kk = k - k0 < kc_max ? k - k0 : kc_max;
      HPL_TRY(launch_ozaki_gemm(m, n, kk, A + k0 * lda, lda, B + k0, ldb, C, ldc, slices, err, st, max_ctas));
    }
    return HPL_OK;
  }
  int s = 0, beta = 0;
  if (!ozaki_params(k, slices, &s, &beta))
    return set_error(HPL_ERR_NOTSUP, "emulated update: no exact slice parameters for k = %lld, %d slices",
                     (long long)k, slices);
  const int64_t kp = (k + 63) / 64 * 64;
  OzakiWork* w = oz_state(st);
  // fused: every level made and summed per tile in one kernel (no level
  // buffer); HPLGB_OZAKI_UNFUSED=1 takes the level products through HBM and
  // a separate sum kernel instead (the same arithmetic, bitwise the same)
  const char* uf = getenv("HPLGB_OZAKI_UNFUSED");
  const bool fused = !(uf && uf[0] == '1');
  // column chunk: s levels of m x nc FP32 within ~12 GB, a multiple of 256
  int64_t nc = (int64_t)((12.0e9 / 4.0) / ((double)s * (double)m));
  nc = nc / 256 * 256;
  if (nc < 256) nc = 256;
  if (nc > n) nc = n;
  HPL_TRY(oz_grow(&w->qa, &w->qa_bytes, (size_t)m * s * kp * 2));
  HPL_TRY(oz_grow(&w->qb, &w->qb_bytes, (size_t)n * s * kp * 2));
  HPL_TRY(oz_grow((void**)&w->E, &w->e_bytes, (size_t)m * sizeof(int)));
  HPL_TRY(oz_grow((void**)&w->F, &w->f_bytes, (size_t)n * sizeof(int)));
  const size_t ez = (size_t)((m > n ? m : n) / 128 + 2) * sizeof(int);
  if (w->ezero_bytes < ez) {
    HPL_TRY(oz_grow((void**)&w->ezero, &w->ezero_bytes, ez));
    fill_zero_int_kernel<<<64, 256, 0, st>>>((int)(ez / sizeof(int)), w->ezero);
    count_launch();
  }
  if (!fused) HPL_TRY(oz_grow((void**)&w->P, &w->p_bytes, (size_t)s * m * nc * sizeof(float)));
  ozaki_split_rows_kernel<<<(unsigned)((m + kSplitRows - 1) / kSplitRows), 256, 0, st>>>(
      m, k, kp, A, lda, s, beta, w->E, (__nv_bfloat16*)w->qa);
  ozaki_split_cols_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(k, n, kp, B, ldb, s, beta, w->F,
                                                                   (__nv_bfloat16*)w->qb);
  count_launch(2);
  HPL_TRY(check_launch("ozaki split kernels"));
  if (fused && join) {
    // both launches read this stream's slices; the caller keeps `st` from
    // reusing them until the joining launch is done
    HPL_CUDA(cudaEventRecord(join->ev, st));
    HPL_CUDA(cudaStreamWaitEvent(join->js, join->ev, 0));
    HPL_TRY(launch_ozaki_fused(m, n, kp, s, beta, int_level(s, beta), w->qa, w->qb, w->E, w->F, C, ldc, err, st,
                               max_ctas, join->ctr));
    return launch_ozaki_fused(m, n, kp, s, beta, int_level(s, beta), w->qa, w->qb, w->E, w->F, C, ldc, err,
                              join->js, join->js_ctas, join->ctr);
  }
  if (fused)
    return launch_ozaki_fused(m, n, kp, s, beta, int_level(s, beta), w->qa, w->qb, w->E, w->F, C, ldc, err, st,
                              max_ctas);
  const int64_t pitch = (int64_t)s * kp;
  const int64_t lvl_stride = m * nc;
  for (int64_t c0 = 0; c0 < n; c0 += nc) {
    const int64_t ncc = n - c0 < nc ? n - c0 : nc;
    const __nv_bfloat16* qbc = (const __nv_bfloat16*)w->qb + c0 * pitch;
    for (int d = 2; d <= s + 1; ++d) {
      // A: slices 1 .. d-1 (the first (d-1) kp of each row); B: slices d-1 .. 1
      // (the last (d-1) kp of each column)
      HPL_TRY(launch_level_product(m, ncc, (int64_t)(d - 1) * kp, pitch, w->qa, qbc + (int64_t)(s - d + 1) * kp,
                                   w->ezero, w->P + (int64_t)(d - 2) * lvl_stride, m, err, st));
    }
    int64_t gx = (m + 255) / 256;
    if (gx > 64) gx = 64;
    int64_t gy = ncc < 4096 ? ncc : 4096;
    ozaki_combine_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(m, ncc, s, beta, w->P, m, lvl_stride, w->E,
                                                                           w->F + c0, C + c0 * ldc, ldc);
    count_launch();
    HPL_TRY(check_launch("ozaki_combine_kernel"));
  }
  return HPL_OK;
}

void ozaki_finalize() {
  std::lock_guard<std::mutex> lk(g_oz_mutex);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& e : g_oz) {
    OzakiWork* w = e.w;
    cudaSetDevice(e.dev);
    cudaDeviceSynchronize();
    dev_free(w->qa, w->qa_bytes);
    dev_free(w->qb, w->qb_bytes);
    dev_free(w->E, w->e_bytes);
    dev_free(w->F, w->f_bytes);
    dev_free(w->ezero, w->ezero_bytes);
    dev_free(w->P, w->p_bytes);
    delete w;
  }
  g_oz.clear();
  cudaSetDevice(cur);
}

}  // namespace hplgb
