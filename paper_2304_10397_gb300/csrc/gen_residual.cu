// gen_residual.cu -- the random system (Sec. II) and the HPL scaled residual.
//
// Generator: 64-bit LCG s' = a s + c (mod 2^64); A(i,j) takes the state after
// t+1 steps, t = i + j n; b(i) takes t = n n + i; the value is
// (s >> 11) 2^-53 - 1/2.  Each thread jumps to its first element by composing
// the affine map with itself (repeated squaring) and then strides with a
// precomputed map, so the output is bit-identical to sequential stepping.
#include <math.h>
#include <stdio.h>

#include "common.cuh"

namespace hplgb {

namespace {

constexpr uint64_t kLcgA = 6364136223846793005ULL;
constexpr uint64_t kLcgC = 1442695040888963407ULL;

struct Affine {
  uint64_t mul, add;  // x -> mul * x + add (mod 2^64)
};

// Map for `steps` LCG steps.
__host__ __device__ inline Affine lcg_power(uint64_t steps) {
  Affine acc{1, 0}, sq{kLcgA, kLcgC};
  while (steps) {
    if (steps & 1) acc = Affine{sq.mul * acc.mul, sq.mul * acc.add + sq.add};
    sq = Affine{sq.mul * sq.mul, sq.mul * sq.add + sq.add};
    steps >>= 1;
  }
  return acc;
}

__device__ __forceinline__ double lcg_to_double(uint64_t s) {
  return __dsub_rn(__dmul_rn(__ull2double_rn(s >> 11), 0x1p-53), 0.5);
}

constexpr int kGenThreads = 256;

// One block per column (grid-stride over columns); thread r handles rows
// r, r + 256, ... of that column.
__global__ void __launch_bounds__(kGenThreads)
generate_kernel(int64_t n, uint64_t seed, double* __restrict__ A, int64_t lda, Affine stride) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    int64_t i = threadIdx.x;
    if (i >= n) continue;
    Affine f = lcg_power((uint64_t)j * (uint64_t)n + (uint64_t)i + 1);
    uint64_t s = f.mul * seed + f.add;
    double* col = A + j * lda;
    for (; i < n; i += kGenThreads) {
      col[i] = lcg_to_double(s);
      s = stride.mul * s + stride.add;
    }
  }
}

__global__ void generate_b_kernel(int64_t n, uint64_t seed, double* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  Affine f = lcg_power((uint64_t)n * (uint64_t)n + (uint64_t)i + 1);
  b[i] = lcg_to_double(f.mul * seed + f.add);
}

// Diagonal of the diagonally dominant system: sum over j != i of |A(i,j)| in
// ascending j with plain FP64 adds (the fixed order defines the value).
// Thread per row; reads A (coalesced across rows).
__global__ void dd_diag_kernel(int64_t n, double* __restrict__ A, int64_t lda) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int64_t j = 0; j < n; ++j)
    if (j != i) d = __dadd_rn(d, fabs(A[i + j * lda]));
  A[i + i * lda] = d;
}

// Same diagonal with the entries regenerated from the seed (no stored A).
__global__ void dd_diag_regen_kernel(int64_t n, uint64_t seed, Affine colstep, double* __restrict__ diag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  Affine f = lcg_power((uint64_t)i + 1);
  uint64_t s = f.mul * seed + f.add;  // element (i, 0)
  double d = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    if (j != i) d = __dadd_rn(d, fabs(lcg_to_double(s)));
    s = colstep.mul * s + colstep.add;
  }
  diag[i] = d;
}

// ---------------------------------------------------------------- residual
// Error-free transformations (Ogita, Rump, Oishi 2005): TwoProduct by FMA and
// Knuth's TwoSum, written with explicit round-to-nearest intrinsics so that
// the compiler cannot contract or reassociate them.
__device__ __forceinline__ void dot2_add(double& hi, double& lo, double a, double x) {
  double p = __dmul_rn(a, x);
  double pe = __fma_rn(a, x, -p);
  double s = __dadd_rn(hi, p);
  double z = __dsub_rn(s, hi);
  double e = __dadd_rn(__dsub_rn(hi, __dsub_rn(s, z)), __dsub_rn(p, z));
  hi = s;
  lo = __dadd_rn(lo, __dadd_rn(e, pe));
}

__device__ __forceinline__ void two_sum_into(double& hi, double& lo, double v) {
  double s = __dadd_rn(hi, v);
  double z = __dsub_rn(s, hi);
  double e = __dadd_rn(__dsub_rn(hi, __dsub_rn(s, z)), __dsub_rn(v, z));
  hi = s;
  lo = __dadd_rn(lo, e);
}

constexpr int kResThreads = 256;
constexpr int64_t kResChunk = 4096;  // columns per partial sum

// partial[(c * 3 + q) * n + i], q = 0 hi, 1 lo, 2 sum |a|, for chunk c.
// regen: entries from the seed (skipping j == i when dd: the diagonal is added
// in the combine step); else from A.
__global__ void __launch_bounds__(kResThreads)
residual_partial_kernel(int64_t n, uint64_t seed, int regen, int dd, Affine colstep,
                        const double* __restrict__ A, int64_t lda, const double* __restrict__ x,
                        double* __restrict__ partial) {
  int64_t i = blockIdx.x * (int64_t)kResThreads + threadIdx.x;
  int64_t c = blockIdx.y;
  int64_t j0 = c * kResChunk, j1 = min(n, j0 + kResChunk);
  if (i >= n) return;
  double hi = 0.0, lo = 0.0, ab = 0.0;
  if (regen) {
    Affine f = lcg_power((uint64_t)j0 * (uint64_t)n + (uint64_t)i + 1);
    uint64_t s = f.mul * seed + f.add;
    for (int64_t j = j0; j < j1; ++j) {
      double v = lcg_to_double(s);
      s = colstep.mul * s + colstep.add;
      if (dd && j == i) continue;
      dot2_add(hi, lo, v, x[j]);
      ab = __dadd_rn(ab, fabs(v));
    }
  } else {
    for (int64_t j = j0; j < j1; ++j) {
      double v = A[i + j * lda];
      dot2_add(hi, lo, v, x[j]);
      ab = __dadd_rn(ab, fabs(v));
    }
  }
  partial[(c * 3 + 0) * n + i] = hi;
  partial[(c * 3 + 1) * n + i] = lo;
  partial[(c * 3 + 2) * n + i] = ab;
}

// NaN-propagating max of non-negative values.
__device__ __forceinline__ double nmax(double a, double b) {
  if (isnan(a) || isnan(b)) return __longlong_as_double(0x7ff8000000000000LL);
  return a > b ? a : b;
}

// Per row: r_i = sum of chunk partials - b_i (+ diag_i x_i for the regenerated
// dd system), then block maxima of |r|, rowabs, |x|, |b| into blockmax[4*blk].
__global__ void __launch_bounds__(kResThreads)
residual_combine_kernel(int64_t n, int64_t nchunks, const double* __restrict__ partial,
                        const double* __restrict__ x, const double* __restrict__ b,
                        const double* __restrict__ diag, double* __restrict__ blockmax) {
  __shared__ double red[4][kResThreads / 32];
  int64_t i = blockIdx.x * (int64_t)kResThreads + threadIdx.x;
  double mr = 0, ma = 0, mx = 0, mb = 0;
  if (i < n) {
    double hi = -b[i], lo = 0.0, ab = 0.0;
    for (int64_t c = 0; c < nchunks; ++c) {
      two_sum_into(hi, lo, partial[(c * 3 + 0) * n + i]);
      lo = __dadd_rn(lo, partial[(c * 3 + 1) * n + i]);
      ab = __dadd_rn(ab, partial[(c * 3 + 2) * n + i]);
    }
    if (diag) {
      dot2_add(hi, lo, diag[i], x[i]);
      ab = __dadd_rn(ab, diag[i]);
    }
    double r = __dadd_rn(hi, lo);
    mr = fabs(r);
    ma = ab;
    mx = fabs(x[i]);
    mb = fabs(b[i]);
  }
  for (int off = 16; off; off >>= 1) {
    mr = nmax(mr, __shfl_xor_sync(0xffffffffu, mr, off));
    ma = nmax(ma, __shfl_xor_sync(0xffffffffu, ma, off));
    mx = nmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    mb = nmax(mb, __shfl_xor_sync(0xffffffffu, mb, off));
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { red[0][w] = mr; red[1][w] = ma; red[2][w] = mx; red[3][w] = mb; }
  __syncthreads();
  if (threadIdx.x < 4) {
    double m = 0;
    for (int k = 0; k < kResThreads / 32; ++k) m = nmax(m, red[threadIdx.x][k]);
    blockmax[blockIdx.x * 4 + threadIdx.x] = m;
  }
}

__global__ void residual_final_kernel(int64_t nblocks, int64_t n, const double* __restrict__ blockmax,
                                      double* __restrict__ out5) {
  __shared__ double red[4][32];
  double m[4] = {0, 0, 0, 0};
  for (int64_t k = threadIdx.x; k < nblocks; k += blockDim.x)
    for (int q = 0; q < 4; ++q) m[q] = nmax(m[q], blockmax[k * 4 + q]);
  for (int q = 0; q < 4; ++q)
    for (int off = 16; off; off >>= 1) m[q] = nmax(m[q], __shfl_xor_sync(0xffffffffu, m[q], off));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
    for (int q = 0; q < 4; ++q) red[q][w] = m[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    double r[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q)
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r[q] = nmax(r[q], red[q][k]);
    const double eps = 0x1p-53;
    double nn = (double)(n > 0 ? n : 1);
    out5[0] = r[0] / (eps * (r[1] * r[2] + r[3]) * nn);
    out5[1] = r[0];
    out5[2] = r[1];
    out5[3] = r[2];
    out5[4] = r[3];
  }
}

}  // namespace

int launch_generate(int64_t n, uint64_t seed, double* A, int64_t lda, double* b, cudaStream_t s) {
  if (n == 0) return HPL_OK;
  Affine stride = lcg_power(kGenThreads);
  int64_t blocks = n < 65536 * 4 ? n : 65536 * 4;
  generate_kernel<<<(unsigned)blocks, kGenThreads, 0, s>>>(n, seed, A, lda, stride);
  count_launch();
  HPL_TRY(check_launch("generate_kernel"));
  if (b) {
    generate_b_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, seed, b);
    count_launch();
    HPL_TRY(check_launch("generate_b_kernel"));
  }
  return HPL_OK;
}

int launch_dd_diag(int64_t n, double* A, int64_t lda, cudaStream_t s) {
  if (n == 0) return HPL_OK;
  dd_diag_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, A, lda);
  count_launch();
  return check_launch("dd_diag_kernel");
}

int launch_residual(Workspace* ws, int64_t n, uint64_t seed, int dd, const double* A, int64_t lda,
                    const double* x, const double* b, double* out5_host, cudaStream_t s) {
  if (n == 0) {
    for (int q = 0; q < 5; ++q) out5_host[q] = 0.0;
    return HPL_OK;
  }
  int64_t nchunks = (n + kResChunk - 1) / kResChunk;
  int64_t rblocks = (n + kResThreads - 1) / kResThreads;
  // scratch: partials | b (if regenerated) | diag (dd, regenerated) | blockmax | out5
  size_t off_partial = 0;
  size_t off_b = off_partial + (size_t)nchunks * 3 * n;
  size_t off_diag = off_b + (size_t)n;
  size_t off_bm = off_diag + (size_t)n;
  size_t off_out = off_bm + (size_t)rblocks * 4;
  size_t total = off_out + 8;
  HPL_TRY(ensure_scratch(ws, total * sizeof(double)));
  double* base = ws->scratch;
  double* partial = base + off_partial;
  double* bb = base + off_b;
  double* diag = base + off_diag;
  double* bm = base + off_bm;
  double* out = base + off_out;
  Affine colstep = lcg_power((uint64_t)n);
  const double* bsrc = b;
  if (!b) {
    generate_b_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, seed, bb);
    count_launch();
    HPL_TRY(check_launch("generate_b_kernel"));
    bsrc = bb;
  }
  int regen = A == nullptr;
  const double* dptr = nullptr;
  if (regen && dd) {
    dd_diag_regen_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, seed, colstep, diag);
    count_launch();
    HPL_TRY(check_launch("dd_diag_regen_kernel"));
    dptr = diag;
  }
  if (nchunks > 65535) return set_error(HPL_ERR_NOTSUP, "residual: n too large");
  dim3 grid((unsigned)rblocks, (unsigned)nchunks);
  residual_partial_kernel<<<grid, kResThreads, 0, s>>>(n, seed, regen, regen ? dd : 0, colstep, A,
                                                        lda, x, partial);
  count_launch();
  HPL_TRY(check_launch("residual_partial_kernel"));
  residual_combine_kernel<<<(unsigned)rblocks, kResThreads, 0, s>>>(n, nchunks, partial, x, bsrc,
                                                                     dptr, bm);
  count_launch();
  HPL_TRY(check_launch("residual_combine_kernel"));
  residual_final_kernel<<<1, 1024, 0, s>>>(rblocks, n, bm, out);
  count_launch();
  HPL_TRY(check_launch("residual_final_kernel"));
  HPL_CUDA(cudaMemcpyAsync(out5_host, out, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  HPL_CUDA(cudaStreamSynchronize(s));
  return HPL_OK;
}

}  // namespace hplgb
