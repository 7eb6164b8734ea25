// mxp.cu -- the mixed-precision variant: unpivoted LU of a diagonally dominant
// system whose trailing update runs on the tensor cores with BF16 or FP8-E4M3
// operands (one power-of-two scale per 128-row tile of L21 and per 128-column
// tile of U12, FP32 accumulation), FP32 factors, and FP64 GMRES iterative
// refinement that wins FP64 accuracy back.  (The paper only names HPL-MxP,
// Sec. I; the steps follow the definition written out in the oracle.)
//
// Per panel of nb columns (k0 .. e = k0 + jb):
//   1. FP32 LU of the m x jb panel without interchanges: the jb x jb diagonal
//      block A11 = L11 U11 by one cooperative kernel (mxp_diag.cu), L11^-1 and
//      U11^-1 by recursive doubling (mxp_trinv.cu), then L21 = A21 U11^-1 as one FP32-accurate product
//      on tcgen05 (three BF16 pieces per FP32 operand, six partial products,
//      FP32 accumulation);
//   2. U12 <- L11^-1 A12, the same kind of product;
//   3. tile maxima -> exponents e with amax 2^e <= qmax (exact, from the binary
//      exponents), then qL = cast(L21 2^eL) written K-major (transposed) and
//      qU = cast(U12 2^eU) (already K-major), K padded with zeros to 128 bytes;
//   4. A22 -= 2^-(eL+eU) qL qU^T on tcgen05 (mxp_gemm.cu).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace hplgb {

int launch_mxp_gemm(int prec, int64_t m, int64_t n, int64_t kp, const void* qL, const void* qU, const int* eL,
                    const int* eU, float* C, int64_t ldc, int* err, cudaStream_t s);
int launch_strsm_llnu_strip(int64_t m, int64_t n, const float* L, int64_t ldl, float* B, int64_t ldb,
                            cudaStream_t s);
int launch_gemm_x3(int64_t m, int64_t n, int64_t kpiece, const void* qL, const void* qU, const int* ezero, float* C,
                   int64_t ldc, int tri, int* err, cudaStream_t s, unsigned* amax, int amax_by);
int diag_scratch_floats(int64_t jb);
// max_ctas > 0 caps the kernel's CTAs (it needs all of them resident at once);
// mxp_diag_min_ctas(jb) is the fewest that can hold jb columns.
int launch_mxp_diag(Workspace* ws, int64_t jb, float* D, int64_t ldd, float* sc, int32_t* info, int64_t info_shift,
                    cudaStream_t s, int max_ctas = 0);
int mxp_diag_min_ctas(int64_t jb);
int mxp_update_tiles(int64_t m, int64_t n);
int launch_mxp_gemm_part(int prec, int64_t m, int64_t n, int64_t kp, const void* qL, const void* qU, const int* eL,
                         const int* eU, float* C, int64_t ldc, int* err, cudaStream_t s, int tile_lo, int tile_hi,
                         int max_ctas, int* tile_ctr);
int trinv_work_floats(int64_t jb);
int launch_mxp_trinv(int64_t jb, const float* D, int64_t ldd, float* X, float* Y, float* wk, cudaStream_t s);

namespace {

// ------------------------------------------------------------- conversion
__global__ void cvt_f64_f32_kernel(int64_t n, const double* __restrict__ A, int64_t lda, float* __restrict__ W,
                                   int64_t ldw) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) W[i + j * ldw] = __double2float_rn(A[i + j * lda]);
}

// --------------------------------- FP32-accurate products on the tensor cores
// x = p0 + p1 + p2 with BF16 pieces, each rounded to nearest even: for normal
// x the two remainders are exact in FP32 and the last one has at most 8
// significant bits, so the split is exact.
__device__ __forceinline__ void split3_bf16(float x, __nv_bfloat16& p0, __nv_bfloat16& p1, __nv_bfloat16& p2) {
  p0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(p0);
  p1 = __float2bfloat16_rn(r1);
  p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
}

// Four pieces of one level packed for an 8-byte store.
__device__ __forceinline__ uint2 pack4(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c, __nv_bfloat16 d) {
  uint2 r;
  r.x = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
  r.y = (uint32_t)__bfloat16_as_ushort(c) | ((uint32_t)__bfloat16_as_ushort(d) << 16);
  return r;
}

// Columns of S (K x J, column-major) as rows of q: q[j][p kpiece + k] = piece p
// of S(k, j), zero for K <= k < kpiece.  One CTA per 4 columns; each thread
// takes 4 consecutive k (a float4 load where the column is 16-byte aligned)
// and stores 8 bytes per piece.
__global__ void __launch_bounds__(256)
split3_cols_kernel(int K, int64_t J, int kpiece, const float* __restrict__ S, int64_t ld,
                   __nv_bfloat16* __restrict__ q) {
  const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(S) & 15) == 0);
  for (int u = 0; u < 4; ++u) {
    const int64_t j = (int64_t)blockIdx.x * 4 + u;
    if (j >= J) return;
    const float* col = S + j * ld;
    __nv_bfloat16* row = q + j * 3 * (int64_t)kpiece;
    for (int k = 4 * threadIdx.x; k < kpiece; k += 4 * 256) {
      float x[4];
      if (vec && k + 3 < K) {
        const float4 v = *reinterpret_cast<const float4*>(col + k);
        x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = k + i < K ? col[k + i] : 0.0f;
      }
      __nv_bfloat16 p[3][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) split3_bf16(x[i], p[0][i], p[1][i], p[2][i]);
#pragma unroll
      for (int l = 0; l < 3; ++l)
        *reinterpret_cast<uint2*>(row + l * kpiece + k) = pack4(p[l][0], p[l][1], p[l][2], p[l][3]);
    }
  }
}

// Rows of S (I x K, column-major) as rows of q, through a 64 (k) x 32 (i)
// shared-memory transpose: loads run along S's columns, and each thread
// stores two consecutive k of a row (4 bytes per piece).  Grid
// (ceil(I / 32), kpiece / 64).
__global__ void __launch_bounds__(256)
split3_rows_kernel(int64_t I, int K, int kpiece, const float* __restrict__ S, int64_t ld,
                   __nv_bfloat16* __restrict__ q) {
  __shared__ float tile[64][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 64;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int kk = k0 + ty + 8 * r;
    const int64_t i = i0 + tx;
    tile[ty + 8 * r][tx] = (kk < K && i < I) ? S[i + (int64_t)kk * ld] : 0.0f;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ty + 8 * r;
    const int kk = k0 + 2 * tx;
    if (i < I) {
      __nv_bfloat16 a0, a1, a2, b0, b1, b2;
      split3_bf16(tile[2 * tx][ty + 8 * r], a0, a1, a2);
      split3_bf16(tile[2 * tx + 1][ty + 8 * r], b0, b1, b2);
      __nv_bfloat16* row = q + i * 3 * (int64_t)kpiece + kk;
      *reinterpret_cast<__nv_bfloat162*>(row) = __halves2bfloat162(a0, b0);
      *reinterpret_cast<__nv_bfloat162*>(row + kpiece) = __halves2bfloat162(a1, b1);
      *reinterpret_cast<__nv_bfloat162*>(row + 2 * kpiece) = __halves2bfloat162(a2, b2);
    }
  }
}

__global__ void identity_kernel(int n, float* __restrict__ X, int64_t ld) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    X[i + j * ld] = i == j ? 1.0f : 0.0f;
  }
}

// ------------------------------------------------------------ quantization
__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < (int)(blockDim.x >> 5) ? red[l] : 0.0f;
#pragma unroll
    for (int off = 16; off; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  }
  return v;
}

// Largest e with amax 2^e <= qmax = fq 2^Eq, from the binary exponents of amax
// (exact; subnormal amax scaled by 2^64 first); 0 for amax == 0 or non-finite;
// clamped to [-126, 126].
__device__ int scale_exp_dev(float amax, float fq, int Eq) {
  if (!(amax > 0.0f) || isinf(amax)) return 0;
  int shift = 0;
  uint32_t b = __float_as_uint(amax);
  if (((b >> 23) & 0xff) == 0) {
    b = __float_as_uint(amax * 0x1p64f);
    shift = 64;
  }
  int Ea = (int)((b >> 23) & 0xff) - 126 - shift;
  float fa = __uint_as_float((b & 0x7fffffu) | (126u << 23));
  int e = Eq - Ea - (fa > fq ? 1 : 0);
  return e > 126 ? 126 : (e < -126 ? -126 : e);
}

// Tile maxima of |x| as the bit patterns of non-negative floats (ordered like
// the values), accumulated with atomicMax; amax arrays start at zero.
// L21 (m2 x jb): blockIdx.x = 128-row tile, blockIdx.y = chunk of 64 columns;
// thread (r = t % 128, c = t / 128) walks its rows' columns in steps of 2.
__global__ void __launch_bounds__(256)
amax_rows_kernel(int64_t m2, int jb, const float* __restrict__ L, int64_t ld, unsigned* __restrict__ amax) {
  __shared__ float red[8];
  const int t = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * 128 + (t & 127);
  const int cb = blockIdx.y * 64, ce = min(jb, cb + 64);
  float v = 0.0f;
  if (i < m2)
    for (int c = cb + (t >> 7); c < ce; c += 2) v = fmaxf(v, fabsf(L[i + (int64_t)c * ld]));
  v = block_max(v, red);
  if (t == 0) atomicMax(&amax[blockIdx.x], __float_as_uint(v));
}

// U12 (jb x n2): blockIdx.x = group of 8 columns (inside one 128-column tile),
// threads walk the rows of each column (contiguous).
__global__ void __launch_bounds__(256)
amax_cols_kernel(int jb, int64_t n2, const float* __restrict__ U, int64_t ld, unsigned* __restrict__ amax) {
  __shared__ float red[8];
  const int64_t cbeg = (int64_t)blockIdx.x * 8;
  float v = 0.0f;
  for (int q = 0; q < 8; ++q) {
    const int64_t c = cbeg + q;
    if (c >= n2) break;
    for (int r = threadIdx.x; r < jb; r += 256) v = fmaxf(v, fabsf(U[r + c * ld]));
  }
  v = block_max(v, red);
  if (threadIdx.x == 0) atomicMax(&amax[cbeg / 128], __float_as_uint(v));
}

__global__ void exps_from_amax_kernel(int nt, const unsigned* __restrict__ amax, float fq, int Eq, int* __restrict__ exps) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nt) exps[t] = scale_exp_dev(__uint_as_float(amax[t]), fq, Eq);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

template <int KIND>
__device__ __forceinline__ void put_code(void* q, int64_t idx, float y) {
  if (KIND == 0) {
    reinterpret_cast<__nv_bfloat16*>(q)[idx] = __float2bfloat16_rn(y);
  } else {
    reinterpret_cast<__nv_fp8_storage_t*>(q)[idx] = __nv_cvt_float_to_fp8(y, __NV_SATFINITE, __NV_E4M3);
  }
}

// Four codes packed for one store: 4 bytes (E4M3) or 8 bytes (BF16).
template <int KIND>
__device__ __forceinline__ void put_code4(void* q, int64_t idx, const float (&y)[4]) {
  if (KIND == 0) {
    uint2 r;
    r.x = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(y[0])) |
          ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(y[1])) << 16);
    r.y = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(y[2])) |
          ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(y[3])) << 16);
    *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(q) + idx) = r;
  } else {
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) r |= (uint32_t)__nv_cvt_float_to_fp8(y[i], __NV_SATFINITE, __NV_E4M3) << (8 * i);
    *reinterpret_cast<uint32_t*>(reinterpret_cast<__nv_fp8_storage_t*>(q) + idx) = r;
  }
}

// qL[i * kp + k] = code(L21(i, k) 2^eL[i / 128]) for k < jb, 0 for jb <= k < kp:
// a 128 (k) x 32 (i) shared-memory transpose: loads run along L21's columns,
// and each thread stores 4 consecutive codes of a row in one packed store.
// Grid (ceil(m2 / 32), ceil(kp / 128)).
template <int KIND>
__global__ void __launch_bounds__(256)
quant_L_kernel(int64_t m2, int jb, int kp, const float* __restrict__ L, int64_t ld, const int* __restrict__ eL,
               void* __restrict__ qL) {
  __shared__ float tile[128][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 128;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int kk = k0 + ty + 8 * r;
    const int64_t i = i0 + tx;
    tile[ty + 8 * r][tx] = (kk < jb && i < m2) ? L[i + (int64_t)kk * ld] : 0.0f;
  }
  __syncthreads();
  const int kk = k0 + 4 * tx;
  if (kk >= kp) return;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ty + 8 * r;
    if (i < m2) {
      const float sc = pow2f(eL[i / 128]);
      float y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) y[q] = tile[4 * tx + q][ty + 8 * r] * sc;
      put_code4<KIND>(qL, i * kp + kk, y);
    }
  }
}

// qU[j * kp + k] = code(U12(k, j) 2^eU[j / 128]) (U12 column-major is K-major):
// one CTA per 4 columns, each thread 4 consecutive k (a float4 load where the
// column is 16-byte aligned, one packed store of 4 codes).
template <int KIND>
__global__ void __launch_bounds__(256)
quant_U_kernel(int jb, int64_t n2, int kp, const float* __restrict__ U, int64_t ld, const int* __restrict__ eU,
               void* __restrict__ qU) {
  const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(U) & 15) == 0);
  for (int q = 0; q < 4; ++q) {
    const int64_t j = (int64_t)blockIdx.x * 4 + q;
    if (j >= n2) return;
    const float sc = pow2f(eU[j / 128]);
    const float* col = U + j * ld;
    for (int kk = 4 * threadIdx.x; kk < kp; kk += 4 * 256) {
      float y[4];
      if (vec && kk + 3 < jb) {
        const float4 v = *reinterpret_cast<const float4*>(col + kk);
        y[0] = v.x * sc, y[1] = v.y * sc, y[2] = v.z * sc, y[3] = v.w * sc;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) y[i] = kk + i < jb ? col[kk + i] * sc : 0.0f;
      }
      put_code4<KIND>(qU, j * kp + kk, y);
    }
  }
}

struct QFmt {
  float fq;
  int Eq;
};
QFmt qfmt(int prec) { return prec == 0 ? QFmt{0.5f, 1} : QFmt{0.875f, 9}; }  // qmax 1 = 0.5 2^1; 448 = 0.875 2^9

// amax scratch: 2 * ceil(m2 / 128) unsigned words, tile maxima of L21 then of
// U12.  Zeroed and filled here unless amax_ready (the products that wrote
// L21 and U12 took the maxima on the way out).
int quantize_panel(int prec, int64_t m2, int jb, int kp, const float* L21, const float* U12, int64_t ld, int* eL,
                   int* eU, void* qL, void* qU, unsigned* amax, int num_sms, cudaStream_t s, bool amax_ready = false) {
  (void)num_sms;
  QFmt f = qfmt(prec);
  const int64_t nt = (m2 + 127) / 128;
  if (!amax_ready) {
    HPL_CUDA(cudaMemsetAsync(amax, 0, 2 * nt * sizeof(unsigned), s));
    dim3 gA((unsigned)nt, (unsigned)((jb + 63) / 64));
    amax_rows_kernel<<<gA, 256, 0, s>>>(m2, jb, L21, ld, amax);
    amax_cols_kernel<<<(unsigned)((m2 + 7) / 8), 256, 0, s>>>(jb, m2, U12, ld, amax + nt);
    count_launch(2);
  }
  exps_from_amax_kernel<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>((int)nt, amax, f.fq, f.Eq, eL);
  exps_from_amax_kernel<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>((int)nt, amax + nt, f.fq, f.Eq, eU);
  count_launch(2);
  HPL_TRY(check_launch("exps kernels"));
  dim3 gL((unsigned)((m2 + 31) / 32), (unsigned)((kp + 127) / 128));
  const unsigned gu = (unsigned)((m2 + 3) / 4);
  if (prec == 0) {
    quant_L_kernel<0><<<gL, 256, 0, s>>>(m2, jb, kp, L21, ld, eL, qL);
    quant_U_kernel<0><<<gu, 256, 0, s>>>(jb, m2, kp, U12, ld, eU, qU);
  } else {
    quant_L_kernel<1><<<gL, 256, 0, s>>>(m2, jb, kp, L21, ld, eL, qL);
    quant_U_kernel<1><<<gu, 256, 0, s>>>(jb, m2, kp, U12, ld, eU, qU);
  }
  count_launch(2);
  return check_launch("quantize kernels");
}

// -------------------------------------------- FP32-factor solves (precond.)
// x <- U^-1 L^-1 x with the FP32 factors, in FP32.  Each sweep is one
// "wavefront" launch with one CTA per 128-row block: a CTA takes a ticket from
// a counter (tickets are handed out in the order CTAs start, so a CTA only
// ever waits for CTAs that are already running or done), subtracts the
// contributions of the blocks it depends on as their entries appear, applies
// the precomputed inverse of its diagonal block (staged in shared memory while
// it waits) and publishes its block.  Each published entry is one 64-bit word,
// the sweep's epoch above the FP32 bits, so a reader polls the entry itself:
// no flag, no fence, one round trip to L2.  Every wait is bounded (~1 s, then
// DEV_TIMEOUT).
constexpr int kTb = 128;  // block of the substitution

// Inverses of the diagonal kTb x kTb blocks: Dinv[b][k][t] = (T_bb^-1)(t, k),
// T = unit-lower L (LOWER) or upper U.  One CTA per block, thread t builds
// column t of the inverse by substitution in shared memory.
template <bool LOWER>
__global__ void __launch_bounds__(kTb)
invert_diag_blocks_kernel(int64_t n, const float* __restrict__ F, int64_t ldf, float* __restrict__ Dinv) {
  extern __shared__ float inv_smem[];
  float (*T)[kTb + 1] = reinterpret_cast<float (*)[kTb + 1]>(inv_smem);
  float (*Y)[kTb + 1] = reinterpret_cast<float (*)[kTb + 1]>(inv_smem + kTb * (kTb + 1));  // Y[i][t]: column t
  const int b = blockIdx.x, t = threadIdx.x;
  const int64_t r0 = (int64_t)b * kTb;
  const int nb = (int)((n - r0) < kTb ? (n - r0) : kTb);
  for (int c = 0; c < nb; ++c)
    if (t < nb) T[t][c] = F[(r0 + t) + (r0 + c) * ldf];
  __syncthreads();
  if (t < nb) {
    if (LOWER) {
      for (int i = 0; i < t; ++i) Y[i][t] = 0.0f;
      Y[t][t] = 1.0f;
      for (int i = t + 1; i < nb; ++i) {
        float acc = 0.0f;
        for (int k = t; k < i; ++k) acc = fmaf(T[i][k], Y[k][t], acc);
        Y[i][t] = -acc;
      }
    } else {
      for (int i = t + 1; i < nb; ++i) Y[i][t] = 0.0f;
      Y[t][t] = 1.0f / T[t][t];
      for (int i = t - 1; i >= 0; --i) {
        float acc = 0.0f;
        for (int k = i + 1; k <= t; ++k) acc = fmaf(T[i][k], Y[k][t], acc);
        Y[i][t] = -acc / T[i][i];
      }
    }
  }
  __syncthreads();
  float* D = Dinv + (int64_t)b * kTb * kTb;
  for (int k = 0; k < kTb; ++k) D[(int64_t)k * kTb + t] = (t < nb && k < nb) ? Y[t][k] : 0.0f;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// 512 threads = 16 warps.  For every block j the CTA depends on, warp w
// takes columns 8w..8w+7 of the 128 x 128 block of F and lane l rows
// 4l..4l+3 (float4 loads where the rows are 16-byte aligned): the warp loads
// its 4 KB of the block before it waits for the 8 entries of x it needs, so
// every CTA keeps a whole block of loads in flight, and it waits on its own
// (no CTA barrier per block).  The 16 partial sums per row are reduced once,
// at the end.
constexpr int kTrsvThreads = 512;
constexpr size_t kTrsvSmem = (size_t)kTb * kTb * sizeof(float);  // the inverse of the diagonal block

__device__ __forceinline__ float4 load_rows4(const float* __restrict__ F, int64_t ldf, int64_t r, int64_t c,
                                             int64_t n, bool vec) {
  const float* p = F + r + c * ldf;
  if (vec && r + 3 < n) return __ldg(reinterpret_cast<const float4*>(p));
  float4 v;
  v.x = r < n ? __ldg(p) : 0.0f;
  v.y = r + 1 < n ? __ldg(p + 1) : 0.0f;
  v.z = r + 2 < n ? __ldg(p + 2) : 0.0f;
  v.w = r + 3 < n ? __ldg(p + 3) : 0.0f;
  return v;
}

template <bool LOWER>
__global__ void __launch_bounds__(kTrsvThreads, 2)
trsv_wavefront_kernel(int64_t n, int nblk, const float* __restrict__ F, int64_t ldf, const float* __restrict__ Dinv,
                      const float* __restrict__ xin, float* __restrict__ xout, unsigned long long* __restrict__ xtag,
                      unsigned epoch, int* __restrict__ ticket, int* __restrict__ err) {
  constexpr int kWarps = kTrsvThreads / 32;
  extern __shared__ __align__(16) float Ds[];  // Ds[k * kTb + t] = (T_bb^-1)(t, k)
  __shared__ int s_q;
  __shared__ int s_fail;
  __shared__ __align__(16) float part[kWarps][kTb];
  __shared__ float acc_s[kTb];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t == 0) {
    s_q = atomicAdd(ticket, 1);
    s_fail = 0;
  }
  __syncthreads();
  const int q = s_q;
  const int b = LOWER ? q : nblk - 1 - q;
  const int64_t r0 = (int64_t)b * kTb;
  {
    const float* D = Dinv + (int64_t)b * kTb * kTb;
    for (int i = t; i < kTb * kTb / 4; i += kTrsvThreads) cp_async16(Ds + 4 * i, D + 4 * i);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const int64_t rl = r0 + 4 * lane;  // this lane's first row
  const bool vec = ((ldf & 3) == 0) && ((reinterpret_cast<uintptr_t>(F) & 15) == 0);
  float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
  bool ok = true;
  for (int jj = 0; jj < q && ok; ++jj) {
    const int j = LOWER ? jj : nblk - 1 - jj;
    const int64_t c0 = (int64_t)j * kTb + 8 * warp;  // this warp's first column
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      v[u] = c0 + u < n ? load_rows4(F, ldf, rl, c0 + u, n, vec) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float xv = 0.0f;
    if (lane < 8 && c0 + lane < n) {
      unsigned long long wv = ld_relaxed_u64(&xtag[c0 + lane]);
      if ((unsigned)(wv >> 32) != epoch) {
        const unsigned long long t0 = gtimer();
        while ((unsigned)((wv = ld_relaxed_u64(&xtag[c0 + lane])) >> 32) != epoch) {
          __nanosleep(32);
          if (gtimer() - t0 > 1000000000ULL || *(volatile int*)err == DEV_TIMEOUT) {
            atomicExch(err, DEV_TIMEOUT);
            ok = false;
            break;
          }
        }
      }
      xv = __uint_as_float((unsigned)wv);
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) break;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float xk = __shfl_sync(0xffffffffu, xv, u);
      a0 = fmaf(v[u].x, xk, a0);
      a1 = fmaf(v[u].y, xk, a1);
      a2 = fmaf(v[u].z, xk, a2);
      a3 = fmaf(v[u].w, xk, a3);
    }
  }
  if (!ok && lane == 0) atomicExch(&s_fail, 1);
  *reinterpret_cast<float4*>(&part[warp][4 * lane]) = make_float4(a0, a1, a2, a3);
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (s_fail) return;  // uniform: the block is not published, waiters time out fast
  if (t < kTb) {
    float acc = r0 + t < n ? xin[r0 + t] : 0.0f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) acc -= part[w][t];
    acc_s[t] = r0 + t < n ? acc : 0.0f;
  }
  __syncthreads();
  // x_b = (T_bb)^-1 acc: the same split over the inverse (128 x 128, zero padded)
  a0 = a1 = a2 = a3 = 0.0f;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int k = 8 * warp + u;
    const float4 d = *reinterpret_cast<const float4*>(Ds + k * kTb + 4 * lane);
    const float xk = acc_s[k];
    a0 = fmaf(d.x, xk, a0);
    a1 = fmaf(d.y, xk, a1);
    a2 = fmaf(d.z, xk, a2);
    a3 = fmaf(d.w, xk, a3);
  }
  __syncthreads();  // every warp has read part[] above
  *reinterpret_cast<float4*>(&part[warp][4 * lane]) = make_float4(a0, a1, a2, a3);
  __syncthreads();
  if (t < kTb && r0 + t < n) {
    float x = 0.0f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) x += part[w][t];
    xout[r0 + t] = x;
    st_relaxed_u64(&xtag[r0 + t], ((unsigned long long)epoch << 32) | __float_as_uint(x));
  }
}

struct TrsvState {
  float* dinvL = nullptr;
  float* dinvU = nullptr;
  size_t dinv_bytes = 0;
  int* flags = nullptr;   // 2 ticket counters
  size_t flag_ints = 0;
  unsigned long long* xtag = nullptr;  // [2][n]: published entries of the two sweeps, epoch << 32 | bits
  size_t xtag_n = 0;
  unsigned epoch = 0;
  const float* cached_lu = nullptr;
  int64_t cached_n = -1, cached_ld = -1;
};

// Buffers of the mixed-precision entry points, one set per device: grown on
// demand (growing synchronizes the device first) and freed by hpl_finalize.
struct MxpWork {
  void* qL = nullptr;
  void* qU = nullptr;
  int* eL = nullptr;
  int* eU = nullptr;
  unsigned* amax = nullptr;
  int* ctr = nullptr;      // tile counters of the look-ahead's shared updates, one per panel
  size_t q_bytes = 0, e_ints = 0, amax_bytes = 0, ctr_bytes = 0;
};

// Workspace of the FP32-accurate products on the tensor cores.
struct X3Work {
  float* linv = nullptr;   // L11^-1 (nb x nb)
  float* uinv = nullptr;   // U11^-1 (nb x nb)
  float* sc = nullptr;     // diagonal-kernel scratch
  float* wk = nullptr;     // work of the triangular inverses
  void* qa = nullptr;      // pieces of the rows of A
  void* qb = nullptr;      // pieces of the columns of B
  int* ezero = nullptr;    // zero tile exponents
  size_t linv_bytes = 0, uinv_bytes = 0, sc_bytes = 0, wk_bytes = 0, qa_bytes = 0, qb_bytes = 0, ezero_bytes = 0;
};

// Workspace for the solves and GMRES.
struct SolveWork {
  double* d = nullptr;
  size_t d_bytes = 0;
  float* f = nullptr;
  size_t f_bytes = 0;
};

struct MxpDevice {
  TrsvState trsv;
  MxpWork mxp;
  X3Work x3;
  SolveWork sw;
};
std::mutex g_mxp_mutex;
std::vector<MxpDevice*> g_mxp_dev;

// The current device's buffers (created empty on first use).
MxpDevice& mxp_state() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mxp_mutex);
  if ((int)g_mxp_dev.size() <= dev) g_mxp_dev.resize(dev + 1, nullptr);
  if (!g_mxp_dev[dev]) g_mxp_dev[dev] = new MxpDevice();
  return *g_mxp_dev[dev];
}

int trsv_prepare(int64_t n, const float* F, int64_t ldf, bool force, cudaStream_t s) {
  MxpDevice& st = mxp_state();
  const int64_t nblk = (n + kTb - 1) / kTb;
  const size_t bytes = (size_t)nblk * kTb * kTb * sizeof(float);
  if (st.trsv.dinv_bytes < bytes || st.trsv.xtag_n < (size_t)(2 * n) || st.trsv.flags == nullptr) {
    HPL_CUDA(cudaDeviceSynchronize());
    dev_free(st.trsv.dinvL, st.trsv.dinv_bytes);
    dev_free(st.trsv.dinvU, st.trsv.dinv_bytes);
    dev_free(st.trsv.flags, st.trsv.flag_ints * sizeof(int));
    dev_free(st.trsv.xtag, st.trsv.xtag_n * sizeof(unsigned long long));
    st.trsv.dinvL = st.trsv.dinvU = nullptr;
    st.trsv.flags = nullptr;
    st.trsv.xtag = nullptr;
    st.trsv.dinv_bytes = 0;
    st.trsv.flag_ints = 0;
    st.trsv.xtag_n = 0;
    HPL_TRY(dev_alloc((void**)&st.trsv.dinvL, bytes));
    st.trsv.dinv_bytes = bytes;  // dinvU below is the same size; freed together
    if (dev_alloc((void**)&st.trsv.dinvU, bytes) != HPL_OK) {
      dev_free(st.trsv.dinvL, bytes);
      st.trsv.dinvL = nullptr;
      st.trsv.dinv_bytes = 0;
      return set_error(HPL_ERR_ALLOC, "preconditioner workspace");
    }
    HPL_TRY(dev_alloc((void**)&st.trsv.flags, 2 * sizeof(int)));
    st.trsv.flag_ints = 2;
    HPL_TRY(dev_alloc((void**)&st.trsv.xtag, (size_t)(2 * n) * sizeof(unsigned long long)));
    HPL_CUDA(cudaMemset(st.trsv.flags, 0, 2 * sizeof(int)));
    HPL_CUDA(cudaMemset(st.trsv.xtag, 0, (size_t)(2 * n) * sizeof(unsigned long long)));
    st.trsv.xtag_n = (size_t)(2 * n);
    st.trsv.epoch = 0;
    force = true;
  }
  if (force || st.trsv.cached_lu != F || st.trsv.cached_n != n || st.trsv.cached_ld != ldf) {
    const int smem = 2 * kTb * (kTb + 1) * (int)sizeof(float);
    HPL_TRY(set_smem_attr((const void*)invert_diag_blocks_kernel<true>, smem));
    HPL_TRY(set_smem_attr((const void*)invert_diag_blocks_kernel<false>, smem));
    HPL_TRY(set_smem_attr((const void*)trsv_wavefront_kernel<true>, (int)kTrsvSmem));
    HPL_TRY(set_smem_attr((const void*)trsv_wavefront_kernel<false>, (int)kTrsvSmem));
    invert_diag_blocks_kernel<true><<<(unsigned)nblk, kTb, smem, s>>>(n, F, ldf, st.trsv.dinvL);
    invert_diag_blocks_kernel<false><<<(unsigned)nblk, kTb, smem, s>>>(n, F, ldf, st.trsv.dinvU);
    count_launch(2);
    HPL_TRY(check_launch("invert_diag_blocks_kernel"));
    st.trsv.cached_lu = F;
    st.trsv.cached_n = n;
    st.trsv.cached_ld = ldf;
  }
  return HPL_OK;
}

// x <- U^-1 L^-1 x (tmp: n floats of scratch).  trsv_prepare must have run
// for these factors.
int f32_solve(int64_t n, const float* F, int64_t ldf, float* x, float* tmp, int* dev_err, cudaStream_t s) {
  MxpDevice& st = mxp_state();
  const int nblk = (int)((n + kTb - 1) / kTb);
  if (st.trsv.xtag_n < (size_t)(2 * n)) return set_error(HPL_ERR_NOTSUP, "preconditioner not prepared for n");
  int* tickets = st.trsv.flags;
  const unsigned epoch = ++st.trsv.epoch;
  HPL_CUDA(cudaMemsetAsync(tickets, 0, 2 * sizeof(int), s));
  trsv_wavefront_kernel<true><<<(unsigned)nblk, kTrsvThreads, kTrsvSmem, s>>>(n, nblk, F, ldf, st.trsv.dinvL, x, tmp,
                                                                             st.trsv.xtag, epoch, tickets, dev_err);
  trsv_wavefront_kernel<false><<<(unsigned)nblk, kTrsvThreads, kTrsvSmem, s>>>(n, nblk, F, ldf, st.trsv.dinvU, tmp, x,
                                                                              st.trsv.xtag + n, epoch, tickets + 1,
                                                                              dev_err);
  count_launch(2);
  return check_launch("trsv_wavefront_kernel");
}

// ----------------------------------------------------- FP64 vector kernels
constexpr int kVec = 256;

// Partial sums of y = A x over column chunks, part[c * n + i], and (ABS) of
// the row sums of |A| from the same pass over A: thread i walks row i of
// chunk c (coalesced across the warp along the column).  On this GPU the FP64
// FMA pipe, not HBM, bounds the product (one DFMA per 8 bytes; conversions
// from double use the same pipe), so the |A| sums, which only feed ||A||_inf
// of the scaled residual, take |a| from the high word of the double with
// integer operations (exponent rebiased to binary32, the top 20 fraction bits
// kept: relative error below 2^-20) and add in FP32.
__device__ __forceinline__ float abs_from_hi(double v) {
  const int hi = __double2hiint(v) & 0x7fffffff;  // exponent (11 bits) and top 20 fraction bits
  if (hi < (897 << 20)) return 0.0f;              // below the binary32 normal range
  if (hi >= (1151 << 20)) return __int_as_float(0x7f800000);  // above it (or not finite)
  return __int_as_float((hi - (896 << 20)) << 3);
}

template <bool ABS>
__global__ void __launch_bounds__(kVec)
matvec_partial_kernel(int64_t n, const double* __restrict__ A, int64_t lda, const double* __restrict__ x,
                      int64_t chunk, double* __restrict__ part, double* __restrict__ part_abs) {
  const int64_t i = blockIdx.x * (int64_t)kVec + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (i >= n) return;
  const int64_t j0 = c * chunk, j1 = min(n, j0 + chunk);
  double s = 0.0;
  float t = 0.0f;
  for (int64_t j = j0; j < j1; ++j) {
    const double v = A[i + j * lda];
    s = fma(v, x[j], s);
    if (ABS) t += abs_from_hi(v);
  }
  part[c * n + i] = s;
  if (ABS) part_abs[c * n + i] = (double)t;
}

// y = alpha * (sum of partials, compensated) + beta * z (z may be null); with
// part_abs, rowabs[i] = the sum of its partials.
__global__ void matvec_reduce_kernel(int64_t n, int64_t nch, const double* __restrict__ part,
                                     const double* __restrict__ part_abs, double alpha, const double* __restrict__ z,
                                     double beta, double* __restrict__ y, double* __restrict__ rowabs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double hi = 0.0, lo = 0.0, ab = 0.0;
    for (int64_t c = 0; c < nch; ++c) {
      const double v = part[c * n + i];
      const double sm = __dadd_rn(hi, v);
      const double zz = __dsub_rn(sm, hi);
      lo = __dadd_rn(lo, __dadd_rn(__dsub_rn(hi, __dsub_rn(sm, zz)), __dsub_rn(v, zz)));
      hi = sm;
      if (part_abs) ab += part_abs[c * n + i];
    }
    const double r = alpha * __dadd_rn(hi, lo);
    y[i] = z ? fma(beta, z[i], r) : r;
    if (part_abs) rowabs[i] = ab;
  }
}

// out[j] (partials per block) of V(:, j)^T w for j < k: grid (chunks, k).
__global__ void __launch_bounds__(kVec)
multi_dot_kernel(int64_t n, const double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
                 double* __restrict__ part) {
  __shared__ double red[kVec / 32];
  const int j = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kVec + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVec)
    acc = fma(V[i + j * ldv], w[i], acc);
#pragma unroll
  for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kVec / 32; ++q) s += red[q];
    part[(int64_t)j * gridDim.x + blockIdx.x] = s;
  }
}

// h[j] = sum of part[j * nparts + p]
__global__ void sum_parts_kernel(int k, int nparts, const double* __restrict__ part, double* __restrict__ h) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += part[(int64_t)j * nparts + p];
  h[j] = s;
}

// w -= V(:, 0..k) h   (h on the device)
__global__ void gemv_sub_kernel(int64_t n, int k, const double* __restrict__ V, int64_t ldv, const double* __restrict__ h,
                                double* __restrict__ w) {
  __shared__ double hs[128];
  for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int j = 0; j < k; ++j) acc = fma(-V[i + j * ldv], hs[j], acc);
    w[i] = acc;
  }
}

// y = a x + b y (y is not read when b = 0).  x and y may be the same vector
// (the in-place scaling of GMRES), so neither is declared restrict.
__global__ void axpby_kernel(int64_t n, double a, const double* x, double b, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b == 0.0 ? 0.0 : b * y[i]);
}

// y = V(:, 0..k) c   (c on the device)
__global__ void gemv_n_kernel(int64_t n, int k, const double* __restrict__ V, int64_t ldv, const double* __restrict__ c,
                              double* __restrict__ y) {
  __shared__ double cs[128];
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = c[j];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(V[i + j * ldv], cs[j], acc);
    y[i] = acc;
  }
}

// FP64 <-> FP32 with scaling (the preconditioner works on r / m in FP32,
// m = max|r_i|).  m is reduced on the device from the per-block partial maxima
// of amax_f64_kernel (every block repeats the small reduction), so the solve
// needs no host round trip; m = 0 or a non-finite m is replaced by 1.
__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || isnan(b)) ? b : a; }

__device__ double scale_from_parts(const double* __restrict__ part, int nparts) {
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) v = nan_max(v, part[i]);
#pragma unroll
  for (int off = 16; off; off >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int off = 16; off; off >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (threadIdx.x == 0) red[0] = (v == 0.0 || !isfinite(v)) ? 1.0 : v;
  }
  __syncthreads();
  return red[0];
}

__global__ void scale_to_f32_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ part,
                                    int nparts, float* __restrict__ y) {
  const double s = 1.0 / scale_from_parts(part, nparts);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __double2float_rn(x[i] * s);
}
__global__ void scale_to_f64_kernel(int64_t n, const float* __restrict__ x, const double* __restrict__ part,
                                    int nparts, double* __restrict__ y) {
  const double s = scale_from_parts(part, nparts);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i] * s;
}

// max |x_i| (NaN-propagating) per block into part[blockIdx]
__global__ void amax_f64_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double red[kVec / 32];
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kVec + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVec) {
    double a = fabs(x[i]);
    v = (a > v || isnan(a)) ? a : v;
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    double o = __shfl_xor_sync(0xffffffffu, v, off);
    v = (o > v || isnan(o)) ? o : v;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int q = 0; q < kVec / 32; ++q) m = (red[q] > m || isnan(red[q])) ? red[q] : m;
    part[blockIdx.x] = m;
  }
}


}  // namespace

// ------------------------------------------------------- host-side drivers


static int mxp_grow(void** p, size_t* have, size_t want) {
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

// Frees every device's buffers (hpl_finalize).
void mxp_finalize() {
  std::lock_guard<std::mutex> lk(g_mxp_mutex);
  int cur = 0;
  cudaGetDevice(&cur);
  for (size_t d = 0; d < g_mxp_dev.size(); ++d) {
    MxpDevice* md = g_mxp_dev[d];
    if (!md) continue;
    cudaSetDevice((int)d);
    cudaDeviceSynchronize();
    dev_free(md->trsv.dinvL, md->trsv.dinv_bytes);
    dev_free(md->trsv.dinvU, md->trsv.dinv_bytes);
    dev_free(md->trsv.flags, md->trsv.flag_ints * sizeof(int));
    dev_free(md->trsv.xtag, md->trsv.xtag_n * sizeof(unsigned long long));
    dev_free(md->mxp.qL, md->mxp.q_bytes);
    dev_free(md->mxp.qU, md->mxp.q_bytes);
    dev_free(md->mxp.eL, md->mxp.e_ints * sizeof(int));
    dev_free(md->mxp.eU, md->mxp.e_ints * sizeof(int));
    dev_free(md->mxp.amax, md->mxp.amax_bytes);
    dev_free(md->mxp.ctr, md->mxp.ctr_bytes);
    dev_free(md->x3.linv, md->x3.linv_bytes);
    dev_free(md->x3.uinv, md->x3.uinv_bytes);
    dev_free(md->x3.sc, md->x3.sc_bytes);
    dev_free(md->x3.wk, md->x3.wk_bytes);
    dev_free(md->x3.qa, md->x3.qa_bytes);
    dev_free(md->x3.qb, md->x3.qb_bytes);
    dev_free(md->x3.ezero, md->x3.ezero_bytes);
    dev_free(md->sw.d, md->sw.d_bytes);
    dev_free(md->sw.f, md->sw.f_bytes);
    delete md;
    g_mxp_dev[d] = nullptr;
  }
  cudaSetDevice(cur);
}


// Sizes the buffers for products with up to `rows` rows or columns and inner
// dimension k (growing synchronizes the device: call before queueing).
static int x3_reserve(int64_t rows, int64_t k) {
  MxpDevice& st = mxp_state();
  const int64_t kpiece = (k + 63) / 64 * 64;
  HPL_TRY(mxp_grow(&st.x3.qa, &st.x3.qa_bytes, (size_t)rows * 3 * kpiece * 2));
  HPL_TRY(mxp_grow(&st.x3.qb, &st.x3.qb_bytes, (size_t)rows * 3 * kpiece * 2));
  HPL_TRY(mxp_grow((void**)&st.x3.linv, &st.x3.linv_bytes, (size_t)k * k * sizeof(float)));
  HPL_TRY(mxp_grow((void**)&st.x3.uinv, &st.x3.uinv_bytes, (size_t)k * k * sizeof(float)));
  HPL_TRY(mxp_grow((void**)&st.x3.sc, &st.x3.sc_bytes, (size_t)diag_scratch_floats(k) * sizeof(float)));
  HPL_TRY(mxp_grow((void**)&st.x3.wk, &st.x3.wk_bytes, (size_t)trinv_work_floats(k) * sizeof(float)));
  const size_t ez = (size_t)(rows / 128 + 2) * sizeof(int);
  if (st.x3.ezero_bytes < ez) {
    HPL_TRY(mxp_grow((void**)&st.x3.ezero, &st.x3.ezero_bytes, ez));
    HPL_CUDA(cudaMemset(st.x3.ezero, 0, ez));
  }
  return HPL_OK;
}

// C = A B in FP32 accuracy on the tensor cores: A (m x k, lda), B (k x n, ldb),
// C (m x n, ldc), all column-major FP32.  A and B are split into BF16 pieces
// first, so C may overlap either of them.  tri = 1 when A is lower triangular
// (m = k), 2 when B is upper triangular (n = k): the products skip the zero
// half.  amax / amax_by: see launch_gemm_x3 (tile maxima of C for the
// quantization that follows).  x3_reserve(max(m, n), k) first.
static int gemm_x3_apply(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda, const float* B, int64_t ldb,
                         float* C, int64_t ldc, int tri, int* err, cudaStream_t s, unsigned* amax = nullptr,
                         int amax_by = 0) {
  MxpDevice& st = mxp_state();
  if (m <= 0 || n <= 0 || k <= 0) return HPL_OK;
  const int64_t kpiece = (k + 63) / 64 * 64;
  if ((size_t)(m > n ? m : n) * 3 * kpiece * 2 > st.x3.qa_bytes ||
      (size_t)((m > n ? m : n) / 128 + 2) * sizeof(int) > st.x3.ezero_bytes)
    return set_error(HPL_ERR_NOTSUP, "x3 product workspace not reserved");
  dim3 gr((unsigned)((m + 31) / 32), (unsigned)(kpiece / 64));
  split3_rows_kernel<<<gr, 256, 0, s>>>(m, (int)k, (int)kpiece, A, lda, (__nv_bfloat16*)st.x3.qa);
  split3_cols_kernel<<<(unsigned)((n + 3) / 4), 256, 0, s>>>((int)k, n, (int)kpiece, B, ldb, (__nv_bfloat16*)st.x3.qb);
  count_launch(2);
  HPL_TRY(check_launch("split kernels"));
  return launch_gemm_x3(m, n, kpiece, st.x3.qa, st.x3.qb, st.x3.ezero, C, ldc, tri, err, s, amax, amax_by);
}

// B <- L^-1 B for the unit-lower m x m triangle L (m <= 2048) and B (m x n),
// FP32: X = L^-1 by substitution on the identity (the strip kernel of trsm.cu),
// then B = X B by gemm_x3_apply.
int strsm_x3(int64_t m, int64_t n, const float* L, int64_t ldl, float* B, int64_t ldb, int* err, cudaStream_t s) {
  MxpDevice& st = mxp_state();
  if (m <= 0 || n <= 0) return HPL_OK;
  if (m > 2048) return set_error(HPL_ERR_NOTSUP, "strsm: triangle larger than 2048 rows");
  HPL_TRY(x3_reserve(m > n ? m : n, m));
  int64_t g = (m * m + 255) / 256;
  if (g > 4096) g = 4096;
  identity_kernel<<<(unsigned)g, 256, 0, s>>>((int)m, st.x3.linv, m);
  count_launch();
  HPL_TRY(launch_strsm_llnu_strip(m, m, L, ldl, st.x3.linv, m, s));
  return gemm_x3_apply(m, n, m, st.x3.linv, m, B, ldb, B, ldb, 1, err, s);
}

// Look-ahead of the mixed-precision LU (on unless HPLGB_MXP_LOOKAHEAD=0, and
// off under the phase timers, whose marks assume one stream).  After panel k
// is quantized, block column k+1 of its update runs first, on every SM; then
// panel k+1's diagonal kernel and inverses run on the look-ahead stream, on G
// CTAs (the fewest that hold the block; HPLGB_MXP_LA_DIAG_CTAS raises it),
// beside the rest of the update on the other SMs; a second launch of the
// update joins on the look-ahead stream when the inverses are done, and the
// two take their tiles from one counter.  Only the diagonal kernel gains from
// the overlap: it is bound by its barrier latency and leaves its SMs mostly
// idle, while the L21 / U12 products, run the same way, took as much from the
// update beside them as they gave.  Every entry is computed as without the
// look-ahead (the same products, K in the same order).  Returns G, or 0 for
// no look-ahead.
int mxp_lookahead_ctas(const Workspace* ws, int64_t n, int64_t nb) {
  const char* e = getenv("HPLGB_MXP_LOOKAHEAD");
  const char* tv = getenv("HPLGB_TIMERS");
  if ((e && e[0] == '0') || (tv && tv[0] == '1') || nb % 128 != 0 || n <= nb) return 0;
  int g = mxp_diag_min_ctas(nb);
  const char* c = getenv("HPLGB_MXP_LA_DIAG_CTAS");
  if (c && atoi(c) > g) g = atoi(c);
  return g > 0 && g + 16 <= ws->num_sms ? g : 0;
}

int mxp_getrf_impl(Workspace* ws, int64_t n, int64_t nb, int prec, const double* A64, int64_t lda, float* W,
                   int64_t ldw, int32_t* info, cudaStream_t s) {
  MxpDevice& st = mxp_state();
  const int eb = prec == 0 ? 2 : 1;
  const int64_t per128 = 128 / eb;  // elements per 128 bytes of K
  const int64_t kp_max = (nb + per128 - 1) / per128 * per128;
  const int64_t m2_max = n > nb ? n - nb : 0;
  size_t qb = (size_t)(m2_max > 0 ? m2_max : 1) * (size_t)kp_max * eb;
  size_t have_q = st.mxp.q_bytes, have_q2 = st.mxp.q_bytes;
  HPL_TRY(mxp_grow(&st.mxp.qL, &have_q, qb));
  HPL_TRY(mxp_grow(&st.mxp.qU, &have_q2, qb));
  st.mxp.q_bytes = have_q < have_q2 ? have_q : have_q2;
  size_t ei = (size_t)((m2_max + 127) / 128 + 1);
  size_t have_e = st.mxp.e_ints * sizeof(int), have_e2 = st.mxp.e_ints * sizeof(int);
  HPL_TRY(mxp_grow((void**)&st.mxp.eL, &have_e, ei * sizeof(int)));
  HPL_TRY(mxp_grow((void**)&st.mxp.eU, &have_e2, ei * sizeof(int)));
  st.mxp.e_ints = (have_e < have_e2 ? have_e : have_e2) / sizeof(int);
  HPL_TRY(mxp_grow((void**)&st.mxp.amax, &st.mxp.amax_bytes, 2 * ei * sizeof(unsigned)));
  const int64_t npanels = (n + nb - 1) / nb;
  const int la_diag = mxp_lookahead_ctas(ws, n, nb);
  if (la_diag) HPL_TRY(mxp_grow((void**)&st.mxp.ctr, &st.mxp.ctr_bytes, (size_t)npanels * sizeof(int)));
  HPL_TRY(x3_reserve(n, nb));
  if (info) HPL_CUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  HPL_CUDA(cudaMemsetAsync(ws->bar, 0, sizeof(unsigned long long), s));
  if (la_diag) HPL_CUDA(cudaMemsetAsync(st.mxp.ctr, 0, (size_t)npanels * sizeof(int), s));
  ws->bar_next = 0;
  cudaStream_t ls = ws->la_stream;
  cudaEvent_t ev_cols = ws->ev[1], ev_join = ws->ev[2];
  // HPLGB_MXP_DIAG_CTAS caps the diagonal kernel outside the look-ahead (default: up to 145 CTAs)
  const char* dc = getenv("HPLGB_MXP_DIAG_CTAS");
  const int diag_cap = dc ? atoi(dc) : 0;
  cvt_f64_f32_kernel<<<(unsigned)(n < 65536 ? n : 65536), 256, 0, s>>>(n, A64, lda, W, ldw);
  count_launch();
  HPL_TRY(check_launch("cvt_f64_f32_kernel"));
  phase_timing_begin(s);
  bool factored = false;  // this panel's diagonal block and inverses came from the look-ahead
  for (int64_t k0 = 0, kk = 0; k0 < n; k0 += nb, ++kk) {
    const int64_t jb = nb < n - k0 ? nb : n - k0;
    const int64_t e = k0 + jb, m2 = n - e;
    float* P = W + k0 + k0 * ldw;
    if (!factored) {
      HPL_TRY(launch_mxp_diag(ws, jb, P, ldw, st.x3.sc, info, k0, s, diag_cap));
      HPL_TRY(launch_mxp_trinv(jb, P, ldw, st.x3.linv, st.x3.uinv, st.x3.wk, s));
    }
    factored = false;
    // the two products take the tile maxima for the quantization as they write
    const int64_t nt = (m2 + 127) / 128;
    if (m2 > 0) HPL_CUDA(cudaMemsetAsync(st.mxp.amax, 0, 2 * nt * sizeof(unsigned), s));
    HPL_TRY(gemm_x3_apply(m2, jb, jb, P + jb, ldw, st.x3.uinv, jb, P + jb, ldw, 2, ws->dev_err, s, st.mxp.amax,
                          1));  // L21
    phase_mark(PH_PANEL);
    if (m2 <= 0) break;
    HPL_TRY(gemm_x3_apply(jb, m2, jb, st.x3.linv, jb, W + k0 + e * ldw, ldw, W + k0 + e * ldw, ldw, 1, ws->dev_err,
                          s, st.mxp.amax + nt, 2));  // U12
    phase_mark(PH_TRSM);
    const int64_t kp = (jb + per128 - 1) / per128 * per128;
    HPL_TRY(quantize_panel(prec, m2, (int)jb, (int)kp, W + e + k0 * ldw, W + k0 + e * ldw, ldw, st.mxp.eL, st.mxp.eU,
                           st.mxp.qL, st.mxp.qU, st.mxp.amax, ws->num_sms, s, true));
    phase_mark(PH_QUANT);
    HPL_TRY(gemm_timing_begin(s));
    const int64_t jb2 = nb < m2 ? nb : m2;  // the next panel's width
    if (la_diag && jb2 % 128 == 0) {
      float* C2 = W + e + e * ldw;
      HPL_TRY(launch_mxp_gemm(prec, m2, jb2, kp, st.mxp.qL, st.mxp.qU, st.mxp.eL, st.mxp.eU, C2, ldw, ws->dev_err,
                              s));  // block column k+1
      HPL_CUDA(cudaEventRecord(ev_cols, s));
      HPL_CUDA(cudaStreamWaitEvent(ls, ev_cols, 0));
      HPL_TRY(launch_mxp_diag(ws, jb2, C2, ldw, st.x3.sc, info, e, ls, la_diag));
      HPL_TRY(launch_mxp_trinv(jb2, C2, ldw, st.x3.linv, st.x3.uinv, st.x3.wk, ls));
      const int64_t nr = m2 - jb2;
      if (nr > 0) {
        const void* qU2 = static_cast<const char*>(st.mxp.qU) + jb2 * kp * eb;
        const int* eU2 = st.mxp.eU + jb2 / 128;
        float* C3 = W + e + (e + jb2) * ldw;
        const int T = mxp_update_tiles(m2, nr);
        HPL_TRY(launch_mxp_gemm_part(prec, m2, nr, kp, st.mxp.qL, qU2, st.mxp.eL, eU2, C3, ldw, ws->dev_err, s, 0, T,
                                     ws->num_sms - la_diag, st.mxp.ctr + kk));
        HPL_TRY(launch_mxp_gemm_part(prec, m2, nr, kp, st.mxp.qL, qU2, st.mxp.eL, eU2, C3, ldw, ws->dev_err, ls, 0, T,
                                     la_diag, st.mxp.ctr + kk));
      }
      HPL_CUDA(cudaEventRecord(ev_join, ls));
      HPL_CUDA(cudaStreamWaitEvent(s, ev_join, 0));
      factored = true;
    } else {
      HPL_TRY(launch_mxp_gemm(prec, m2, m2, kp, st.mxp.qL, st.mxp.qU, st.mxp.eL, st.mxp.eU, W + e + e * ldw, ldw,
                              ws->dev_err, s));
    }
    // algorithmic: 2 m2^2 kp flop; bytes: C read and written (FP32) and both code blocks read once.  With
    // the look-ahead the bracket also holds the next diagonal kernel and inverses that ran beside the update.
    HPL_TRY(gemm_timing_end(s, 2.0 * (double)m2 * (double)m2 * (double)kp,
                            8.0 * (double)m2 * (double)m2 + 2.0 * (double)m2 * (double)kp * eb));
    phase_mark(PH_GEMM);
  }
  return HPL_OK;
}

int mxp_precond(Workspace* ws, int64_t n, const float* LU, int64_t ldl, const double* r, double* z, cudaStream_t s,
                double* amax_part, int nparts) {
  MxpDevice& st = mxp_state();
  phase_mark(PH_ORTH);
  // z = U^-1 L^-1 r computed in FP32 on r / max|r| (FP32 range), rescaled;
  // max|r| stays on the device
  amax_f64_kernel<<<nparts, kVec, 0, s>>>(n, r, amax_part);
  count_launch();
  float* x32 = st.sw.f;
  float* t32 = st.sw.f + n;
  int64_t g = (n + 255) / 256;
  if (g > ws->num_sms * 8) g = ws->num_sms * 8;
  scale_to_f32_kernel<<<(unsigned)g, 256, 0, s>>>(n, r, amax_part, nparts, x32);
  count_launch();
  HPL_TRY(f32_solve(n, LU, ldl, x32, t32, ws->dev_err, s));
  scale_to_f64_kernel<<<(unsigned)g, 256, 0, s>>>(n, x32, amax_part, nparts, z);
  count_launch();
  phase_mark(PH_PRECOND);
  return check_launch("mxp_precond");
}

}  // namespace hplgb

using namespace hplgb;

extern "C" {

int hpl_mxp_getrf(int64_t n, int64_t nb, int prec, const double* A64, int64_t lda, float* LU32, int64_t ldl,
                  int32_t* info, void* stream) {
  if (n < 0) return set_error(-1, "hpl_mxp_getrf: n < 0");
  if (nb < 32 || nb > 2048 || nb % 32) return set_error(-2, "hpl_mxp_getrf: nb must be a multiple of 32 in [32, 2048]");
  if (prec != 0 && prec != 1) return set_error(-3, "hpl_mxp_getrf: prec must be 0 (BF16) or 1 (E4M3)");
  if (n > 0 && !A64) return set_error(-4, "hpl_mxp_getrf: A64 is NULL");
  if (lda < (n > 1 ? n : 1)) return set_error(-5, "hpl_mxp_getrf: lda < max(1,n)");
  if (n > 0 && !LU32) return set_error(-6, "hpl_mxp_getrf: LU32 is NULL");
  if (ldl < (n > 1 ? n : 1)) return set_error(-7, "hpl_mxp_getrf: ldl < max(1,n)");
  HPL_TRY(fault_point("mxp_getrf"));
  if (n == 0) return HPL_OK;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  return mxp_getrf_impl(ws, n, nb, prec, A64, lda, LU32, ldl, info, (cudaStream_t)stream);
}

int hpl_mxp_getrs(int64_t n, const float* LU32, int64_t ldl, double* x, void* stream) {
  MxpDevice& st = mxp_state();
  if (n < 0) return set_error(-1, "hpl_mxp_getrs: n < 0");
  if (n > 0 && (!LU32 || !x)) return set_error(-2, "hpl_mxp_getrs: NULL pointer");
  if (ldl < (n > 1 ? n : 1)) return set_error(-3, "hpl_mxp_getrs: ldl < max(1,n)");
  HPL_TRY(fault_point("mxp_getrs"));
  if (n == 0) return HPL_OK;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  HPL_TRY(mxp_grow((void**)&st.sw.f, &st.sw.f_bytes, (size_t)2 * n * sizeof(float)));
  HPL_TRY(ensure_scratch(ws, 1024 * sizeof(double)));
  phase_timing_begin((cudaStream_t)stream);
  HPL_TRY(trsv_prepare(n, LU32, ldl, true, (cudaStream_t)stream));
  return mxp_precond(ws, n, LU32, ldl, x, x, (cudaStream_t)stream, ws->scratch, 256);
}

// Step 3 of the mixed-precision LU on its own (for testing): exponents of the
// 128-row tiles of L21 (m2 x jb) and the 128-column tiles of U12 (jb x m2),
// and their codes, K-major with row pitch kp (kp a multiple of 128 bytes).
int hpl_mxp_quantize(int prec, int64_t m2, int64_t jb, const float* L21, const float* U12, int64_t ld, int64_t kp,
                     int* eL, int* eU, void* qL, void* qU, void* stream) {
  MxpDevice& st = mxp_state();
  if (prec != 0 && prec != 1) return set_error(-1, "hpl_mxp_quantize: prec must be 0 or 1");
  if (m2 < 0 || jb < 0) return set_error(-2, "hpl_mxp_quantize: negative size");
  const int eb = prec == 0 ? 2 : 1;
  if (kp < jb || (kp * eb) % 128) return set_error(-7, "hpl_mxp_quantize: kp must be >= jb and a multiple of 128 bytes");
  if (ld < (m2 > jb ? m2 : jb)) return set_error(-6, "hpl_mxp_quantize: ld too small");
  if (m2 > 0 && jb > 0) {  // every operand is read or written (a NULL one would fault on the device)
    if (!L21) return set_error(-4, "hpl_mxp_quantize: L21 is NULL");
    if (!U12) return set_error(-5, "hpl_mxp_quantize: U12 is NULL");
    if (!eL) return set_error(-8, "hpl_mxp_quantize: eL is NULL");
    if (!eU) return set_error(-9, "hpl_mxp_quantize: eU is NULL");
    if (!qL) return set_error(-10, "hpl_mxp_quantize: qL is NULL");
    if (!qU) return set_error(-11, "hpl_mxp_quantize: qU is NULL");
  }
  HPL_TRY(fault_point("mxp_quantize"));
  if (m2 == 0 || jb == 0) return HPL_OK;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  HPL_TRY(mxp_grow((void**)&st.mxp.amax, &st.mxp.amax_bytes, (size_t)(2 * ((m2 + 127) / 128) + 2) * sizeof(unsigned)));
  return quantize_panel(prec, m2, (int)jb, (int)kp, L21, U12, ld, eL, eU, qL, qU, st.mxp.amax, ws->num_sms,
                        (cudaStream_t)stream);
}

int hpl_strsm_llnu(int64_t m, int64_t n, const float* L, int64_t ldl, float* B, int64_t ldb, void* stream) {
  if (m < 0 || m > 2048) return set_error(-1, "hpl_strsm_llnu: need 0 <= m <= 2048");
  if (n < 0) return set_error(-2, "hpl_strsm_llnu: n < 0");
  if (ldl < (m > 1 ? m : 1)) return set_error(-4, "hpl_strsm_llnu: ldl < max(1,m)");
  if (ldb < (m > 1 ? m : 1)) return set_error(-6, "hpl_strsm_llnu: ldb < max(1,m)");
  if (m > 0 && n > 0 && !L) return set_error(-3, "hpl_strsm_llnu: L is NULL");
  if (m > 0 && n > 0 && !B) return set_error(-5, "hpl_strsm_llnu: B is NULL");
  HPL_TRY(fault_point("strsm"));
  if (m == 0 || n == 0) return HPL_OK;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  return strsm_x3(m, n, L, ldl, B, ldb, ws->dev_err, (cudaStream_t)stream);
}

// Step 4 on its own (for testing): C (m x n, FP32) -= 2^-(eL+eU) qL qU^T.
int hpl_mxp_gemm(int prec, int64_t m, int64_t n, int64_t kp, const void* qL, const void* qU, const int* eL,
                 const int* eU, float* C, int64_t ldc, void* stream) {
  if (prec != 0 && prec != 1) return set_error(-1, "hpl_mxp_gemm: prec must be 0 or 1");
  if (m < 0 || n < 0 || kp < 0) return set_error(-2, "hpl_mxp_gemm: negative size");
  if (ldc < (m > 1 ? m : 1)) return set_error(-10, "hpl_mxp_gemm: ldc < max(1,m)");
  if (m > 0 && n > 0 && kp > 0) {  // nothing is read or written otherwise
    if (!qL) return set_error(-5, "hpl_mxp_gemm: qL is NULL");
    if (!qU) return set_error(-6, "hpl_mxp_gemm: qU is NULL");
    if (!eL) return set_error(-7, "hpl_mxp_gemm: eL is NULL");
    if (!eU) return set_error(-8, "hpl_mxp_gemm: eU is NULL");
    if (!C) return set_error(-9, "hpl_mxp_gemm: C is NULL");
  }
  HPL_TRY(fault_point("mxp_gemm"));
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  return launch_mxp_gemm(prec, m, n, kp, qL, qU, eL, eU, C, ldc, ws->dev_err, (cudaStream_t)stream);
}

// GMRES-IR (Carson and Higham 2018): x_{i+1} = x_i + d_i, where d_i solves
// A d = r_i = b - A x_i by left-preconditioned restarted GMRES in FP64 with
// M = L U the low-precision factors.  The Arnoldi basis is orthogonalized by
// classical Gram-Schmidt applied twice (CGS2: two batched projections per
// step instead of MGS's j sequential ones; equally stable in FP64).  The
// outer loop stops when the HPL scaled residual of x is below `target`; the
// inner solve stops at a preconditioned residual reduction of inner_tol or at
// `restart` steps.  stats (host, 6 doubles): outer iterations, total inner
// iterations, final scaled residual, ||r||_inf, ||A||_inf, ||x||_inf.
int hpl_gmres_ir(int64_t n, const double* A, int64_t lda, const float* LU32, int64_t ldl, const double* b, double* x,
                 int restart, int max_outer, double inner_tol, double target, double* stats, void* stream) {
  MxpDevice& st = mxp_state();
  if (n <= 0) return set_error(-1, "hpl_gmres_ir: n must be > 0");
  if (!A || !LU32 || !b || !x || !stats) return set_error(-2, "hpl_gmres_ir: NULL pointer");
  if (lda < n || ldl < n) return set_error(-3, "hpl_gmres_ir: leading dimension < n");
  if (restart < 1 || restart > 120) return set_error(-8, "hpl_gmres_ir: restart must be in [1, 120]");
  if (max_outer < 1) return set_error(-9, "hpl_gmres_ir: max_outer must be >= 1");
  HPL_TRY(fault_point("gmres_ir"));
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  phase_timing_begin(s);
  const int m = restart;
  const int64_t chunk = 1024;
  const int64_t nch = (n + chunk - 1) / chunk;
  const int nparts = 256;
  // device doubles: V (n x (m+1)) | w | r | z | d | partial hi/lo (2 nch n) | dot parts | h
  size_t nd = (size_t)n * (m + 1) + 4 * (size_t)n + 2 * (size_t)nch * n + (size_t)(m + 2) * nparts + (m + 2) + nparts;
  HPL_TRY(mxp_grow((void**)&st.sw.d, &st.sw.d_bytes, nd * sizeof(double)));
  HPL_TRY(mxp_grow((void**)&st.sw.f, &st.sw.f_bytes, (size_t)2 * n * sizeof(float)));
  double* V = st.sw.d;
  double* w = V + (size_t)n * (m + 1);
  double* r = w + n;
  double* z = r + n;
  double* d = z + n;
  double* phi = d + n;
  double* plo = phi + (size_t)nch * n;
  double* dparts = plo + (size_t)nch * n;
  double* hdev = dparts + (size_t)(m + 2) * nparts;
  double* apart = hdev + (m + 2);
  int64_t gv = (n + 255) / 256;
  if (gv > ws->num_sms * 8) gv = ws->num_sms * 8;
  dim3 gmv((unsigned)((n + kVec - 1) / kVec), (unsigned)nch);

  auto amax = [&](const double* v, double* out) -> int {
    amax_f64_kernel<<<nparts, kVec, 0, s>>>(n, v, apart);
    count_launch();
    std::vector<double> h(nparts);
    HPL_CUDA(cudaMemcpyAsync(h.data(), apart, nparts * sizeof(double), cudaMemcpyDeviceToHost, s));
    HPL_CUDA(cudaStreamSynchronize(s));
    double mm = 0.0;
    for (double q : h) mm = (q > mm || std::isnan(q)) ? q : mm;
    *out = mm;
    return HPL_OK;
  };
  // dots V(:,0..k)^T v -> host hh[0..k)
  auto dots = [&](const double* Vb, int k, const double* v, double* hh) -> int {
    dim3 g(nparts, k);
    multi_dot_kernel<<<g, kVec, 0, s>>>(n, Vb, n, v, dparts);
    sum_parts_kernel<<<1, 128, 0, s>>>(k, nparts, dparts, hdev);
    count_launch(2);
    HPL_CUDA(cudaMemcpyAsync(hh, hdev, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    HPL_CUDA(cudaStreamSynchronize(s));
    return check_launch("dots");
  };
  // y = A v or r = b - A x, FP64 FMA over column chunks, chunks summed with
  // TwoSum; rowabs (may be null) receives the row sums of |A| from the same pass
  auto matvec = [&](const double* v, double* y, bool residual, double* rowabs) -> int {
    phase_mark(PH_ORTH);
    if (rowabs) matvec_partial_kernel<true><<<gmv, kVec, 0, s>>>(n, A, lda, v, chunk, phi, plo);
    else matvec_partial_kernel<false><<<gmv, kVec, 0, s>>>(n, A, lda, v, chunk, phi, nullptr);
    matvec_reduce_kernel<<<(unsigned)gv, 256, 0, s>>>(n, nch, phi, rowabs ? plo : nullptr, residual ? -1.0 : 1.0,
                                                       residual ? b : nullptr, 1.0, y, rowabs);
    count_launch(2);
    phase_mark(PH_MATVEC);
    return check_launch("matvec");
  };

  double anorm = -1.0, bnorm = 0.0;  // ||A||_inf comes with the first residual
  HPL_TRY(amax(b, &bnorm));

  int outer = 0, inner_total = 0;
  double res_scaled = INFINITY, rn = 0.0, xn = 0.0;
  // inverses of the diagonal blocks of L and U, once for this solve
  HPL_TRY(trsv_prepare(n, LU32, ldl, true, s));
  // x0 = M^-1 b
  HPL_TRY(mxp_precond(ws, n, LU32, ldl, b, x, s, apart, nparts));
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hh(m + 1), y(m);
  for (outer = 0; outer < max_outer; ++outer) {
    HPL_TRY(matvec(x, r, true, anorm < 0.0 ? w : nullptr));  // r = b - A x (FP64, over column chunks)
    if (anorm < 0.0) HPL_TRY(amax(w, &anorm));                 // ||A||_inf: the largest row sum of |A|
    HPL_TRY(amax(r, &rn));
    HPL_TRY(amax(x, &xn));
    const double eps = 0x1p-53;
    res_scaled = rn / (eps * (anorm * xn + bnorm) * (double)n);
    if (res_scaled < target || !std::isfinite(res_scaled)) break;
    // GMRES on A d = r, left preconditioned: z = M^-1 r
    HPL_TRY(mxp_precond(ws, n, LU32, ldl, r, z, s, apart, nparts));
    double beta = 0.0;
    HPL_TRY(dots(z, 1, z, &beta));
    beta = sqrt(beta);
    if (beta == 0.0 || !std::isfinite(beta)) break;
    axpby_kernel<<<(unsigned)gv, 256, 0, s>>>(n, 1.0 / beta, z, 0.0, V);
    count_launch();
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * n;
      double* vn = V + (size_t)(j + 1) * n;
      HPL_TRY(matvec(vj, w, false, nullptr));                     // w = A v_j
      HPL_TRY(mxp_precond(ws, n, LU32, ldl, w, vn, s, apart, nparts));  // v_{j+1} = M^-1 A v_j
      // CGS2 against v_0..v_j
      for (int q = 0; q <= j; ++q) H[(size_t)j * (m + 1) + q] = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        HPL_TRY(dots(V, j + 1, vn, hh.data()));
        HPL_CUDA(cudaMemcpyAsync(hdev, hh.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
        gemv_sub_kernel<<<(unsigned)gv, 256, 0, s>>>(n, j + 1, V, n, hdev, vn);
        count_launch();
        for (int q = 0; q <= j; ++q) H[(size_t)j * (m + 1) + q] += hh[q];
      }
      double hn = 0.0;
      HPL_TRY(dots(vn, 1, vn, &hn));
      hn = sqrt(hn);
      H[(size_t)j * (m + 1) + j + 1] = hn;
      if (hn > 0.0) {
        axpby_kernel<<<(unsigned)gv, 256, 0, s>>>(n, 1.0 / hn, vn, 0.0, vn);
        count_launch();
      }
      // Givens rotations on column j
      double* hc = &H[(size_t)j * (m + 1)];
      for (int q = 0; q < j; ++q) {
        double t = cs[q] * hc[q] + sn[q] * hc[q + 1];
        hc[q + 1] = -sn[q] * hc[q] + cs[q] * hc[q + 1];
        hc[q] = t;
      }
      double den = hypot(hc[j], hc[j + 1]);
      cs[j] = den > 0 ? hc[j] / den : 1.0;
      sn[j] = den > 0 ? hc[j + 1] / den : 0.0;
      hc[j] = den;
      hc[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++inner_total;
      if (fabs(g[j + 1]) <= inner_tol * beta || hn == 0.0) {
        ++j;
        break;
      }
    }
    const int k = j < m ? j : m;
    // back substitution H(0:k,0:k) y = g
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int q = i + 1; q < k; ++q) t -= H[(size_t)q * (m + 1) + i] * y[q];
      y[i] = t / H[(size_t)i * (m + 1) + i];
    }
    HPL_CUDA(cudaMemcpyAsync(hdev, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
    gemv_n_kernel<<<(unsigned)gv, 256, 0, s>>>(n, k, V, n, hdev, d);
    axpby_kernel<<<(unsigned)gv, 256, 0, s>>>(n, 1.0, d, 1.0, x);  // x += d
    count_launch(2);
    HPL_TRY(check_launch("gmres update"));
  }
  phase_mark(PH_ORTH);
  stats[0] = outer;
  stats[1] = inner_total;
  stats[2] = res_scaled;
  stats[3] = rn;
  stats[4] = anorm;
  stats[5] = xn;
  HPL_CUDA(cudaStreamSynchronize(s));
  return HPL_OK;
}

}  // extern "C"
