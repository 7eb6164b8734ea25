// mxp_diag.cu -- the diagonal block of a mixed-precision panel: unpivoted LU
// A11 = L11 U11 of the jb x jb block (FP32, in place) together with X = L11^-1
// and Y = U11^-1, so that the rest of the panel and the U12 block row become
// products on the tensor cores (L21 = A21 U11^-1, U12 = L11^-1 A12).
//
// One launch of G = kRG x CG cooperating CTAs, blocked by 32:
//  forward, p = 0 .. nblk-1 (b = 32p, w = min(32, jb - b), e = b + w):
//    every CTA loads the diagonal block, factors it in shared memory (one
//    warp) and forms Li = L_pp^-1 and Ui = U_pp^-1 (one warp each); the
//    columns eliminated at step p are the trailing columns of A11 (c >= e) and
//    the columns of X that are already nonzero (c < e, X starts as I).  Column
//    group cg takes every CG-th of them and row group rg every kRG-th 32-row
//    chunk below the block:
//      z' = Li z for the block row of each of its columns (U_p,c, or X_p,c);
//      L_r = A_r U_pp^-1 for each of its rows;
//      col_r -= L_r z' for each of its (row, column) pairs;
//    then one grid barrier.
//  backward, p = nblk-1 .. 0: Y = U11^-1 by block back substitution on the
//    identity: y' = Ui y for the block row of each column c >= b, then
//    Y_r,c -= U_r,p y' for the rows r < b; the column block p of L (rows below
//    the block) and the factored diagonal block are written back in the same
//    sweep; one grid barrier per step.
// A value that other CTAs read during a step (the block row z, the column
// block A_r,p, the diagonal block) is written back only in the next step or
// in the backward sweep, so no CTA overwrites what another may still be
// reading.  Every barrier wait is bounded (~2 s, then DEV_TIMEOUT).
#include "common.cuh"

namespace hplgb {

namespace {

constexpr int kDB = 32;
constexpr int kDThreads = 256;
constexpr int kRG = 8;
constexpr unsigned long long kDiagTimeoutNs = 2000000000ULL;

__device__ __forceinline__ unsigned long long diag_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long diag_ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier on a monotone counter: false (and DEV_TIMEOUT) if it gave up.
__device__ bool diag_barrier(unsigned long long* ctr, unsigned long long target, int* err, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(ctr, 1ULL);
    const unsigned long long t0 = diag_now_ns();
    unsigned spins = 0;
    while (diag_ld_acquire(ctr) < target) {
      if (++spins > 32) __nanosleep(32);
      if ((spins & 255) == 0) {
        if (*(volatile int*)err == DEV_TIMEOUT || diag_now_ns() - t0 > kDiagTimeoutNs) {
          atomicExch(err, DEV_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

struct DiagArgs {
  int jb, cg;
  float* D;            // jb x jb block, factored in place
  int64_t ldd;
  float* X;            // out: L11^-1 (jb x jb)
  int64_t ldx;
  float* Y;            // out: U11^-1 (jb x jb)
  int64_t ldy;
  float* sc;           // scratch [nblk][2][32 x 32]: factored diagonal block, U_pp^-1
  int32_t* info;
  int64_t info_shift;
  unsigned long long* bar;
  unsigned long long bar_base;
  int* err;
};

struct DiagSmem {
  float T[kDB][kDB + 1];   // diagonal block: strict lower L_pp, upper U_pp
  float Li[kDB][kDB + 1];  // L_pp^-1
  float Ui[kDB][kDB + 1];  // U_pp^-1
  float Ac[kDB][kDB + 1];  // Ac[m][i] = D(r0 + i, b + m)
  float Lr[kDB][kDB + 1];  // Lr[k][i] = L(r0 + i, b + k)
  int flag;
};

// Column v of the step with block end e: X's column for v < e, else A11's.
__device__ __forceinline__ float* step_column(const DiagArgs& a, int v, int e) {
  return v < e ? a.X + (int64_t)v * a.ldx : a.D + (int64_t)v * a.ldd;
}

__global__ void __launch_bounds__(kDThreads)
mxp_diag_kernel(DiagArgs a) {
  __shared__ DiagSmem sm;
  extern __shared__ float Zs[];  // [own columns][32]: z' (forward) or y' (backward)
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = gridDim.x, g = blockIdx.x;
  const int rg = g % kRG, cgi = g / kRG, CG = a.cg;
  const int jb = a.jb, nblk = (jb + kDB - 1) / kDB, nch = (jb + 31) / 32;
  const int nown = cgi < jb ? (jb - cgi + CG - 1) / CG : 0;  // columns v = cgi + jj CG < jb
  unsigned long long target = a.bar_base;

  // X = Y = I
  for (int64_t idx = (int64_t)g * kDThreads + t; idx < (int64_t)jb * jb; idx += (int64_t)G * kDThreads) {
    const int i = (int)(idx % jb), j = (int)(idx / jb);
    a.X[i + (int64_t)j * a.ldx] = i == j ? 1.0f : 0.0f;
    a.Y[i + (int64_t)j * a.ldy] = i == j ? 1.0f : 0.0f;
  }
  target += G;
  if (!diag_barrier(a.bar, target, a.err, &sm.flag)) return;

  int prev_b = -1, prev_w = 0, prev_e = 0;  // block row whose write is deferred
  for (int p = 0; p < nblk; ++p) {
    const int b = p * kDB, w = min(kDB, jb - b), e = b + w;
    // the previous step's block row, now that every CTA has read it
    if (prev_b >= 0 && rg == 0)
      for (int jj = warp; jj < nown; jj += kDThreads / 32) {
        float* col = step_column(a, cgi + jj * CG, prev_e);
        if (lane < prev_w) col[prev_b + lane] = Zs[jj * kDB + lane];
      }
    // (1) diagonal block, padded with the identity
    for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
      const int r = idx & 31, c = idx >> 5;
      sm.T[r][c] = (r < w && c < w) ? a.D[b + r + (int64_t)(b + c) * a.ldd] : (r == c ? 1.0f : 0.0f);
    }
    __syncthreads();
    // (2) factor: lane i owns row i; a zero pivot leaves its column as it is
    if (warp == 0) {
      for (int j = 0; j < kDB; ++j) {
        const float piv = sm.T[j][j];
        if (lane > j && piv != 0.0f) {
          const float l = sm.T[lane][j] / piv;
          sm.T[lane][j] = l;
          for (int c = j + 1; c < kDB; ++c) sm.T[lane][c] = fmaf(-l, sm.T[j][c], sm.T[lane][c]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (warp == 0) {  // column `lane` of L_pp^-1 by forward substitution
      float x[kDB];
#pragma unroll
      for (int i = 0; i < kDB; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < i; ++k)
          if (k >= lane) acc = fmaf(sm.T[i][k], x[k], acc);
        x[i] = i < lane ? 0.0f : (i == lane ? 1.0f : -acc);
        sm.Li[i][lane] = x[i];
      }
    } else if (warp == 1) {  // column `lane` of U_pp^-1 by back substitution
      float y[kDB];
#pragma unroll
      for (int i = kDB - 1; i >= 0; --i) {
        float acc = 0.0f;
#pragma unroll
        for (int k = i + 1; k < kDB; ++k)
          if (k <= lane) acc = fmaf(sm.T[i][k], y[k], acc);
        y[i] = i > lane ? 0.0f : (i == lane ? 1.0f / sm.T[i][i] : -acc / sm.T[i][i]);
        sm.Ui[i][lane] = y[i];
      }
    }
    __syncthreads();
    if (g == 0) {  // for the backward sweep (no CTA reads the scratch before it)
      float* s = a.sc + (int64_t)p * 2 * kDB * kDB;
      for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
        const int r = idx & 31, c = idx >> 5;
        s[c * kDB + r] = sm.T[r][c];
        s[kDB * kDB + c * kDB + r] = sm.Ui[r][c];
      }
      if (t == 0 && a.info)
        for (int j = 0; j < w; ++j)
          if (sm.T[j][j] == 0.0f) {
            atomicCAS(a.info, 0, (int32_t)(a.info_shift + b + j + 1));
            break;
          }
    }
    // (3) block row of this CTA's columns: z' = L_pp^-1 z
    for (int jj = warp; jj < nown; jj += kDThreads / 32) {
      const float* col = step_column(a, cgi + jj * CG, e);
      const float zi = lane < w ? col[b + lane] : 0.0f;
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < kDB; ++k) acc = fmaf(sm.Li[lane][k], __shfl_sync(0xffffffffu, zi, k), acc);
      Zs[jj * kDB + lane] = acc;
    }
    __syncthreads();
    // (4) this row group's chunks below the block
    for (int q = rg; q < nch; q += kRG) {
      const int r0 = q * 32;
      if (r0 < e) continue;
      for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
        const int i = idx & 31, m = idx >> 5;
        sm.Ac[m][i] = (r0 + i < jb && m < w) ? a.D[r0 + i + (int64_t)(b + m) * a.ldd] : 0.0f;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 4; ++u) {  // L = A U_pp^-1
        const int k = warp * 4 + u;
        float acc = 0.0f;
#pragma unroll
        for (int m = 0; m < kDB; ++m) acc = fmaf(sm.Ac[m][lane], sm.Ui[m][k], acc);
        sm.Lr[k][lane] = acc;
      }
      __syncthreads();
      const int r = r0 + lane;
      for (int jj = warp; jj < nown; jj += kDThreads / 32) {
        float* col = step_column(a, cgi + jj * CG, e);
        if (r < jb) {
          float acc = col[r];
#pragma unroll
          for (int k = 0; k < kDB; ++k) acc = fmaf(-sm.Lr[k][lane], Zs[jj * kDB + k], acc);
          col[r] = acc;
        }
      }
      __syncthreads();
    }
    prev_b = b;
    prev_w = w;
    prev_e = e;
    target += G;
    if (!diag_barrier(a.bar, target, a.err, &sm.flag)) return;
  }
  if (rg == 0)
    for (int jj = warp; jj < nown; jj += kDThreads / 32) {
      float* col = step_column(a, cgi + jj * CG, prev_e);
      if (lane < prev_w) col[prev_b + lane] = Zs[jj * kDB + lane];
    }
  target += G;
  if (!diag_barrier(a.bar, target, a.err, &sm.flag)) return;

  // backward: Y = U11^-1; L's column blocks and the diagonal blocks written back
  prev_b = -1;
  for (int p = nblk - 1; p >= 0; --p) {
    const int b = p * kDB, w = min(kDB, jb - b), e = b + w;
    if (prev_b >= 0 && rg == 0)
      for (int jj = warp; jj < nown; jj += kDThreads / 32) {
        const int c = cgi + jj * CG;
        if (c >= prev_b && lane < prev_w) a.Y[prev_b + lane + (int64_t)c * a.ldy] = Zs[jj * kDB + lane];
      }
    const float* s = a.sc + (int64_t)p * 2 * kDB * kDB;
    for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
      const int r = idx & 31, c = idx >> 5;
      sm.Ui[r][c] = s[kDB * kDB + c * kDB + r];
    }
    __syncthreads();
    for (int jj = warp; jj < nown; jj += kDThreads / 32) {  // y' = U_pp^-1 y for columns c >= b
      const int c = cgi + jj * CG;
      if (c < b) continue;
      const float yi = lane < w ? a.Y[b + lane + (int64_t)c * a.ldy] : 0.0f;
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < kDB; ++k) acc = fmaf(sm.Ui[lane][k], __shfl_sync(0xffffffffu, yi, k), acc);
      Zs[jj * kDB + lane] = acc;
    }
    __syncthreads();
    for (int q = rg; q * 32 < b; q += kRG) {  // rows above: Y_r,c -= U_r,p y'
      const int r0 = q * 32;
      for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
        const int i = idx & 31, m = idx >> 5;
        sm.Ac[m][i] = m < w ? a.D[r0 + i + (int64_t)(b + m) * a.ldd] : 0.0f;
      }
      __syncthreads();
      for (int jj = warp; jj < nown; jj += kDThreads / 32) {
        const int c = cgi + jj * CG;
        if (c < b) continue;
        float* yc = a.Y + (int64_t)c * a.ldy;
        float acc = yc[r0 + lane];
#pragma unroll
        for (int k = 0; k < kDB; ++k) acc = fmaf(-sm.Ac[k][lane], Zs[jj * kDB + k], acc);
        yc[r0 + lane] = acc;
      }
      __syncthreads();
    }
    if (cgi == p % CG) {  // column block p of L below the block, and the block itself
      if (rg == 0)
        for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
          const int r = idx & 31, c = idx >> 5;
          if (r < w && c < w) a.D[b + r + (int64_t)(b + c) * a.ldd] = s[c * kDB + r];
        }
      for (int q = rg; q < nch; q += kRG) {
        const int r0 = q * 32;
        if (r0 < e) continue;
        for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
          const int i = idx & 31, m = idx >> 5;
          sm.Ac[m][i] = (r0 + i < jb && m < w) ? a.D[r0 + i + (int64_t)(b + m) * a.ldd] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = warp * 4 + u;
          float acc = 0.0f;
#pragma unroll
          for (int m = 0; m < kDB; ++m) acc = fmaf(sm.Ac[m][lane], sm.Ui[m][k], acc);
          if (k < w && r0 + lane < jb) a.D[r0 + lane + (int64_t)(b + k) * a.ldd] = acc;
        }
        __syncthreads();
      }
    }
    prev_b = b;
    prev_w = w;
    target += G;
    if (!diag_barrier(a.bar, target, a.err, &sm.flag)) return;
  }
  if (rg == 0)
    for (int jj = warp; jj < nown; jj += kDThreads / 32) {
      const int c = cgi + jj * CG;
      if (c >= prev_b && lane < prev_w) a.Y[prev_b + lane + (int64_t)c * a.ldy] = Zs[jj * kDB + lane];
    }
}

}  // namespace

int diag_scratch_floats(int64_t jb) { return (int)(((jb + kDB - 1) / kDB) * 2 * kDB * kDB); }

// Factor the jb x jb block D (ldd) in place and write X = L^-1, Y = U^-1
// (jb x jb, leading dimension jb).  jb <= 2048; sc holds
// diag_scratch_floats(jb) floats.
int launch_mxp_diag(Workspace* ws, int64_t jb, float* D, int64_t ldd, float* X, float* Y, float* sc, int32_t* info,
                    int64_t info_shift, cudaStream_t s) {
  if (jb <= 0) return HPL_OK;
  if (jb > 2048) return set_error(HPL_ERR_NOTSUP, "mxp diagonal block larger than 2048");
  int cg = (int)(jb / 64);
  if (cg < 1) cg = 1;
  if (cg > 16) cg = 16;
  while (kRG * cg > ws->num_sms && cg > 1) --cg;
  const int G = kRG * cg;
  const int nown = (int)((jb + cg - 1) / cg);
  const size_t dyn = (size_t)nown * kDB * sizeof(float);
  static bool attr = false;
  if (!attr) {
    HPL_CUDA(cudaFuncSetAttribute(mxp_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    attr = true;
  }
  DiagArgs a;
  a.jb = (int)jb;
  a.cg = cg;
  a.D = D;
  a.ldd = ldd;
  a.X = X;
  a.ldx = jb;
  a.Y = Y;
  a.ldy = jb;
  a.sc = sc;
  a.info = info;
  a.info_shift = info_shift;
  a.bar = ws->bar;
  a.bar_base = ws->bar_next;
  a.err = ws->dev_err;
  const int nblk = (int)((jb + kDB - 1) / kDB);
  ws->bar_next += (unsigned long long)G * (unsigned long long)(2 + 2 * nblk);
  mxp_diag_kernel<<<G, kDThreads, dyn, s>>>(a);
  count_launch();
  return check_launch("mxp_diag_kernel");
}

}  // namespace hplgb
