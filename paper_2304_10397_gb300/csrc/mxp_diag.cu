// mxp_diag.cu -- the diagonal block of a mixed-precision panel: unpivoted LU
// A11 = L11 U11 of the jb x jb block (FP32, in place) together with X = L11^-1
// and Y = U11^-1, so that the rest of the panel and the U12 block row become
// products on the tensor cores (L21 = A21 U11^-1, U12 = L11^-1 A12).
//
// One launch of G = kRG x CG cooperating CTAs, blocked by 32:
//  forward, p = 0 .. nblk-1 (b = 32p, w = min(32, jb - b), e = b + w):
//    every CTA factors the diagonal block and forms Li = L_pp^-1 and
//    Ui = U_pp^-1 with all its threads (elimination of [T | I], then back
//    substitution on [U | I]) while its block-row and column-block entries
//    arrive by cp.async; the
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

constexpr int kMaxChunks = 8;   // 32-row chunks per row group: jb <= 2048 = 8 x 8 x 32

struct DiagSmem {
  float T[kDB][kDB + 1];                 // diagonal block: strict lower L_pp, upper U_pp
  float Li[kDB][kDB + 1];                // L_pp^-1
  float Ui[kDB][kDB + 1];                // U_pp^-1
  float Ac[kMaxChunks][kDB][kDB + 1];    // Ac[q][m][i] = D(r0_q + i, b + m)
  float Lr[kMaxChunks][kDB][kDB + 1];    // Lr[q][k][i] = L(r0_q + i, b + k)  (or U_r,p backward)
  float Lsv[kDB][kDB + 1];               // multipliers of the diagonal block, kept apart while it is factored
  float Wk[kDB][kDB + 1];                // work array of the back substitution
  int flag;
};
// Zs (read as float4) follows DiagSmem at a 16-byte aligned offset.
constexpr size_t kZsOffset = (sizeof(DiagSmem) + 15) / 16 * 16;

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Column v of the step with block end e: X's column for v < e, else A11's.
__device__ __forceinline__ float* step_column(const DiagArgs& a, int v, int e) {
  return v < e ? a.X + (int64_t)v * a.ldx : a.D + (int64_t)v * a.ldd;
}

// Queue the copies of this CTA's 32-row chunks of columns b..b+w-1 (rows
// r0 = 32 q for q = rg, rg + kRG, ... with first_row <= r0 < last_row) into
// sm.Ac; entries outside the block read as zero.  Returns the chunk count.
__device__ __forceinline__ int queue_chunks(DiagSmem& sm, const DiagArgs& a, int rg, int b, int w, int first_row,
                                            int last_row) {
  int nq = 0;
  for (int q = rg; q * 32 < last_row; q += kRG) {
    const int r0 = q * 32;
    if (r0 < first_row) continue;
    for (int idx = threadIdx.x; idx < kDB * kDB; idx += kDThreads) {
      const int i = idx & 31, m = idx >> 5;
      if (r0 + i < a.jb && m < w) cp_async4(&sm.Ac[nq][m][i], a.D + r0 + i + (int64_t)(b + m) * a.ldd);
      else sm.Ac[nq][m][i] = 0.0f;
    }
    ++nq;
  }
  return nq;
}

// col_r -= sum_k Lr[q][k][r - r0_q] Z[jj][k] over this CTA's (chunk, column)
// pairs: lane = row within the chunk, pairs spread over the warps, kBatch
// loads in flight per lane.  FWD selects the forward columns (X below e,
// A11 above) or the backward ones (Y, columns c >= b only).
// First chunk index q = rg (mod kRG) with 32 q >= first_row.
__device__ __forceinline__ int first_chunk(int rg, int first_row) {
  const int q0 = (first_row + 31) / 32;
  return q0 <= rg ? rg : rg + (q0 - rg + kRG - 1) / kRG * kRG;
}

template <bool FWD>
__device__ __forceinline__ float* pair_column(const DiagArgs& a, int c, int b, int e) {
  return FWD ? step_column(a, c, e) : (c >= b ? a.Y + (int64_t)c * a.ldy : nullptr);
}

constexpr int kMaxCW = 16;  // columns per warp: ceil(jb / cg / 8) <= 16 for jb <= 2048

// col_r -= sum_k Lr[q][k][r - r0_q] Z[jj][k] over this CTA's (chunk, column)
// pairs.  Warp w takes the columns jj = w, w + 8, ...; lane = row within the
// chunk.  Per chunk the lane's 32 multipliers sit in registers and Z is read
// as float4 broadcasts; the next chunk's column entries are loaded while the
// current one is computed.  FWD selects the forward columns (X below e, A11
// above) or the backward ones (Y, columns c >= b only).
template <bool FWD>
__device__ __forceinline__ void apply_updates(DiagSmem& sm, const float* Zs, const DiagArgs& a, int rg, int cgi,
                                              int nown, int nq, int b, int e, int first_row) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qf = first_chunk(rg, first_row);
  float* cols[kMaxCW];
#pragma unroll
  for (int u = 0; u < kMaxCW; ++u) {
    const int jj = warp + 8 * u;
    cols[u] = jj < nown ? pair_column<FWD>(a, cgi + jj * a.cg, b, e) : nullptr;
  }
  float vcur[kMaxCW], vnext[kMaxCW];
  auto load = [&](int qi, float* v) {
    const int r = (qf + qi * kRG) * 32 + lane;
#pragma unroll
    for (int u = 0; u < kMaxCW; ++u) v[u] = (cols[u] && r < a.jb) ? cols[u][r] : 0.0f;
  };
  if (nq > 0) load(0, vcur);
  for (int qi = 0; qi < nq; ++qi) {
    if (qi + 1 < nq) load(qi + 1, vnext);
    float lr[kDB];
#pragma unroll
    for (int k = 0; k < kDB; ++k) lr[k] = sm.Lr[qi][k][lane];
    const int r = (qf + qi * kRG) * 32 + lane;
#pragma unroll
    for (int u = 0; u < kMaxCW; ++u) {
      if (!cols[u] || r >= a.jb) continue;
      const float4* z4 = reinterpret_cast<const float4*>(Zs + (warp + 8 * u) * kDB);
      float acc = vcur[u];
#pragma unroll
      for (int k4 = 0; k4 < kDB / 4; ++k4) {
        const float4 z = z4[k4];
        acc = fmaf(-lr[4 * k4], z.x, acc);
        acc = fmaf(-lr[4 * k4 + 1], z.y, acc);
        acc = fmaf(-lr[4 * k4 + 2], z.z, acc);
        acc = fmaf(-lr[4 * k4 + 3], z.w, acc);
      }
      cols[u][r] = acc;
    }
#pragma unroll
    for (int u = 0; u < kMaxCW; ++u) vcur[u] = vnext[u];
  }
}

// T (32 x 32, padded with the identity) -> packed L\U in T, Li = L^-1 and
// Ui = U^-1, by all threads: forward elimination of [T | I] (the right half
// becomes L^-1; the multipliers are kept in Lsv until the end, since every
// thread reads column j during step j), then back substitution on [U | I].
// A zero pivot leaves its column as it is: no multipliers, no update.
__device__ void factor_and_invert(DiagSmem& sm) {
  const int t = threadIdx.x;
  for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
    const int r = idx & 31, c = idx >> 5;
    sm.Li[r][c] = r == c ? 1.0f : 0.0f;
    sm.Wk[r][c] = r == c ? 1.0f : 0.0f;
  }
  __syncthreads();
  const int c = t & 63, r4 = t >> 6;  // column of [T | Li]; rows r4 + 4 k
  for (int j = 0; j < kDB; ++j) {
    const float piv = sm.T[j][j];
    const float rcp = piv != 0.0f ? 1.0f / piv : 0.0f;
    const float rowj = c < kDB ? sm.T[j][c] : sm.Li[j][c - kDB];
    // every load of the step before any store, so they overlap
    float trj[kDB / 4], cur[kDB / 4];
#pragma unroll
    for (int k = 0; k < kDB / 4; ++k) {
      const int r = r4 + 4 * k;
      trj[k] = sm.T[r][j];
      cur[k] = c < kDB ? sm.T[r][c] : sm.Li[r][c - kDB];
    }
#pragma unroll
    for (int k = 0; k < kDB / 4; ++k) {
      const int r = r4 + 4 * k;
      if (r <= j) continue;
      const float l = trj[k] * rcp;
      if (c < kDB) {
        if (c > j) sm.T[r][c] = fmaf(-l, rowj, cur[k]);
        else if (c == j) sm.Lsv[r][j] = piv != 0.0f ? l : trj[k];
      } else if (c - kDB <= j) {
        sm.Li[r][c - kDB] = fmaf(-l, rowj, cur[k]);
      }
    }
    __syncthreads();
  }
  for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
    const int r = idx & 31, cc = idx >> 5;
    if (r > cc) sm.T[r][cc] = sm.Lsv[r][cc];
  }
  const int cu = t & 31, r8 = t >> 5;  // column of U^-1; rows r8 + 8 k
  for (int j = kDB - 1; j >= 0; --j) {
    const float sj = sm.Wk[j][cu] * (1.0f / sm.T[j][j]);  // row j of U^-1
    float trj[kDB / 8], cur[kDB / 8];
#pragma unroll
    for (int k = 0; k < kDB / 8; ++k) {
      const int r = r8 + 8 * k;
      trj[k] = sm.T[r][j];
      cur[k] = sm.Wk[r][cu];
    }
#pragma unroll
    for (int k = 0; k < kDB / 8; ++k) {
      const int r = r8 + 8 * k;
      if (r < j) sm.Wk[r][cu] = fmaf(-trj[k], sj, cur[k]);
      else if (r == j) sm.Ui[j][cu] = sj;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kDThreads)
mxp_diag_kernel(DiagArgs a) {
  extern __shared__ __align__(16) unsigned char diag_smem_raw[];
  DiagSmem& sm = *reinterpret_cast<DiagSmem*>(diag_smem_raw);
  float* Zs = reinterpret_cast<float*>(diag_smem_raw + kZsOffset);  // [own][32]: z' or y'
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = gridDim.x, g = blockIdx.x;
  const int rg = g % kRG, cgi = g / kRG, CG = a.cg;
  const int jb = a.jb, nblk = (jb + kDB - 1) / kDB;
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
    __syncthreads();
    // (1) queue: the block row z of this CTA's columns and its chunks below the block
    for (int jj = warp; jj < nown; jj += kDThreads / 32) {
      const float* col = step_column(a, cgi + jj * CG, e);
      if (lane < w) cp_async4(&Zs[jj * kDB + lane], col + b + lane);
      else Zs[jj * kDB + lane] = 0.0f;
    }
    const int nq = queue_chunks(sm, a, rg, b, w, e, jb);
    // (2) the diagonal block (padded with the identity), factored and inverted
    for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
      const int r = idx & 31, c = idx >> 5;
      sm.T[r][c] = (r < w && c < w) ? a.D[b + r + (int64_t)(b + c) * a.ldd] : (r == c ? 1.0f : 0.0f);
    }
    __syncthreads();
    factor_and_invert(sm);
    cp_async_wait_all();
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
    // (3) z' = L_pp^-1 z in place (four columns per warp pass), and L = A U_pp^-1
    // for every chunk (four multipliers per lane)
    for (int jj0 = warp * 4; jj0 < nown; jj0 += 4 * (kDThreads / 32)) {
      float z[4], acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        z[u] = jj0 + u < nown ? Zs[(jj0 + u) * kDB + lane] : 0.0f;
        acc[u] = 0.0f;
      }
#pragma unroll
      for (int k = 0; k < kDB; ++k) {
        const float li = sm.Li[lane][k];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fmaf(li, __shfl_sync(0xffffffffu, z[u], k), acc[u]);
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (jj0 + u < nown) Zs[(jj0 + u) * kDB + lane] = acc[u];
    }
    for (int qk = warp; qk < nq * (kDB / 4); qk += kDThreads / 32) {
      const int qi = qk / (kDB / 4), k0 = (qk % (kDB / 4)) * 4;
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int m = 0; m < kDB; ++m) {
        const float av = sm.Ac[qi][m][lane];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fmaf(av, sm.Ui[m][k0 + u], acc[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) sm.Lr[qi][k0 + u][lane] = acc[u];
    }
    __syncthreads();
    // (4) the rank-32 update of this CTA's (row, column) pairs
    apply_updates<true>(sm, Zs, a, rg, cgi, nown, nq, b, e, e);
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
    __syncthreads();
    const float* s = a.sc + (int64_t)p * 2 * kDB * kDB;
    for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
      const int r = idx & 31, c = idx >> 5;
      cp_async4(&sm.Ui[r][c], s + kDB * kDB + c * kDB + r);
    }
    for (int jj = warp; jj < nown; jj += kDThreads / 32) {
      const int c = cgi + jj * CG;
      if (c >= b && lane < w) cp_async4(&Zs[jj * kDB + lane], a.Y + b + lane + (int64_t)c * a.ldy);
      else Zs[jj * kDB + lane] = 0.0f;
    }
    const int nq = queue_chunks(sm, a, rg, b, w, 0, b);  // U_r,p for the rows r < b
    cp_async_wait_all();
    __syncthreads();
    for (int jj0 = warp * 4; jj0 < nown; jj0 += 4 * (kDThreads / 32)) {  // y' = U_pp^-1 y
      float y[4], acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        y[u] = jj0 + u < nown ? Zs[(jj0 + u) * kDB + lane] : 0.0f;
        acc[u] = 0.0f;
      }
#pragma unroll
      for (int k = 0; k < kDB; ++k) {
        const float ui = sm.Ui[lane][k];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fmaf(ui, __shfl_sync(0xffffffffu, y[u], k), acc[u]);
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (jj0 + u < nown) Zs[(jj0 + u) * kDB + lane] = acc[u];
    }
    for (int qk = warp; qk < nq * kDB; qk += kDThreads / 32) {  // Lr[q][k][i] = U(r0 + i, b + k)
      const int qi = qk / kDB, k = qk % kDB;
      sm.Lr[qi][k][lane] = sm.Ac[qi][k][lane];
    }
    __syncthreads();
    apply_updates<false>(sm, Zs, a, rg, cgi, nown, nq, b, e, 0);
    if (cgi == p % CG) {  // column block p of L below the block, and the block itself
      if (rg == 0)
        for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
          const int r = idx & 31, c = idx >> 5;
          if (r < w && c < w) a.D[b + r + (int64_t)(b + c) * a.ldd] = s[c * kDB + r];
        }
      __syncthreads();
      const int nl = queue_chunks(sm, a, rg, b, w, e, jb);
      cp_async_wait_all();
      __syncthreads();
      for (int qk = warp; qk < nl * (kDB / 4); qk += kDThreads / 32) {
        const int qi = qk / (kDB / 4), k0 = (qk % (kDB / 4)) * 4;
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int m = 0; m < kDB; ++m) {
          const float av = sm.Ac[qi][m][lane];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] = fmaf(av, sm.Ui[m][k0 + u], acc[u]);
        }
        const int r = (first_chunk(rg, e) + qi * kRG) * 32 + lane;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (k0 + u < w && r < jb) a.D[r + (int64_t)(b + k0 + u) * a.ldd] = acc[u];
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
  if ((nown + 7) / 8 > kMaxCW) return set_error(HPL_ERR_NOTSUP, "mxp diagonal block: too few CTAs for %d columns", (int)jb);
  const size_t dyn = kZsOffset + (size_t)nown * kDB * sizeof(float);
  static bool attr = false;
  if (!attr) {
    HPL_CUDA(cudaFuncSetAttribute(mxp_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
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
