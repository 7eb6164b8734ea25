// mxp_diag.cu -- the diagonal block of a mixed-precision panel: unpivoted LU
// A11 = L11 U11 of the jb x jb block (FP32, in place) together with X = L11^-1
// and Y = U11^-1, so that the rest of the panel and the U12 block row become
// products on the tensor cores (L21 = A21 U11^-1, U12 = L11^-1 A12).
//
// One launch of G = kRG x CG work CTAs plus one diagonal CTA, cooperating,
// blocked by 32:
//  forward, p = 0 .. nblk-1 (b = 32p, w = min(32, jb - b), e = b + w):
//    the diagonal CTA has factored the diagonal block p during step p-1 and
//    published T = L_pp\U_pp, Li = L_pp^-1 and Ui = U_pp^-1; during step p it
//    applies step p's update to block p+1 (the work CTAs skip those entries),
//    factors it and publishes its T, Li, Ui before the barrier.  The columns
//    eliminated at step p are the trailing columns of A11 (c >= e) and the
//    columns of X that are already nonzero (c < e, X starts as I).  Column
//    group cg takes every CG-th of them and row group rg every kRG-th 32-row
//    chunk below the block:
//      z' = Li z for the block row of each of its columns (U_p,c, or X_p,c);
//      L_r = A_r U_pp^-1 for each of its rows;
//      col_r -= L_r z' for each of its (row, column) pairs;
//    then one grid barrier.
//    Two steps behind, the same CTAs build Y = U11^-1 by column blocks
//    (right-looking: Y_q = R_q U_qq^-1, then R_r -= Y_q U_qr), and at the
//    start of step p+1 they write back step p's block row of U, column block
//    of L and factored diagonal block.
// A value that other CTAs read during a step (the block row z, the column
// block A_r,p, the diagonal block) is written back only in the next step, so
// no CTA overwrites what another may still be reading.  Every barrier wait is
// bounded (~2 s, then DEV_TIMEOUT).
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
  int nwork;           // CTAs that own rows and columns; CTA nwork is the diagonal CTA
  float* D;            // jb x jb block, factored in place
  int64_t ldd;
  float* X;            // out: L11^-1 (jb x jb)
  int64_t ldx;
  float* Y;            // out: U11^-1 (jb x jb)
  int64_t ldy;
  float* sc;           // scratch [nblk][3][32 x 32]: factored diagonal block, L_pp^-1, U_pp^-1
  int32_t* info;
  int64_t info_shift;
  unsigned long long* bar;
  unsigned long long bar_base;
  int* err;
};

constexpr int kMaxChunks = 9;   // 32-row chunks per row group (jb <= 2048 = 8 x 8 x 32), plus one work slot

struct DiagSmem {
  float T[kDB][kDB + 1];                 // diagonal block: strict lower L_pp, upper U_pp
  float Li[kDB][kDB + 1];                // L_pp^-1
  float Ui[kDB][kDB + 1];                // U_pp^-1
  float Ac[kMaxChunks][kDB][kDB + 1];    // Ac[q][m][i] = D(r0_q + i, b + m)
  float Lr[kMaxChunks][kDB][kDB + 1];    // Lr[q][k][i] = L(r0_q + i, b + k), kept for the next step's write-back
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

// First chunk index q = rg (mod kRG) with 32 q >= first_row.
__device__ __forceinline__ int first_chunk(int rg, int first_row) {
  const int q0 = (first_row + 31) / 32;
  return q0 <= rg ? rg : rg + (q0 - rg + kRG - 1) / kRG * kRG;
}

constexpr int kMaxCW = 16;  // columns per warp: ceil(jb / cg / 8) <= 16 for jb <= 2048

// col_r -= sum_k Lr[q][k][r - r0_q] Z[jj][k] over this CTA's (chunk, column)
// pairs.  Warp w takes the columns jj = w, w + 8, ...; lane = row within the
// chunk.  Per chunk the lane's 32 multipliers sit in registers and Z is read
// as float4 broadcasts; the next chunk's column entries are loaded while the
// current one is computed.  The entries of the next diagonal block are skipped:
// the diagonal CTA updates them.
__device__ __forceinline__ void apply_updates(DiagSmem& sm, const float* Zs, const DiagArgs& a, int rg, int cgi,
                                              int nown, int nq, int e) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qf = first_chunk(rg, e);
  float* cols[kMaxCW];
  unsigned skip = 0;  // columns of the next diagonal block
#pragma unroll
  for (int u = 0; u < kMaxCW; ++u) {
    const int jj = warp + 8 * u;
    const int c = cgi + jj * a.cg;
    cols[u] = jj < nown ? step_column(a, c, e) : nullptr;
    if (c >= e && c < e + kDB) skip |= 1u << u;
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
    const int r0 = (qf + qi * kRG) * 32, r = r0 + lane;
    const unsigned skip_q = r0 == e ? skip : 0u;
#pragma unroll
    for (int u = 0; u < kMaxCW; ++u) {
      if (!cols[u] || r >= a.jb || ((skip_q >> u) & 1u)) continue;
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

// One LU step on the live part of a row: a[0] holds column j, a[1..W-1]
// columns j+1.., the rest are zero.  Stores the multiplier (below the
// diagonal; the unscaled entry for a zero pivot) or the U entry to T, updates
// and shifts the row left by one column.
template <int W>
__device__ __forceinline__ void lu_step(float (&a)[kDB], DiagSmem& sm, int lane, int j) {
  const float piv = __shfl_sync(0xffffffffu, a[0], j);
  const float rcp = piv != 0.0f ? 1.0f / piv : 0.0f;
  const bool below = lane > j;
  const float l = below ? a[0] * rcp : 0.0f;
  sm.T[lane][j] = (below && piv != 0.0f) ? l : a[0];
#pragma unroll
  for (int c = 1; c < W; ++c) a[c - 1] = fmaf(-l, __shfl_sync(0xffffffffu, a[c], j), a[c]);
  a[W - 1] = 0.0f;
}

// One forward-elimination step of [L | I]: row j of L^-1 is nonzero only in
// columns < W.
template <int W>
__device__ __forceinline__ void linv_step(float (&e)[kDB], float lij, int j) {
#pragma unroll
  for (int c = 0; c < W; ++c) e[c] = fmaf(-lij, __shfl_sync(0xffffffffu, e[c], j), e[c]);
}

// One back-substitution step of [U | I]: row j of U^-1 is nonzero only in
// columns >= 32 - W.
template <int W>
__device__ __forceinline__ void uinv_step(float (&w)[kDB], float uij, float rj, int lane, int j) {
#pragma unroll
  for (int c = kDB - W; c < kDB; ++c) {
    const float sj = __shfl_sync(0xffffffffu, w[c], j) * rj;  // U^-1(j, c)
    w[c] = lane == j ? sj : fmaf(-uij, sj, w[c]);
  }
}

// T (32 x 32, padded with the identity) -> packed L\U in T, Li = L^-1 and
// Ui = U^-1.  Warp 0 factors T in registers: lane i keeps the live columns
// of row i, shifted left one column per step, so the pivot column is always
// a[0] and every register index is static (a zero pivot leaves its column as
// it is: no multipliers, no update).  Then warp 0 forms U^-1 by back
// substitution on the rows of [U | I] while warp 1 forms L^-1 by forward
// elimination of [L | I].  Each sweep runs in four phases of eight steps over
// the 32, 24, 16 or 8 columns that can still be nonzero.  The step loops stay
// rolled: while this runs the other CTAs keep L2 busy, and fully unrolled
// versions, larger than the instruction cache, ran 1.7 times slower.
__device__ __forceinline__ void factor_and_invert(DiagSmem& sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    float a[kDB];
#pragma unroll
    for (int c = 0; c < kDB; ++c) a[c] = sm.T[lane][c];
#pragma unroll 1
    for (int j = 0; j < 8; ++j) lu_step<32>(a, sm, lane, j);
#pragma unroll 1
    for (int j = 8; j < 16; ++j) lu_step<24>(a, sm, lane, j);
#pragma unroll 1
    for (int j = 16; j < 24; ++j) lu_step<16>(a, sm, lane, j);
#pragma unroll 1
    for (int j = 24; j < 32; ++j) lu_step<8>(a, sm, lane, j);
  }
  __syncthreads();
  if (warp == 0) {  // U^-1: w = row `lane` of the right half of [U | I]
    float w[kDB];
#pragma unroll
    for (int c = 0; c < kDB; ++c) w[c] = lane == c ? 1.0f : 0.0f;
    const float rd = 1.0f / sm.T[lane][lane];  // all reciprocals of the diagonal at once
#pragma unroll 1
    for (int j = kDB - 1; j >= 0; --j) {
      const float rj = __shfl_sync(0xffffffffu, rd, j);
      const float uij = lane < j ? sm.T[lane][j] : 0.0f;  // U(lane, j)
      if (j >= 24) uinv_step<8>(w, uij, rj, lane, j);
      else if (j >= 16) uinv_step<16>(w, uij, rj, lane, j);
      else if (j >= 8) uinv_step<24>(w, uij, rj, lane, j);
      else uinv_step<32>(w, uij, rj, lane, j);
    }
#pragma unroll
    for (int c = 0; c < kDB; ++c) sm.Ui[lane][c] = w[c];
  } else if (warp == 1) {  // L^-1: e = row `lane` of the right half of [L | I]
    float e[kDB];
#pragma unroll
    for (int c = 0; c < kDB; ++c) e[c] = lane == c ? 1.0f : 0.0f;
#pragma unroll 1
    for (int j = 0; j < kDB; ++j) {
      const float lij = lane > j ? sm.T[lane][j] : 0.0f;  // L(lane, j)
      if (j < 8) linv_step<8>(e, lij, j);
      else if (j < 16) linv_step<16>(e, lij, j);
      else if (j < 24) linv_step<24>(e, lij, j);
      else linv_step<32>(e, lij, j);
    }
#pragma unroll
    for (int c = 0; c < kDB; ++c) sm.Li[lane][c] = e[c];
  }
}

// Writes that were deferred from step pp (b = 32 pp, width w, e = b + w) to
// the start of the next step, when no CTA reads those entries any more: the
// block row z' of this CTA's columns (row group 0), the column block pp of L
// below the block from sm.Lr (column group pp % CG, nq chunks) and the
// factored diagonal block from the scratch (row group 0 of that column group).
__device__ __forceinline__ void deferred_writes(const DiagSmem& sm, const float* Zs, const DiagArgs& a, int rg,
                                                int cgi, int nown, int pp, int nq) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = pp * kDB, w = min(kDB, a.jb - b), e = b + w;
  if (rg == 0)
    for (int jj = warp; jj < nown; jj += kDThreads / 32) {
      float* col = step_column(a, cgi + jj * a.cg, e);
      if (lane < w) col[b + lane] = Zs[jj * kDB + lane];
    }
  if (cgi == pp % a.cg) {
    const int qf = first_chunk(rg, e);
    for (int qk = warp; qk < nq * kDB; qk += kDThreads / 32) {
      const int qi = qk / kDB, k = qk % kDB;
      const int r = (qf + qi * kRG) * 32 + lane;
      if (k < w && r < a.jb) a.D[r + (int64_t)(b + k) * a.ldd] = sm.Lr[qi][k][lane];
    }
    if (rg == 0) {
      const float* s = a.sc + (int64_t)pp * 3 * kDB * kDB;
      for (int idx = threadIdx.x; idx < kDB * kDB; idx += kDThreads) {
        const int r = idx & 31, c = idx >> 5;
        if (r < w && c < w) a.D[b + r + (int64_t)(b + c) * a.ldd] = s[c * kDB + r];
      }
    }
  }
}

// Y = U11^-1 by column blocks, right-looking, two forward steps behind:
// Y_q = R_q U_qq^-1 once R_q (starting as I) has every update from the
// blocks before it, and R_r -= Y_q U_qr for r > q.  Column block r of Y
// belongs to column group r % CG, its rows to their row groups.  At step s:
//   (Y1) R_r -= Y_q U_qr for q = s - 2 and this CTA's blocks r > q, rows
//        < e_q (Y_q was finished at step s-1, the block row q of U written
//        back at step q + 1 = s - 1);
//   (Y2) Y_q2 = R_q2 U_q2q2^-1 for q2 = s - 1 if this CTA owns it (after its
//        own (Y1) update of that block; U_q2q2^-1 is in the scratch).
// Uses sm.Ac as work space.
__device__ void y_step(DiagSmem& sm, const DiagArgs& a, int rg, int cgi, int s, int nblk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int jb = a.jb, CG = a.cg;
  const int q = s - 2, q2 = s - 1;
  if (q >= 0) {
    const int bq = q * kDB, wq = min(kDB, jb - bq), eq = bq + wq;
    const int r1 = q + 1 + ((cgi - (q + 1)) % CG + CG) % CG;  // this CTA's first block after q
    int nc = 0;  // this row group's chunks above e_q: Ys[1 + c][k][i] = Y(r0_c + i, bq + k), loaded once
    for (int qq = rg; qq * 32 < eq && r1 < nblk; qq += kRG, ++nc) {
      for (int idx = threadIdx.x; idx < kDB * kDB; idx += kDThreads) {
        const int i = idx & 31, k = idx >> 5;
        if (k < wq) cp_async4(&sm.Ac[1 + nc][k][i], a.Y + qq * 32 + i + (int64_t)(bq + k) * a.ldy);
        else sm.Ac[1 + nc][k][i] = 0.0f;
      }
    }
    for (int r = r1; r < nblk && nc > 0; r += CG) {
      const int br = r * kDB, wr = min(kDB, jb - br);
      for (int idx = threadIdx.x; idx < kDB * kDB; idx += kDThreads) {  // Us[k][c] = U(bq + k, br + c)
        const int k = idx & 31, c = idx >> 5;
        if (k < wq && c < wr) cp_async4(&sm.Ac[0][k][c], a.D + bq + k + (int64_t)(br + c) * a.ldd);
        else sm.Ac[0][k][c] = 0.0f;
      }
      cp_async_wait_all();
      __syncthreads();
      for (int ci = 0; ci < nc; ++ci) {
        const int row = (rg + ci * kRG) * 32 + lane;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = warp * 4 + u;
          if (c < wr && row < jb) {
            float* dst = a.Y + row + (int64_t)(br + c) * a.ldy;
            float acc = *dst;
#pragma unroll
            for (int k = 0; k < kDB; ++k) acc = fmaf(-sm.Ac[1 + ci][k][lane], sm.Ac[0][k][c], acc);
            *dst = acc;
          }
        }
      }
      __syncthreads();
    }
  }
  if (q2 >= 0 && q2 % CG == cgi) {
    const int b2 = q2 * kDB, w2 = min(kDB, jb - b2), e2 = b2 + w2;
    const float* sui = a.sc + (int64_t)q2 * 3 * kDB * kDB + 2 * kDB * kDB;
    for (int idx = threadIdx.x; idx < kDB * kDB; idx += kDThreads) {  // Ui[m][c] = U_q2q2^-1(m, c)
      const int m = idx & 31, c = idx >> 5;
      sm.Ac[2][m][c] = sui[c * kDB + m];
    }
    for (int qq = rg; qq * 32 < e2; qq += kRG) {
      const int r0 = qq * 32;
      for (int idx = threadIdx.x; idx < kDB * kDB; idx += kDThreads) {  // Rs[m][i] = R(r0 + i, b2 + m)
        const int i = idx & 31, m = idx >> 5;
        sm.Ac[3][m][i] = (m < w2) ? a.Y[r0 + i + (int64_t)(b2 + m) * a.ldy] : 0.0f;
      }
      __syncthreads();
      const int i = lane, row = r0 + i;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = warp * 4 + u;
        if (c < w2 && row < jb) {
          float acc = 0.0f;
#pragma unroll
          for (int m = 0; m < kDB; ++m) acc = fmaf(sm.Ac[3][m][i], sm.Ac[2][m][c], acc);
          a.Y[row + (int64_t)(b2 + c) * a.ldy] = acc;
        }
      }
      __syncthreads();
    }
  }
}

// The diagonal CTA's results for step p: scratch slot p = {packed L\U, L^-1,
// U^-1} (column-major 32 x 32 each), read by the work CTAs after the next
// barrier; the first zero pivot of the block goes to info.
__device__ __forceinline__ void publish_block(const DiagSmem& sm, const DiagArgs& a, int p, int w) {
  float* s = a.sc + (int64_t)p * 3 * kDB * kDB;
  for (int idx = threadIdx.x; idx < kDB * kDB; idx += kDThreads) {
    const int r = idx & 31, c = idx >> 5;
    s[c * kDB + r] = sm.T[r][c];
    s[kDB * kDB + c * kDB + r] = sm.Li[r][c];
    s[2 * kDB * kDB + c * kDB + r] = sm.Ui[r][c];
  }
  if (threadIdx.x == 0 && a.info)
    for (int j = 0; j < w; ++j)
      if (sm.T[j][j] == 0.0f) {
        atomicCAS(a.info, 0, (int32_t)(a.info_shift + p * kDB + j + 1));
        break;
      }
}

__global__ void __launch_bounds__(kDThreads)
mxp_diag_kernel(DiagArgs a) {
  extern __shared__ __align__(16) unsigned char diag_smem_raw[];
  DiagSmem& sm = *reinterpret_cast<DiagSmem*>(diag_smem_raw);
  float* Zs = reinterpret_cast<float*>(diag_smem_raw + kZsOffset);  // [own][32]: z' or y'
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = gridDim.x, g = blockIdx.x;
  const bool diag_cta = g == a.nwork;
  const int rg = g % kRG, cgi = g / kRG, CG = a.cg;
  const int jb = a.jb, nblk = (jb + kDB - 1) / kDB;
  const int nown = (!diag_cta && cgi < jb) ? (jb - cgi + CG - 1) / CG : 0;  // columns v = cgi + jj CG < jb
  unsigned long long target = a.bar_base;

  // X = Y = I; the diagonal CTA factors block 0
  for (int64_t idx = (int64_t)g * kDThreads + t; idx < (int64_t)jb * jb; idx += (int64_t)G * kDThreads) {
    const int i = (int)(idx % jb), j = (int)(idx / jb);
    a.X[i + (int64_t)j * a.ldx] = i == j ? 1.0f : 0.0f;
    a.Y[i + (int64_t)j * a.ldy] = i == j ? 1.0f : 0.0f;
  }
  if (diag_cta) {
    const int w0 = min(kDB, jb);
    for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
      const int r = idx & 31, c = idx >> 5;
      sm.T[r][c] = (r < w0 && c < w0) ? a.D[r + (int64_t)c * a.ldd] : (r == c ? 1.0f : 0.0f);
    }
    __syncthreads();
    factor_and_invert(sm);
    __syncthreads();
    publish_block(sm, a, 0, w0);
  }
  target += G;
  if (!diag_barrier(a.bar, target, a.err, &sm.flag)) return;

  int prev_nq = 0;  // chunks of L held in sm.Lr from the previous step
  for (int p = 0; p < nblk; ++p) {
    const int b = p * kDB, w = min(kDB, jb - b), e = b + w;
    if (diag_cta) {
      // step p+1's diagonal block: apply step p's rank-32 update to it (the
      // work CTAs skip those entries) with the same operation order, factor
      // it and publish T, L^-1, U^-1; sm.Li / sm.Ui hold step p's
      if (e < jb) {
        const int w1 = min(kDB, jb - e);
        for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
          const int i = idx & 31, m = idx >> 5;
          if (i < w1 && m < w) cp_async4(&sm.Ac[0][m][i], a.D + e + i + (int64_t)(b + m) * a.ldd);  // A(e+i, b+m)
          else sm.Ac[0][m][i] = 0.0f;
          if (m < w && i < w1) cp_async4(&sm.Ac[1][m][i], a.D + b + m + (int64_t)(e + i) * a.ldd);  // z_i(m)
          else sm.Ac[1][m][i] = 0.0f;
          if (i < w1 && m < w1) cp_async4(&sm.T[i][m], a.D + e + i + (int64_t)(e + m) * a.ldd);
          else sm.T[i][m] = i == m ? 1.0f : 0.0f;
        }
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = warp * 4 + u;
          float accl = 0.0f, accz = 0.0f;
#pragma unroll
          for (int m = 0; m < kDB; ++m) {
            accl = fmaf(sm.Ac[0][m][lane], sm.Ui[m][k], accl);  // L(e+lane, b+k)
            accz = fmaf(sm.Li[k][m], sm.Ac[1][m][lane], accz);  // z'_lane(k) = U(b+k, e+lane)
          }
          sm.Lr[0][k][lane] = accl;
          sm.Lr[1][k][lane] = accz;
        }
        __syncthreads();
        for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
          const int i = idx & 31, c = idx >> 5;
          if (i < w1 && c < w1) {
            float acc = sm.T[i][c];
#pragma unroll
            for (int k = 0; k < kDB; ++k) acc = fmaf(-sm.Lr[0][k][i], sm.Lr[1][k][c], acc);
            sm.T[i][c] = acc;
          }
        }
        __syncthreads();
        factor_and_invert(sm);
        __syncthreads();
        publish_block(sm, a, p + 1, w1);
      }
      target += G;
      if (!diag_barrier(a.bar, target, a.err, &sm.flag)) return;
      continue;
    }
    // the previous step's block row, L column block and diagonal block, now
    // that no CTA reads them
    if (p > 0) deferred_writes(sm, Zs, a, rg, cgi, nown, p - 1, prev_nq);
    __syncthreads();
    // (1) queue: L_pp^-1 and U_pp^-1 from the diagonal CTA, the block row z of
    // this CTA's columns and its chunks below the block
    {
      const float* s = a.sc + (int64_t)p * 3 * kDB * kDB;
      for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
        const int r = idx & 31, c = idx >> 5;
        cp_async4(&sm.Li[r][c], s + kDB * kDB + c * kDB + r);
        cp_async4(&sm.Ui[r][c], s + 2 * kDB * kDB + c * kDB + r);
      }
    }
    for (int jj = warp; jj < nown; jj += kDThreads / 32) {
      const float* col = step_column(a, cgi + jj * CG, e);
      if (lane < w) cp_async4(&Zs[jj * kDB + lane], col + b + lane);
      else Zs[jj * kDB + lane] = 0.0f;
    }
    const int nq = queue_chunks(sm, a, rg, b, w, e, jb);
    cp_async_wait_all();
    __syncthreads();
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
    apply_updates(sm, Zs, a, rg, cgi, nown, nq, e);
    __syncthreads();
    // (5) two steps behind: U11^-1
    y_step(sm, a, rg, cgi, p, nblk);
    prev_nq = nq;
    target += G;
    if (!diag_barrier(a.bar, target, a.err, &sm.flag)) return;
  }
  if (!diag_cta) deferred_writes(sm, Zs, a, rg, cgi, nown, nblk - 1, prev_nq);
  target += G;
  if (!diag_barrier(a.bar, target, a.err, &sm.flag)) return;
  if (!diag_cta) y_step(sm, a, rg, cgi, nblk, nblk);  // the last column block of U11^-1

}

}  // namespace

int diag_scratch_floats(int64_t jb) { return (int)(((jb + kDB - 1) / kDB) * 3 * kDB * kDB); }

// Factor the jb x jb block D (ldd) in place and write X = L^-1, Y = U^-1
// (jb x jb, leading dimension jb).  jb <= 2048; sc holds
// diag_scratch_floats(jb) floats.
int launch_mxp_diag(Workspace* ws, int64_t jb, float* D, int64_t ldd, float* X, float* Y, float* sc, int32_t* info,
                    int64_t info_shift, cudaStream_t s) {
  if (jb <= 0) return HPL_OK;
  if (jb > 2048) return set_error(HPL_ERR_NOTSUP, "mxp diagonal block larger than 2048");
  int cg = (int)(jb / 64);
  if (cg < 1) cg = 1;
  if (cg > 18) cg = 18;  // 145 CTAs at most, one per SM
  while (kRG * cg + 1 > ws->num_sms && cg > 1) --cg;
  const int G = kRG * cg + 1;  // work CTAs and the diagonal CTA
  const int nown = (int)((jb + cg - 1) / cg);
  if ((nown + 7) / 8 > kMaxCW) return set_error(HPL_ERR_NOTSUP, "mxp diagonal block: too few CTAs for %d columns", (int)jb);
  // more than half of an SM's shared memory, so that no two CTAs share an SM:
  // the diagonal CTA's serial chain is the critical path of every step, and a
  // work CTA beside it would take its issue slots
  size_t dyn = kZsOffset + (size_t)nown * kDB * sizeof(float);
  if (dyn < 120 * 1024) dyn = 120 * 1024;
  static bool attr = false;
  if (!attr) {
    HPL_CUDA(cudaFuncSetAttribute(mxp_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    attr = true;
  }
  DiagArgs a;
  a.jb = (int)jb;
  a.cg = cg;
  a.nwork = G - 1;
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
  ws->bar_next += (unsigned long long)G * (unsigned long long)(2 + nblk);
  mxp_diag_kernel<<<G, kDThreads, dyn, s>>>(a);
  count_launch();
  return check_launch("mxp_diag_kernel");
}

}  // namespace hplgb
