// mxp_diag.cu -- the diagonal block of a mixed-precision panel: unpivoted LU
// A11 = L11 U11 of the jb x jb block (FP32, in place).  Its inverses, which
// turn the rest of the panel and the U12 block row into products on the
// tensor cores, follow in mxp_trinv.cu.
//
// One launch of G = kRG x CG work CTAs plus one diagonal CTA, cooperating,
// blocked by 32:
//  forward, p = 0 .. nblk-1 (b = 32p, w = min(32, jb - b), e = b + w):
//    the diagonal CTA has factored the diagonal block p during step p-1 and
//    published it, T = L_pp\U_pp; during step p it applies step p's update
//    to block p+1 (the work CTAs skip those entries), factors it and
//    publishes it before the barrier.  Column group cg takes every CG-th
//    trailing column (c >= e) and row group rg every kRG-th 32-row chunk
//    below the block:
//      z' = L_pp^-1 z for the block row U_p,c of each of its columns
//         (forward substitution, one column per lane);
//      L_r = A_r U_pp^-1 for each of its rows (substitution along the row,
//         one row per lane);
//      col_r -= L_r z' for each of its (row, column) pairs;
//    then one grid barrier.  At the start of step p+1 the same CTAs write back
//    step p's block row of U, column block of L and factored diagonal block.
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
  float* sc;           // scratch [nblk][kSlot]: the factored diagonal blocks
  int32_t* info;
  int64_t info_shift;
  unsigned long long* bar;
  unsigned long long bar_base;
  int* err;
};

constexpr int kMaxChunks = 8;   // 32-row chunks per row group (jb <= 2048 = 8 x 8 x 32)

constexpr int kSS = 36;  // row stride of Us / Ls: 16-byte aligned rows
// Scratch slot of a factored diagonal block: packed L\U (column-major), then
// its Us, Ls (32 x 32, row-major) and Ud (32) as below.
constexpr int kSlot = 3 * kDB * kDB + kDB;

struct DiagSmem {
  float T[kDB][kDB + 1];                 // the diagonal block being factored (diagonal CTA)
  // the factored block p, shifted for the substitutions (zero past the block):
  float Us[kDB][kSS];                    // Us[k][c] = U(k, k + 1 + c)
  float Ls[kDB][kSS];                    // Ls[k][c] = L(k + 1 + c, k)
  float Ud[kDB];                         // U(k, k)
  float R[2][kDB];                       // pivot rows of the LU (diagonal CTA)
  float Ac[kMaxChunks][kDB][kDB + 1];    // Ac[q][m][i] = D(r0_q + i, b + m)
  float Lr[kMaxChunks][kDB][kDB + 1];    // Lr[q][k][i] = L(r0_q + i, b + k), kept for the next step's write-back
  int flag;
};
// Zs[jj][kZS] (read as float4) follows DiagSmem at a 16-byte aligned offset;
// the stride of 36 keeps float4 accesses down a column conflict-free.
constexpr size_t kZsOffset = (sizeof(DiagSmem) + 15) / 16 * 16;
constexpr int kZS = 36;

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// This CTA's first column index jj (column v = cgi + jj CG) with v >= e.
__device__ __forceinline__ int first_live(int cgi, int cg, int e) { return cgi >= e ? 0 : (e - cgi + cg - 1) / cg; }

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

// The CTA's entries of the trailing block for this step, Cs[(qi nown + jj)
// 32 + i] = D(r0_qi + i, column jj), copied in with the step's other operands
// (16-byte pieces where the rows are aligned, zero past the block's rows), so
// that the update below reads them from shared memory, all requests in flight
// at once.
__device__ __forceinline__ void stage_trailing(float* Cs, const DiagArgs& a, int rg, int cgi, int nown, int nq, int e) {
  const int qf = first_chunk(rg, e), jl = first_live(cgi, a.cg, e), nlive = nown - jl;
  if (nlive <= 0 || nq <= 0) return;
  const bool vec = ((a.ldd & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.D) & 15) == 0);
  for (int idx = threadIdx.x; idx < nq * nlive * 8; idx += kDThreads) {
    const int piece = idx & 7, pair = idx >> 3;
    const int qi = pair / nlive, jj = jl + pair % nlive;
    const int r = (qf + qi * kRG) * 32 + 4 * piece;
    const float* src = a.D + r + (int64_t)(cgi + jj * a.cg) * a.ldd;
    float* dst = Cs + ((qi * nown + jj) * kDB + 4 * piece);
    if (vec && r + 4 <= a.jb) {
      cp_async16(dst, src);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (r + i < a.jb) cp_async4(dst + i, src + i);
        else dst[i] = 0.0f;
      }
    }
  }
}

// col_r -= sum_k Lr[q][k][r - r0_q] Z[jj][k] over this CTA's (chunk, column)
// pairs.  Warp w takes the live columns jj = jl + w, jl + w + 8, ...; lane =
// row within the chunk.  Per chunk the lane's 32 multipliers sit in registers,
// Z is read as float4 broadcasts and the old entry from Cs; the result goes
// straight to D.  The entries of the next diagonal block are skipped: the
// diagonal CTA updates them.
__device__ __forceinline__ void apply_updates(DiagSmem& sm, const float* Zs, const float* Cs, const DiagArgs& a,
                                              int rg, int cgi, int nown, int nq, int e) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qf = first_chunk(rg, e), jl = first_live(cgi, a.cg, e);
  float* cols[kMaxCW];
  unsigned skip = 0;  // columns of the next diagonal block
#pragma unroll
  for (int u = 0; u < kMaxCW; ++u) {
    const int jj = jl + warp + 8 * u;
    const int c = cgi + jj * a.cg;
    cols[u] = jj < nown ? a.D + (int64_t)c * a.ldd : nullptr;
    if (c < e + kDB) skip |= 1u << u;
  }
  for (int qi = 0; qi < nq; ++qi) {
    float lr[kDB];
#pragma unroll
    for (int k = 0; k < kDB; ++k) lr[k] = sm.Lr[qi][k][lane];
    const int r0 = (qf + qi * kRG) * 32, r = r0 + lane;
    const unsigned skip_q = r0 == e ? skip : 0u;
#pragma unroll
    for (int u = 0; u < kMaxCW; ++u) {
      if (!cols[u] || r >= a.jb || ((skip_q >> u) & 1u)) continue;
      const int jj = jl + warp + 8 * u;
      const float4* z4 = reinterpret_cast<const float4*>(Zs + jj * kZS);
      float acc = Cs[(qi * nown + jj) * kDB + lane];
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
  }
}

// One LU step on the live part of a row: a[0] holds column j, a[1..W-1]
// columns j+1.., the rest are zero.  Lane j publishes its row (the pivot
// row) in sm.R[j & 1] as float4s and every lane reads it back, which costs
// fewer instructions than one shuffle per column.  Stores the multiplier
// (below the diagonal; the unscaled entry for a zero pivot) or the U entry to
// T, updates and shifts the row left by one column.
template <int W>
__device__ __forceinline__ void lu_step(float (&a)[kDB], DiagSmem& sm, int lane, int j) {
  float* R = sm.R[j & 1];  // two buffers: one __syncwarp per step
  if (lane == j) {
#pragma unroll
    for (int c4 = 0; c4 < W / 4; ++c4)
      *reinterpret_cast<float4*>(R + 4 * c4) = make_float4(a[4 * c4], a[4 * c4 + 1], a[4 * c4 + 2], a[4 * c4 + 3]);
  }
  __syncwarp();
  float r[W];
#pragma unroll
  for (int c4 = 0; c4 < W / 4; ++c4) {
    const float4 q = *reinterpret_cast<const float4*>(R + 4 * c4);
    r[4 * c4] = q.x, r[4 * c4 + 1] = q.y, r[4 * c4 + 2] = q.z, r[4 * c4 + 3] = q.w;
  }
  const float piv = r[0];
  const float rcp = piv != 0.0f ? 1.0f / piv : 0.0f;
  const bool below = lane > j;
  const float l = below ? a[0] * rcp : 0.0f;
  sm.T[lane][j] = (below && piv != 0.0f) ? l : a[0];
#pragma unroll
  for (int c = 1; c < W; ++c) a[c - 1] = fmaf(-l, r[c], a[c]);
  a[W - 1] = 0.0f;
}

// T (32 x 32, padded with the identity) -> packed L\U in place, on warp 0:
// lane i keeps the live columns of row i, shifted left one column per step,
// so the pivot column is always a[0] and every register index is static (a
// zero pivot leaves its column as it is: no multipliers, no update).  The
// sweep runs in four phases of eight steps over the 32, 24, 16 or 8 columns
// that can still be nonzero.  The step loops stay rolled: while this runs
// the other CTAs keep L2 busy, and fully unrolled versions, larger than the
// instruction cache, ran 1.7 times slower.
__device__ __forceinline__ void lu_factor(DiagSmem& sm) {
  const int lane = threadIdx.x & 31;
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

// Substitutions with the factored block, one vector per lane, in the same
// shifted form: at step k, v[c] holds entry k + c, so entry k is v[0]; the
// multipliers of step k are row k of Ls or Us (entries past the block are
// zero there).
//   forward, z <- L^-1 z (column z):   z_k final, then z_c -= L(c, k) z_k
//   along a row, x <- x U^-1 (row x):  x_k = x_k / U(k, k), then x_c -= x_k U(k, c)
// Entry k of the result goes to out[k * os].  The multipliers of the next
// step are loaded (float4) while this one computes.
template <int W, bool UPPER>
__device__ __forceinline__ void load_mult(float (&mm)[W], const DiagSmem& sm, int k) {
  const float4* m4 = reinterpret_cast<const float4*>(UPPER ? &sm.Us[k][0] : &sm.Ls[k][0]);
#pragma unroll
  for (int c4 = 0; c4 < W / 4; ++c4) {
    const float4 m = m4[c4];
    mm[4 * c4] = m.x, mm[4 * c4 + 1] = m.y, mm[4 * c4 + 2] = m.z, mm[4 * c4 + 3] = m.w;
  }
}
template <int W, bool UPPER>
__device__ __forceinline__ float solve_step(float (&v)[kDB], const float (&mm)[W], float rk) {
  const float vk = UPPER ? v[0] * rk : v[0];
#pragma unroll
  for (int c = 1; c < W; ++c) v[c - 1] = fmaf(-vk, mm[c - 1], v[c]);  // v[c - 1] <- entry k + c
  v[W - 1] = 0.0f;
  return vk;
}
// Steps k0 .. k0 + 7 with W live entries, two per iteration (ping-pong).
template <int W, bool UPPER>
__device__ __forceinline__ void solve_phase(float (&v)[kDB], const DiagSmem& sm, int k0, float rd, float* out, int os) {
  float ma[W], mb[W];
  load_mult<W, UPPER>(ma, sm, k0);
#pragma unroll 1
  for (int k = k0; k < k0 + 8; k += 2) {
    load_mult<W, UPPER>(mb, sm, k + 1);
    const float x0 = solve_step<W, UPPER>(v, ma, UPPER ? __shfl_sync(0xffffffffu, rd, k) : 0.0f);
    out[k * os] = x0;
    load_mult<W, UPPER>(ma, sm, k + 2 < kDB ? k + 2 : k + 1);
    const float x1 = solve_step<W, UPPER>(v, mb, UPPER ? __shfl_sync(0xffffffffu, rd, k + 1) : 0.0f);
    out[(k + 1) * os] = x1;
  }
}
// rd = 1 / U(lane, lane), shuffled to step k (UPPER only).
template <bool UPPER>
__device__ __forceinline__ void solve(float (&v)[kDB], const DiagSmem& sm, float rd, float* out, int os) {
  solve_phase<32, UPPER>(v, sm, 0, rd, out, os);
  solve_phase<24, UPPER>(v, sm, 8, rd, out, os);
  solve_phase<16, UPPER>(v, sm, 16, rd, out, os);
  solve_phase<8, UPPER>(v, sm, 24, rd, out, os);
}
__device__ __forceinline__ void lsolve(float (&v)[kDB], const DiagSmem& sm, float* out, int os) {
  solve<false>(v, sm, 0.0f, out, os);
}
// L rows of chunk qi: row `lane` of Ac[qi] times U_pp^-1 into Lr[qi][.][lane].
__device__ __forceinline__ void row_solve(DiagSmem& sm, int qi) {
  const int lane = threadIdx.x & 31;
  float v[kDB];
#pragma unroll
  for (int m = 0; m < kDB; ++m) v[m] = sm.Ac[qi][m][lane];
  solve<true>(v, sm, 1.0f / sm.Ud[lane], &sm.Lr[qi][0][lane], kDB + 1);
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
    for (int jj = first_live(cgi, a.cg, e) + warp; jj < nown; jj += kDThreads / 32) {
      float* col = a.D + (int64_t)(cgi + jj * a.cg) * a.ldd;
      if (lane < w) col[b + lane] = Zs[jj * kZS + lane];
    }
  if (cgi == pp % a.cg) {
    const int qf = first_chunk(rg, e);
    for (int qk = warp; qk < nq * kDB; qk += kDThreads / 32) {
      const int qi = qk / kDB, k = qk % kDB;
      const int r = (qf + qi * kRG) * 32 + lane;
      if (k < w && r < a.jb) a.D[r + (int64_t)(b + k) * a.ldd] = sm.Lr[qi][k][lane];
    }
    if (rg == 0) {
      const float* s = a.sc + (int64_t)pp * kSlot;
      for (int idx = threadIdx.x; idx < kDB * kDB; idx += kDThreads) {
        const int r = idx & 31, c = idx >> 5;
        if (r < w && c < w) a.D[b + r + (int64_t)(b + c) * a.ldd] = s[c * kDB + r];
      }
    }
  }
}

// The diagonal CTA's result for step p: scratch slot p = {packed L\U
// (column-major), Us, Ls, Ud}, read by the work CTAs after the next barrier,
// and Us, Ls, Ud in its own shared memory for its next step; the first zero
// pivot of the block goes to info.
__device__ __forceinline__ void publish_block(DiagSmem& sm, const DiagArgs& a, int p, int w) {
  float* s = a.sc + (int64_t)p * kSlot;
  for (int idx = threadIdx.x; idx < kDB * kDB; idx += kDThreads) {
    const int r = idx & 31, c = idx >> 5;
    s[c * kDB + r] = sm.T[r][c];
    // row-major shifted copies: idx = k * 32 + c
    const int k = idx >> 5, cc = idx & 31, o = k + 1 + cc;
    const float u = o < kDB ? sm.T[k][o] : 0.0f;
    const float l = o < kDB ? sm.T[o][k] : 0.0f;
    sm.Us[k][cc] = u;
    sm.Ls[k][cc] = l;
    s[kDB * kDB + idx] = u;
    s[2 * kDB * kDB + idx] = l;
  }
  if (threadIdx.x < kDB) {
    const float d = sm.T[threadIdx.x][threadIdx.x];
    sm.Ud[threadIdx.x] = d;
    s[3 * kDB * kDB + threadIdx.x] = d;
    const unsigned zero = __ballot_sync(0xffffffffu, (int)threadIdx.x < w && d == 0.0f);
    if (threadIdx.x == 0 && zero && a.info)
      atomicCAS(a.info, 0, (int32_t)(a.info_shift + p * kDB + __ffs(zero)));
  }
}

__global__ void __launch_bounds__(kDThreads)
mxp_diag_kernel(DiagArgs a) {
  extern __shared__ __align__(16) unsigned char diag_smem_raw[];
  DiagSmem& sm = *reinterpret_cast<DiagSmem*>(diag_smem_raw);
  float* Zs = reinterpret_cast<float*>(diag_smem_raw + kZsOffset);  // [own][kZS]: z, then z'
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = gridDim.x, g = blockIdx.x;
  const bool diag_cta = g == a.nwork;
  const int rg = g % kRG, cgi = g / kRG, CG = a.cg;
  const int jb = a.jb, nblk = (jb + kDB - 1) / kDB;
  const int nown = (!diag_cta && cgi < jb) ? (jb - cgi + CG - 1) / CG : 0;  // columns v = cgi + jj CG < jb
  unsigned long long target = a.bar_base;

  // the diagonal CTA factors block 0
  if (diag_cta) {
    const int w0 = min(kDB, jb);
    for (int idx = t; idx < kDB * kDB; idx += kDThreads) {
      const int r = idx & 31, c = idx >> 5;
      sm.T[r][c] = (r < w0 && c < w0) ? a.D[r + (int64_t)c * a.ldd] : (r == c ? 1.0f : 0.0f);
    }
    __syncthreads();
    if (warp == 0) lu_factor(sm);
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
      // work CTAs skip those entries) with the same operations, so the same
      // results, factor it and publish it; sm.Us / Ls / Ud hold block p
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
        if (warp == 0) {
          row_solve(sm, 0);  // Lr[0][k][i] = L(e+i, b+k)
        } else if (warp == 1) {  // Lr[1][k][i] = z'_i(k) = U(b+k, e+i)
          float v[kDB];
#pragma unroll
          for (int m = 0; m < kDB; ++m) v[m] = sm.Ac[1][m][lane];
          lsolve(v, sm, &sm.Lr[1][0][lane], kDB + 1);
        }
        __syncthreads();
        {  // 2 x 2 entries per thread: each multiplier and z' entry loaded once for two products
          const int i = (t & 15) * 2, c = (t >> 4) * 2;
          float a00 = sm.T[i][c], a10 = sm.T[i + 1][c], a01 = sm.T[i][c + 1], a11 = sm.T[i + 1][c + 1];
#pragma unroll
          for (int k = 0; k < kDB; ++k) {
            const float l0 = -sm.Lr[0][k][i], l1 = -sm.Lr[0][k][i + 1];
            const float z0 = sm.Lr[1][k][c], z1 = sm.Lr[1][k][c + 1];
            a00 = fmaf(l0, z0, a00);
            a10 = fmaf(l1, z0, a10);
            a01 = fmaf(l0, z1, a01);
            a11 = fmaf(l1, z1, a11);
          }
          if (i < w1 && c < w1) sm.T[i][c] = a00;
          if (i + 1 < w1 && c < w1) sm.T[i + 1][c] = a10;
          if (i < w1 && c + 1 < w1) sm.T[i][c + 1] = a01;
          if (i + 1 < w1 && c + 1 < w1) sm.T[i + 1][c + 1] = a11;
        }
        __syncthreads();
        if (warp == 0) lu_factor(sm);
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
    // (1) queue: the factored block p from the diagonal CTA, the block row z
    // of this CTA's live columns and its chunks below the block
    {
      const float* s = a.sc + (int64_t)p * kSlot;
      for (int idx = t; idx < 2 * kDB * (kDB / 4); idx += kDThreads) {  // 16-byte pieces of Us and Ls
        const int k = (idx >> 3) & 31, c4 = idx & 7;
        float* dst = idx < kDB * (kDB / 4) ? &sm.Us[k][4 * c4] : &sm.Ls[k][4 * c4];
        cp_async16(dst, s + kDB * kDB + 4 * idx);
      }
      if (t < kDB / 4) cp_async16(&sm.Ud[4 * t], s + 3 * kDB * kDB + 4 * t);
    }
    const int jl = first_live(cgi, CG, e);
    for (int jj = jl + warp; jj < nown; jj += kDThreads / 32) {
      const float* col = a.D + (int64_t)(cgi + jj * CG) * a.ldd;
      if (lane < w) cp_async4(&Zs[jj * kZS + lane], col + b + lane);
      else Zs[jj * kZS + lane] = 0.0f;
    }
    const int nq = queue_chunks(sm, a, rg, b, w, e, jb);
    asm volatile("cp.async.commit_group;" ::: "memory");
    // the trailing entries as a second group: only the update needs them, so
    // they keep arriving while the substitutions run
    float* Cs = Zs + (nown + 1) * kZS;
    stage_trailing(Cs, a, rg, cgi, nown, nq, e);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    // (2) one warp per task: L = A U_pp^-1 for a chunk (tasks < nq), or
    // z' = L_pp^-1 z in place for 32 live columns
    const int nzt = nown > jl ? (nown - jl + 31) / 32 : 0;
    for (int task = warp; task < nq + nzt; task += kDThreads / 32) {
      if (task < nq) {
        row_solve(sm, task);
      } else {
        const int jj = jl + (task - nq) * 32 + lane;
        float* zc = Zs + (jj < nown ? jj : nown) * kZS;  // row nown: a spare row for idle lanes
        float v[kDB];
#pragma unroll
        for (int i = 0; i < kDB / 4; ++i) {
          const float4 q = reinterpret_cast<const float4*>(zc)[i];
          v[4 * i] = q.x, v[4 * i + 1] = q.y, v[4 * i + 2] = q.z, v[4 * i + 3] = q.w;
        }
        lsolve(v, sm, zc, 1);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    // (4) the rank-32 update of this CTA's (row, column) pairs
    apply_updates(sm, Zs, Cs, a, rg, cgi, nown, nq, e);
    prev_nq = nq;
    target += G;
    if (!diag_barrier(a.bar, target, a.err, &sm.flag)) return;
  }
  if (!diag_cta) {
    __syncthreads();
    deferred_writes(sm, Zs, a, rg, cgi, nown, nblk - 1, prev_nq);
  }
}

}  // namespace

int diag_scratch_floats(int64_t jb) { return (int)(((jb + kDB - 1) / kDB) * kSlot); }

namespace {
constexpr int kMaxDyn = 227 * 1024;

// Dynamic shared memory of the diagonal kernel for jb columns over cg column
// groups: Zs, then Cs for at most ceil(nblk / kRG) chunks of the CTA's
// columns; and more than half of an SM's shared memory, so that no two CTAs
// share an SM: the diagonal CTA's serial chain is the critical path of every
// step, and a work CTA beside it would take its issue slots.  0 when cg
// groups cannot hold jb columns.
size_t diag_smem(int64_t jb, int cg) {
  const int nown = (int)((jb + cg - 1) / cg);
  if ((nown + 7) / 8 > kMaxCW) return 0;
  const int nblk = (int)((jb + kDB - 1) / kDB);
  const int nqmax = (nblk + kRG - 1) / kRG;
  size_t dyn = kZsOffset + (size_t)(nown + 1) * kZS * sizeof(float) + (size_t)nqmax * nown * kDB * sizeof(float);
  if (dyn < 120 * 1024) dyn = 120 * 1024;
  return dyn > (size_t)kMaxDyn ? 0 : dyn;
}
}  // namespace

int mxp_diag_min_ctas(int64_t jb) {
  for (int cg = 1; cg <= 18; ++cg)
    if (diag_smem(jb, cg)) return kRG * cg + 1;
  return 0;
}

// Factor the jb x jb block D (ldd) in place, jb <= 2048; sc holds
// diag_scratch_floats(jb) floats.  At most max_ctas CTAs (0: up to 145).
int launch_mxp_diag(Workspace* ws, int64_t jb, float* D, int64_t ldd, float* sc, int32_t* info, int64_t info_shift,
                    cudaStream_t s, int max_ctas) {
  if (jb <= 0) return HPL_OK;
  if (jb > 2048) return set_error(HPL_ERR_NOTSUP, "mxp diagonal block larger than 2048");
  int cg = (int)(jb / 64);
  if (cg < 1) cg = 1;
  if (cg > 18) cg = 18;  // 145 CTAs at most, one per SM
  const int cap = max_ctas > 0 && max_ctas < ws->num_sms ? max_ctas : ws->num_sms;
  while (kRG * cg + 1 > cap && cg > 1) --cg;
  const int G = kRG * cg + 1;  // work CTAs and the diagonal CTA
  const size_t dyn = diag_smem(jb, cg);
  if (!dyn) return set_error(HPL_ERR_NOTSUP, "mxp diagonal block: %d CTAs cannot hold %d columns", G, (int)jb);
  const int nblk = (int)((jb + kDB - 1) / kDB);
  HPL_TRY(set_smem_attr((const void*)mxp_diag_kernel, kMaxDyn));
  DiagArgs a;
  a.jb = (int)jb;
  a.cg = cg;
  a.nwork = G - 1;
  a.D = D;
  a.ldd = ldd;
  a.sc = sc;
  a.info = info;
  a.info_shift = info_shift;
  a.bar = ws->bar;
  a.bar_base = ws->bar_next;
  a.err = ws->dev_err;
  ws->bar_next += (unsigned long long)G * (unsigned long long)(1 + nblk);
  mxp_diag_kernel<<<G, kDThreads, dyn, s>>>(a);
  count_launch();
  return check_launch("mxp_diag_kernel");
}

}  // namespace hplgb
