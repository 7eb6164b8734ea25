// mxp_gemm.cu -- trailing update of the mixed-precision LU on the 5th-generation
// tensor cores:  C (FP32, column-major) -= 2^-(eL + eU) * qL qU^T
// with qL (m x K) and qU (n x K) stored K-major (row-major, row pitch kp
// elements) in BF16 (tcgen05 kind::f16) or FP8-E4M3 (kind::f8f6f4), one
// power-of-two exponent per 128-row tile of qL (eL) and per 128-row tile of
// qU (eU), and FP32 accumulation in tensor memory.
//
// Persistent kernel, one CTA per SM, 128 x 256 output tiles visited in bands
// of kBand row-tiles (so a band of qL stays in L2 while the column tiles
// stream past it):
//   warp 0    one elected thread issues TMA loads (128B swizzle) of the qL and qU
//             K-slices into a ring of kStages shared-memory stages (mbarriers
//             full/empty), continuing across tiles;
//   warp 1    allocates 512 TMEM columns = two 256-column FP32 accumulators;
//             one elected thread issues tcgen05.mma (M=128, N=256) for tile i
//             into accumulator i % 2, commits each stage back to the producer
//             and the finished accumulator to the epilogue;
//   warps 2-9 read accumulator i % 2 with tcgen05.ld (two warps per 32-lane
//             quarter of TMEM, one per column half), scale it by 2^-(eL+eU),
//             subtract it from C (coalesced along C's columns, 64 loads in
//             flight per thread) and hand the accumulator back -- so the
//             epilogue of tile i overlaps the MMAs of tile i+1.
// Every wait is bounded: a wait that exceeds ~1 s records DEV_TIMEOUT, lets the
// other roles run out, waits (bounded) for copies it issued, frees TMEM and
// returns.  No TMA multicast is used.
#include <cuda.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"

namespace hplgb {

namespace {

constexpr int kBM = 128, kBN = 256;
constexpr int kStageA = kBM * 128;                  // bytes: 128 rows x 128 B
constexpr int kStageB = kBN * 128;                  // bytes: 256 rows x 128 B
constexpr int kStageBytes = kStageA + kStageB;      // 48 KB
constexpr int kEpiWarps = 8;                        // two warps per TMEM lane quarter
// Two epilogue designs (template flag CT):
//  CT = false: C is read and written from registers, 4 operand stages;
//  CT = true:  C moves through shared memory by TMA (needs ldc % 4 == 0 and a
//              16-byte aligned C): a loader warp (warp 10) keeps kCSlots chunks
//              of 128 x 32 FP32 in flight ahead of the epilogue, and the
//              epilogue warps store their 32 x 32 sub-blocks back with TMA;
//              3 operand stages make room.
constexpr int kCSlots = 5;
// The two epilogue halves work four chunks apart, so with four slots or fewer
// a half can wait on a slot whose previous use (the other half's chunk) has not
// landed yet: two phases behind, and the parity wait passes on the older phase.
// Every slot's previous use must belong to the waiting half itself.
static_assert(kCSlots > (kBN / 32) / 2, "a C slot's previous use must be the waiting half's own chunk");
constexpr int kCSlotBytes = kBM * 32 * 4;           // 16 KB: four 32 x 32 sub-blocks
// FP32-accurate products (X3): one stage holds all three BF16 pieces of A
// and of B for one 64-byte K slice (64-byte swizzle), and all six piece
// products run from it, so every operand byte is loaded once instead of
// twice; 3 stages of 72 KB.
constexpr int kX3SliceBytes = 64;
constexpr int kX3StageA = 3 * kBM * kX3SliceBytes;   // 24 KB
constexpr int kX3StageB = 3 * kBN * kX3SliceBytes;   // 48 KB
__host__ __device__ constexpr int stage_a_of(bool x3) { return x3 ? kX3StageA : kStageA; }
__host__ __device__ constexpr int stage_bytes_of(bool x3) { return x3 ? kX3StageA + kX3StageB : kStageBytes; }
__host__ __device__ constexpr int stages_of(bool ct, bool x3 = false) { return x3 ? 3 : (ct ? 3 : 4); }
__host__ __device__ constexpr int threads_of(bool ct) { return 64 + 32 * kEpiWarps + (ct ? 32 : 0); }
__host__ __device__ constexpr int smem_of(bool ct, bool x3 = false) {
  return stages_of(ct, x3) * stage_bytes_of(x3) + (ct ? kCSlots * kCSlotBytes : 0) + 1024 + 512;
}
constexpr int kTmemCols = 512;                      // two 128 x 256 FP32 accumulators
constexpr int kBand = 64;                           // row tiles per band of the tile order
constexpr unsigned long long kWaitLimitNs = 1000000000ULL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and DEV_TIMEOUT) after ~1 s, or at
// once if another role of this CTA already gave up (*abort != 0).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = now_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort) return false;
      if (now_ns() - t0 > kWaitLimitNs) {
        *abort = 1;
        atomicExch(err, DEV_TIMEOUT);
        return false;
      }
    }
  }
}

// L2 policies: the operands are reread by many tiles (keep them), the FP32
// C stream passes once per panel and is larger than L2 (let it go first).
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}

// Bulk tensor store of a box from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y, uint64_t policy) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%2, %3}], [%1], %4;"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(src)), "r"(x), "r"(y), "l"(policy)
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// canonical layout (8-row atoms of 8 x 128 B, atoms 1024 B apart).
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
  uint64_t addr = (smem_u32(p) & 0x3FFFFu) >> 4;
  uint64_t d = 0;
  d |= addr;                       // bits 0-13  start address >> 4
  d |= (uint64_t)1 << 16;          // bits 16-29 leading byte offset >> 4 (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // bits 32-45 stride byte offset >> 4: 8-row atom pitch
  d |= (uint64_t)1 << 46;          // bits 46-48 fixed 0b001
  d |= (uint64_t)2 << 61;          // bits 61-63 swizzle mode: 128-byte
  return d;
}

// The same for the 64-byte swizzle (8-row atoms of 8 x 64 B, 512 B apart).
__device__ __forceinline__ uint64_t smem_desc_sw64(const void* p) {
  uint64_t addr = (smem_u32(p) & 0x3FFFFu) >> 4;
  uint64_t d = 0;
  d |= addr;
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;          // swizzle mode: 64-byte
  return d;
}

// Instruction descriptor: D = F32, A = B = fmt, both K-major, M = 128, N = 256.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt) {
  return (1u << 4)            // D format F32
         | (fmt << 7)         // A format
         | (fmt << 10)        // B format
         | ((uint32_t)(kBN >> 3) << 17)
         | ((uint32_t)(kBM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 2^-e as a float (e in [-126, 126]): the IEEE binary32 pattern with biased
// exponent 127 - e and zero fraction.
__device__ __forceinline__ float pow2_neg(int e) { return __int_as_float((127 - e) << 23); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Tile t of the banded order -> (row tile, column tile).
// With a triangular operand a tile's K range grows with its row (tri == 1,
// lower-triangular A) or its column (tri == 2, upper-triangular B), and the
// persistent CTAs, which take every gridDim.x-th tile, would keep drawing the
// same rows or columns.  So the rows run down in odd columns of a band
// (tri == 1) and the columns run right to left in odd bands (tri == 2): each
// CTA gets long and short tiles alike, while the tiles of one column still run
// together (its qU slice stays in L2).
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int tri, int* tm, int* tn) {
  const int per_band = kBand * tiles_n;
  const int band = t / per_band;
  const int rows_in_band = min(kBand, tiles_m - band * kBand);
  const int idx = t - band * per_band;
  int c = idx / rows_in_band, r = idx % rows_in_band;
  if (tri == 1 && (c & 1)) r = rows_in_band - 1 - r;
  if (tri == 2 && (band & 1)) c = tiles_n - 1 - c;
  *tn = c;
  *tm = band * kBand + r;
}

// K steps of tile (tm, tn): all of them, or only those up to the edge of a
// triangular operand (tri 1: A lower triangular, row i nonzero for k <= i;
// tri 2: B upper triangular, column j nonzero for k <= j).
// Maximum of |stored value| over the warp into amax[idx] (bit patterns of
// non-negative floats order like the values): the tile maxima of a product
// that is quantized next, taken while it is written.
__device__ __forceinline__ void tile_amax(unsigned* amax, int idx, float vm, int lane, bool valid) {
#pragma unroll
  for (int o = 16; o; o >>= 1) vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
  if (lane == 0 && valid) atomicMax(&amax[idx], __float_as_uint(vm));
}

__device__ __forceinline__ int tile_ksteps(int ksteps, int tri, int tm, int tn, int per_step) {
  if (tri != 1 && tri != 2) return ksteps;
  const int kend = tri == 1 ? (tm + 1) * kBM : (tn + 1) * kBN;
  const int s = (kend + per_step - 1) / per_step;
  return s < ksteps ? s : ksteps;
}

// The tiles of one CTA.  Static (ctr null): tiles lo + blockIdx.x + i
// gridDim.x below hi.  Dynamic: the producer thread claims each next tile from
// a counter in global memory that every CTA of the launches taking part in
// one update shares, so that CTAs that start late (on SMs another kernel
// held) take fewer tiles; it hands the tile to the other roles through a ring
// of kSchedSlots shared words, each with a full barrier (the producer's
// arrival) and an empty one (one arrival per reader).  -1 ends the schedule.
constexpr int kSchedSlots = 8;
struct TileSched {
  int* ctr;
  int lo, hi;
  volatile int* slot;
  uint64_t* sfull;
  uint64_t* sempty;

  // producer: the CTA's i-th tile
  __device__ __forceinline__ bool claim(int i, int* t, volatile int* abort, int* err) const {
    if (!ctr) {
      *t = lo + (int)blockIdx.x + i * (int)gridDim.x;
      return *t < hi;
    }
    const int s = i % kSchedSlots, use = i / kSchedSlots;
    if (use > 0 && !mbar_wait(&sempty[s], (use - 1) & 1, abort, err)) return false;
    int v = lo + atomicAdd(ctr, 1);
    if (v >= hi) v = -1;
    slot[s] = v;
    mbar_arrive(&sfull[s]);
    *t = v;
    return v >= 0;
  }
  // one reader thread of a role: the same i-th tile
  __device__ __forceinline__ bool next(int i, int* t, volatile int* abort, int* err) const {
    if (!ctr) {
      *t = lo + (int)blockIdx.x + i * (int)gridDim.x;
      return *t < hi;
    }
    const int s = i % kSchedSlots;
    if (!mbar_wait(&sfull[s], (i / kSchedSlots) & 1, abort, err)) return false;
    const int v = slot[s];
    mbar_arrive(&sempty[s]);
    *t = v;
    return v >= 0;
  }
};

template <int KIND, bool CT, bool X3>
__global__ void __launch_bounds__(threads_of(CT), 1)
mxp_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const __grid_constant__ CUtensorMap tmC, int m, int n, int ksteps, int nterm, uint32_t sched,
                int kpiece, int store, int tri, float* __restrict__ C, int64_t ldc, const int* __restrict__ eL,
                const int* __restrict__ eU, int tiles_m, int tiles_n, int* err, unsigned* __restrict__ amax,
                int amax_by, int tile_lo, int tile_hi, int* tile_ctr) {
  static_assert(!X3 || (KIND == 0 && !CT), "the fused-piece stages are for BF16 store-mode products");
  constexpr int kStages = stages_of(CT, X3);
  constexpr int kSB = stage_bytes_of(X3), kSA = stage_a_of(X3);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* cslots = reinterpret_cast<float*>(smem + kStages * kSB);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kSB + (CT ? kCSlots * kCSlotBytes : 0));
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;   // [2]
  uint64_t* acc_empty = acc_full + 2;     // [2]
  uint64_t* c_full = acc_empty + 2;       // [kCSlots] (CT)
  uint64_t* c_empty = c_full + kCSlots;   // [kCSlots] (CT)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(c_empty + kCSlots);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  TileSched sch;  // this launch takes tiles tile_lo .. tile_hi - 1 of the order
  sch.ctr = tile_ctr;
  sch.lo = tile_lo;
  sch.hi = tile_hi;
  sch.slot = reinterpret_cast<volatile int*>(tmem_slot + 2);
  sch.sfull = reinterpret_cast<uint64_t*>(tmem_slot + 2 + kSchedSlots);
  sch.sempty = sch.sfull + kSchedSlots;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kEpiWarps);  // one arrival per epilogue warp
    }
    if (CT) {
      for (int c = 0; c < kCSlots; ++c) {
        mbar_init(&c_full[c], 1);   // the loader's arrival (with the TMA bytes)
        mbar_init(&c_empty[c], 4);  // the four lane-quarter warps that consumed it
      }
    }
    for (int q = 0; q < kSchedSlots; ++q) {
      mbar_init(&sch.sfull[q], 1);
      mbar_init(&sch.sempty[q], 1 + (CT ? 1 : 0) + kEpiWarps);  // MMA thread, C loader, epilogue warps
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer: K-slices of every tile of this CTA, in order
    const uint64_t keep = policy_evict_last();
    int g = 0;  // global K-step counter of this CTA
    bool ok = true;
    for (int i = 0, t; ok && sch.claim(i, &t, abort, err); ++i) {
      int tm, tn;
      tile_coords(t, tiles_m, tiles_n, tri, &tm, &tn);
      const int kst = tile_ksteps(ksteps, tri, tm, tn, X3 ? kX3SliceBytes / 2 : (KIND == 0 ? 64 : 128));
      if (X3) {
        // slice ks: pieces 0..2 of A's rows and of B's columns, 32 elements each
        for (int ks = 0; ks < kst; ++ks, ++g) {
          const int s = g % kStages, round = g / kStages;
          if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1, abort, err)) { ok = false; break; }
          uint8_t* a = smem + s * kSB;
          uint8_t* b = a + kSA;
          mbar_expect_tx(&full[s], kSB);
          const int kx = ks * (kX3SliceBytes / 2);
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            tma_load_2d(a + p * (kBM * kX3SliceBytes), &tmA, &full[s], p * kpiece + kx, tm * kBM, keep);
            tma_load_2d(b + p * (kBN * kX3SliceBytes), &tmB, &full[s], p * kpiece + kx, tn * kBN, keep);
          }
        }
        continue;
      }
      for (int kt = 0; kt < kst * nterm; ++kt, ++g) {
        const int s = g % kStages, round = g / kStages;
        if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1, abort, err)) { ok = false; break; }
        uint8_t* a = smem + s * kSB;
        uint8_t* b = a + kSA;
        mbar_expect_tx(&full[s], kSB);
        // term kt / kst multiplies piece pa of qL by piece pb of qU; each
        // piece spans kpiece elements of the row, 128 bytes per K step
        const int term = kt / kst, ks = kt - term * kst;
        const int pa = (int)((sched >> (4 * term)) & 3u), pb = (int)((sched >> (4 * term + 2)) & 3u);
        const int kx = ks * (KIND == 0 ? 64 : 128);
        tma_load_2d(a, &tmA, &full[s], pa * kpiece + kx, tm * kBM, keep);
        tma_load_2d(b, &tmB, &full[s], pb * kpiece + kx, tn * kBN, keep);
      }
    }
    if (*abort) {  // wait (bounded) for the copies still in flight
      for (int q = (g > kStages ? g - kStages : 0); q < g; ++q) {
        unsigned long long t0 = now_ns();
        while (!mbar_try_wait(&full[q % kStages], (q / kStages) & 1) && now_ns() - t0 < kWaitLimitNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = make_idesc(KIND == 0 ? 1u : 0u);  // BF16 = 1, E4M3 = 0
    int g = 0, i = 0;
    bool ok = true;
    for (int t; ok && sch.next(i, &t, abort, err); ++i) {
      const int abuf = i & 1, use = i >> 1;
      if (use > 0 && !mbar_wait(&acc_empty[abuf], (use - 1) & 1, abort, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dacc = tmem + (uint32_t)(abuf * kBN);
      int tm, tn;
      tile_coords(t, tiles_m, tiles_n, tri, &tm, &tn);
      const int kst = tile_ksteps(ksteps, tri, tm, tn, X3 ? kX3SliceBytes / 2 : (KIND == 0 ? 64 : 128));
      if (X3) {
        // per slice the six piece products, smallest first, 2 MMAs of 32 bytes of K each
        for (int ks = 0; ks < kst; ++ks, ++g) {
          const int s = g % kStages;
          if (!mbar_wait(&full[s], (g / kStages) & 1, abort, err)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint8_t* a = smem + s * kSB;
          const uint8_t* b = a + kSA;
#pragma unroll
          for (int term = 0; term < 6; ++term) {
            const int pa = (int)((sched >> (4 * term)) & 3u), pb = (int)((sched >> (4 * term + 2)) & 3u);
            const uint64_t ad = smem_desc_sw64(a + pa * (kBM * kX3SliceBytes));
            const uint64_t bd = smem_desc_sw64(b + pb * (kBN * kX3SliceBytes));
#pragma unroll
            for (int k = 0; k < kX3SliceBytes / 32; ++k)
              mma<KIND>(dacc, ad + 2 * k, bd + 2 * k, idesc, (ks > 0 || term > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&acc_full[abuf]);
        continue;
      }
      for (int ks = 0; ks < kst * nterm; ++ks, ++g) {
        const int s = g % kStages;
        if (!mbar_wait(&full[s], (g / kStages) & 1, abort, err)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint8_t* a = smem + s * kSB;
        const uint8_t* b = a + kSA;
        const uint64_t ad = smem_desc_sw128(a), bd = smem_desc_sw128(b);
#pragma unroll
        for (int k = 0; k < 4; ++k)  // 4 MMAs of 32 bytes of K each (K = 16 BF16 or 32 E4M3)
          mma<KIND>(dacc, ad + 2 * k, bd + 2 * k, idesc, (ks > 0 || k > 0) ? 1u : 0u);
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(&acc_full[abuf]);
    }
  } else if (CT && warp == 2 + kEpiWarps) {
    // ---------------- C loader: chunk g (tile i, columns 32c..32c+31, g = 8i + c)
    // goes to slot g % kCSlots, as four 32 x 32 sub-blocks (one per lane
    // quarter); in store mode nothing is read and the slot is only handed over
    if (lane == 0) {
      const uint64_t stream = policy_evict_first();
      int g = 0;
      bool ok = true;
      for (int i = 0, t; ok && sch.next(i, &t, abort, err); ++i) {
        int tm, tn;
        tile_coords(t, tiles_m, tiles_n, tri, &tm, &tn);
        for (int c = 0; c < kBN / 32; ++c, ++g) {
          const int slot = g % kCSlots, use = g / kCSlots;
          if (use > 0 && !mbar_wait(&c_empty[slot], (use - 1) & 1, abort, err)) { ok = false; break; }
          // sub-blocks that start inside C (a box that starts inside is read
          // in full, zero-filled beyond the edge; the others are skipped)
          const int col = tn * kBN + 32 * c;
          int nsub = 0;
          if (!store && col < n)
            for (int q = 0; q < 4; ++q) nsub += (tm * kBM + 32 * q < m) ? 1 : 0;
          if (nsub == 0) {
            mbar_arrive(&c_full[slot]);
          } else {
            mbar_expect_tx(&c_full[slot], (uint32_t)(nsub * 4096));
            float* dst = cslots + slot * (kCSlotBytes / 4);
            for (int q = 0; q < 4; ++q)
              if (tm * kBM + 32 * q < m)
                tma_load_2d(dst + q * 1024, &tmC, &c_full[slot], tm * kBM + 32 * q, col, stream);
          }
        }
      }
      if (*abort && !store) {  // wait (bounded) for the loads still in flight
        for (int q = (g > kCSlots ? g - kCSlots : 0); q < g; ++q) {
          unsigned long long t0 = now_ns();
          while (!mbar_try_wait(&c_full[q % kCSlots], (q / kCSlots) & 1) && now_ns() - t0 < kWaitLimitNs) {
          }
        }
      }
    }
  } else if (CT && warp >= 2) {
    // ---------------- epilogue through shared memory: warp (quarter q, half h)
    // takes chunks 4h..4h+3 of each tile: 32 accumulator columns of its 32
    // lanes per chunk, combined with the C sub-block the loader brought in,
    // written back in place and stored by TMA
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint64_t stream = policy_evict_first();
    int i = 0;
    bool ok = true;
    for (; ok; ++i) {
      int t = 0, have = 0;
      if (lane == 0) have = sch.next(i, &t, abort, err) ? 1 : 0;
      have = __shfl_sync(0xffffffffu, have, 0);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (!have) break;
      const int abuf = i & 1, use = i >> 1;
      int ready = 0;
      if (lane == 0) ready = mbar_wait(&acc_full[abuf], use & 1, abort, err) ? 1 : 0;
      ready = __shfl_sync(0xffffffffu, ready, 0);
      if (!ready) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int tm, tn;
      tile_coords(t, tiles_m, tiles_n, tri, &tm, &tn);
      const int m0 = tm * kBM, n0 = tn * kBN;
      const float sl = pow2_neg(eL[tm]);
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * kBN);
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
        const int c = half * 4 + cc;
        const int g = i * (kBN / 32) + c;
        const int slot = g % kCSlots;
        float v[32];
        tmem_ld32(tbase + (uint32_t)(c * 32), v);
        int got = 0;
        if (lane == 0) got = mbar_wait(&c_full[slot], (g / kCSlots) & 1, abort, err) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) { ok = false; break; }
        const int cA = n0 + c * 32;
        const float su = pow2_neg(eU[min(cA, n - 1) / 128]) * sl;
        float* sub = cslots + slot * (kCSlotBytes / 4) + q * 1024;  // [32 columns][32 rows]
        if (store) {
          float vm = 0.0f;
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const float y = v[k] * su;
            sub[k * 32 + lane] = y;
            vm = fmaxf(vm, fabsf(y));
          }
          if (amax_by) tile_amax(amax, amax_by == 1 ? tm : cA / 128, vm, lane, cA < n && m0 + 32 * q < m);
        } else {
#pragma unroll
          for (int k = 0; k < 32; ++k) sub[k * 32 + lane] = fmaf(-v[k], su, sub[k * 32 + lane]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (cA < n && m0 + 32 * q < m) {
            tma_store_2d(&tmC, sub, m0 + 32 * q, cA, stream);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          }
          mbar_arrive(&c_empty[slot]);
        }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[abuf]);
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  } else if (!CT && warp >= 2) {
    // ---------------- epilogue from registers: warp w reads TMEM lane quarter
    // w % 4 and column half (w - 2) / 4; two 32-column chunks at a time so
    // that 64 loads of C per thread are in flight
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    int i = 0;
    for (;; ++i) {
      int t = 0, have = 0;
      if (lane == 0) have = sch.next(i, &t, abort, err) ? 1 : 0;
      have = __shfl_sync(0xffffffffu, have, 0);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (!have) break;
      const int abuf = i & 1, use = i >> 1;
      int ready = 0;
      if (lane == 0) ready = mbar_wait(&acc_full[abuf], use & 1, abort, err) ? 1 : 0;
      ready = __shfl_sync(0xffffffffu, ready, 0);  // warp-uniform: tcgen05.ld is .sync.aligned
      if (!ready) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int tm, tn;
      tile_coords(t, tiles_m, tiles_n, tri, &tm, &tn);
      const int m0 = tm * kBM, n0 = tn * kBN;
      const int row = m0 + q * 32 + lane;
      const float sl = pow2_neg(eL[tm]);
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * kBN);
#pragma unroll 1
      for (int cp2 = 0; cp2 < 2; ++cp2) {
        const int cc = half * 4 + cp2 * 2;  // chunks cc, cc + 1
        float v[64];
        tmem_ld32(tbase + (uint32_t)(cc * 32), v);
        tmem_ld32(tbase + (uint32_t)((cc + 1) * 32), v + 32);
        const int cA = n0 + cc * 32;
        if (store && amax_by && cA < n) {  // the chunk pair lies in one 128-column group
          float vm = 0.0f;
          if (row < m) {
            const int cn = min(64, n - cA);
            const float su0 = pow2_neg(eU[cA / 128]);
            const float su1 = pow2_neg(eU[min(cA + 32, n - 1) / 128]);
#pragma unroll
            for (int c = 0; c < 64; ++c)
              if (c < cn) vm = fmaxf(vm, fabsf((v[c] * sl) * (c < 32 ? su0 : su1)));
          }
          tile_amax(amax, amax_by == 1 ? tm : cA / 128, vm, lane, true);
        }
        if (cA >= n || row >= m) continue;
        const int cn = min(64, n - cA);
        const float su0 = pow2_neg(eU[cA / 128]);
        const float su1 = pow2_neg(eU[min(cA + 32, n - 1) / 128]);
        float* cp = C + (int64_t)row + (int64_t)cA * ldc;
        if (store) {  // C = 2^-(eL+eU) acc
#pragma unroll
          for (int c = 0; c < 64; ++c)
            if (c < cn) cp[(int64_t)c * ldc] = (v[c] * sl) * (c < 32 ? su0 : su1);
        } else {      // C -= 2^-(eL+eU) acc
          float old[64];
#pragma unroll
          for (int c = 0; c < 64; ++c)
            if (c < cn) old[c] = cp[(int64_t)c * ldc];
#pragma unroll
          for (int c = 0; c < 64; ++c)
            if (c < cn) cp[(int64_t)c * ldc] = fmaf(-(v[c] * sl), c < 32 ? su0 : su1, old[c]);
        }
      }
      // this warp has read its part of the accumulator: hand it back
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[abuf]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ----------------------------------------- trailing update on SM pairs
// The same update, C -= 2^-(eL+eU) qL qU^T with the TMA C epilogue, with
// 256 x 256 tiles on the two SMs of a cluster (tcgen05 cta_group::2): CTA
// rank r of the pair loads its own 128 rows of qL and 128 of the tile's 256
// qU rows into its own shared memory (CTA-local TMA, no multicast); the
// leader's single MMA thread issues M = 256, N = 256 products that read both
// CTAs' stages and write each CTA's 128 x 256 accumulator into that CTA's
// TMEM.  Per SM a K step moves 32 KB (16 KB of qL, half of the 32 KB qU
// slice) instead of 48 KB, for the same flops.
//   full[s]   leader only: both CTAs' copies complete on it (the leader
//             expects the bytes of both);
//   empty[s]  each CTA: the leader's commit arrives on both (multicast);
//   acc_full  each CTA: the leader's commit, multicast;
//   acc_empty leader only: one arrival per epilogue warp of both CTAs.
// Static schedule: pair p of gridDim.x / 2 takes pair tiles p, p + pairs, ...
constexpr int kPairStages = 4;
constexpr int kPairBN = 128;                           // qU rows per CTA (half of N = 256)
constexpr int kPairStageB = kPairBN * 128;             // 16 KB
constexpr int kPairStageBytes = kStageA + kPairStageB; // 32 KB
constexpr int kPairSmem = kPairStages * kPairStageBytes + kCSlots * kCSlotBytes + 1024 + 512;
constexpr int kPairThreads = 64 + 32 * kEpiWarps + 32;  // producer, MMA, 8 epilogue warps, C loader
__host__ __device__ constexpr uint32_t make_idesc_pair(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// this CTA's shared address `a` as the same offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded as mbar_wait, with cluster-scope acquire (arrivals and copies of the peer CTA)
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* bar, uint32_t parity, volatile int* abort, int* err) {
  if (mbar_try_wait_cl(bar, parity)) return true;
  unsigned long long t0 = now_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait_cl(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort) return false;
      if (now_ns() - t0 > kWaitLimitNs) {
        *abort = 1;
        atomicExch(err, DEV_TIMEOUT);
        return false;
      }
    }
  }
}
// TMA load into this CTA's shared memory, completing on an mbarrier of either CTA of the pair
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t cluster_bar, int x, int y,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(cluster_bar), "r"(x), "r"(y), "l"(policy)
      : "memory");
}
template <int KIND>
__device__ __forceinline__ void mma_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  }
}
// arrive on the barrier at this offset in both CTAs once the leader's MMAs are done
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((unsigned short)3)
      : "memory");
}

template <int KIND>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPairThreads, 1)
mxp_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmC, int m, int n, int ksteps, const int* __restrict__ eL,
                     const int* __restrict__ eU, int ptiles_m, int tiles_n, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* cslots = reinterpret_cast<float*>(smem + kPairStages * kPairStageBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPairStages * kPairStageBytes + kCSlots * kCSlotBytes);
  uint64_t* empty = full + kPairStages;
  uint64_t* acc_full = empty + kPairStages;  // [2]
  uint64_t* acc_empty = acc_full + 2;        // [2]
  uint64_t* c_full = acc_empty + 2;          // [kCSlots]
  uint64_t* c_empty = c_full + kCSlots;      // [kCSlots]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(c_empty + kCSlots);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);
  const int nptiles = ptiles_m * tiles_n;

  if (threadIdx.x == 0) {
    for (int q = 0; q < kPairStages; ++q) {
      mbar_init(&full[q], 1);   // the leader's arrival (with the bytes of both CTAs)
      mbar_init(&empty[q], 1);  // the leader's commit
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 2 * kEpiWarps);  // the epilogue warps of both CTAs
    }
    for (int c = 0; c < kCSlots; ++c) {
      mbar_init(&c_full[c], 1);
      mbar_init(&c_empty[c], 4);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();  // both CTAs' barriers exist before any copy or arrival names them
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer (both CTAs): this CTA's halves of every K step
    const uint64_t keep = policy_evict_last();
    const uint32_t full_leader = cluster_addr(smem_u32(full), 0);
    int g = 0;
    bool ok = true;
    for (int t = pair; t < nptiles && ok; t += npairs) {
      int pm, tn;
      tile_coords(t, ptiles_m, tiles_n, 0, &pm, &tn);
      const int arow = (2 * pm + (int)rank) * kBM, brow = tn * kBN + (int)rank * kPairBN;
      for (int ks = 0; ks < ksteps; ++ks, ++g) {
        const int q = g % kPairStages, round = g / kPairStages;
        if (round > 0 && !mbar_wait_cl(&empty[q], (round - 1) & 1, abort, err)) { ok = false; break; }
        uint8_t* a = smem + q * kPairStageBytes;
        uint8_t* b = a + kStageA;
        if (leader) mbar_expect_tx(&full[q], 2 * kPairStageBytes);
        const int kx = ks * (KIND == 0 ? 64 : 128);
        const uint32_t bar = full_leader + (uint32_t)(q * sizeof(uint64_t));
        tma_load_2d_pair(a, &tmA, bar, kx, arow, keep);
        tma_load_2d_pair(b, &tmB, bar, kx, brow, keep);
      }
    }
    if (*abort && leader) {  // wait (bounded) for the copies of both CTAs still in flight
      for (int q = (g > kPairStages ? g - kPairStages : 0); q < g; ++q) {
        unsigned long long t0 = now_ns();
        while (!mbar_try_wait_cl(&full[q % kPairStages], (q / kPairStages) & 1) && now_ns() - t0 < kWaitLimitNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (leader): M = 256 over both CTAs, N = 256
    constexpr uint32_t idesc = make_idesc_pair(KIND == 0 ? 1u : 0u);
    int g = 0, i = 0;
    bool ok = true;
    for (int t = pair; t < nptiles && ok; t += npairs, ++i) {
      const int abuf = i & 1, use = i >> 1;
      if (use > 0 && !mbar_wait_cl(&acc_empty[abuf], (use - 1) & 1, abort, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dacc = tmem + (uint32_t)(abuf * kBN);
      for (int ks = 0; ks < ksteps; ++ks, ++g) {
        const int q = g % kPairStages;
        if (!mbar_wait_cl(&full[q], (g / kPairStages) & 1, abort, err)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint8_t* a = smem + q * kPairStageBytes;
        const uint8_t* b = a + kStageA;
        const uint64_t ad = smem_desc_sw128(a), bd = smem_desc_sw128(b);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma_pair<KIND>(dacc, ad + 2 * k, bd + 2 * k, idesc, (ks > 0 || k > 0) ? 1u : 0u);
        mma_commit_pair(&empty[q]);
      }
      if (ok) mma_commit_pair(&acc_full[abuf]);
    }
  } else if (warp == 2 + kEpiWarps) {
    // ---------------- C loader (both CTAs): this CTA's 128 x 256 block of C
    if (lane == 0) {
      const uint64_t stream = policy_evict_first();
      int g = 0;
      bool ok = true;
      for (int t = pair; t < nptiles && ok; t += npairs) {
        int pm, tn;
        tile_coords(t, ptiles_m, tiles_n, 0, &pm, &tn);
        const int tm = 2 * pm + (int)rank;
        for (int c = 0; c < kBN / 32; ++c, ++g) {
          const int slot = g % kCSlots, use = g / kCSlots;
          if (use > 0 && !mbar_wait(&c_empty[slot], (use - 1) & 1, abort, err)) { ok = false; break; }
          const int col = tn * kBN + 32 * c;
          int nsub = 0;
          if (col < n)
            for (int q = 0; q < 4; ++q) nsub += (tm * kBM + 32 * q < m) ? 1 : 0;
          if (nsub == 0) {
            mbar_arrive(&c_full[slot]);
          } else {
            mbar_expect_tx(&c_full[slot], (uint32_t)(nsub * 4096));
            float* dst = cslots + slot * (kCSlotBytes / 4);
            for (int q = 0; q < 4; ++q)
              if (tm * kBM + 32 * q < m) tma_load_2d(dst + q * 1024, &tmC, &c_full[slot], tm * kBM + 32 * q, col, stream);
          }
        }
      }
      if (*abort) {
        for (int q = (g > kCSlots ? g - kCSlots : 0); q < g; ++q) {
          unsigned long long t0 = now_ns();
          while (!mbar_try_wait(&c_full[q % kCSlots], (q / kCSlots) & 1) && now_ns() - t0 < kWaitLimitNs) {
          }
        }
      }
    }
  } else if (warp >= 2 && warp < 2 + kEpiWarps) {
    // ---------------- epilogue (both CTAs): as the single-SM TMA epilogue, on
    // this CTA's accumulator; the accumulator goes back to the leader's MMA
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint64_t stream = policy_evict_first();
    const uint32_t acc_empty_leader = cluster_addr(smem_u32(acc_empty), 0);
    int i = 0;
    bool ok = true;
    for (int t = pair; t < nptiles && ok; t += npairs, ++i) {
      const int abuf = i & 1, use = i >> 1;
      int ready = 0;
      if (lane == 0) ready = mbar_wait_cl(&acc_full[abuf], use & 1, abort, err) ? 1 : 0;
      ready = __shfl_sync(0xffffffffu, ready, 0);
      if (!ready) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int pm, tn;
      tile_coords(t, ptiles_m, tiles_n, 0, &pm, &tn);
      const int tm = 2 * pm + (int)rank;
      const int m0 = tm * kBM, n0 = tn * kBN;
      const float sl = pow2_neg(eL[min(tm, (m - 1) / kBM)]);
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * kBN);
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
        const int c = half * 4 + cc;
        const int g = i * (kBN / 32) + c;
        const int slot = g % kCSlots;
        float v[32];
        tmem_ld32(tbase + (uint32_t)(c * 32), v);
        int got = 0;
        if (lane == 0) got = mbar_wait(&c_full[slot], (g / kCSlots) & 1, abort, err) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) { ok = false; break; }
        const int cA = n0 + c * 32;
        const float su = pow2_neg(eU[min(cA, n - 1) / 128]) * sl;
        float* sub = cslots + slot * (kCSlotBytes / 4) + q * 1024;
#pragma unroll
        for (int k = 0; k < 32; ++k) sub[k * 32 + lane] = fmaf(-v[k], su, sub[k * 32 + lane]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (cA < n && m0 + 32 * q < m) {
            tma_store_2d(&tmC, sub, m0 + 32 * q, cA, stream);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          }
          mbar_arrive(&c_empty[slot]);
        }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        if (leader) mbar_arrive(&acc_empty[abuf]);
        else mbar_arrive_remote(acc_empty_leader + (uint32_t)(abuf * sizeof(uint64_t)));
      }
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync_all();  // neither CTA leaves while the pair's MMAs or copies may touch it
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ----------------------------------------- fused emulated FP64 update
// C (FP64, column-major) -= 2^(E_r + F_c - 2 beta) S with S the level sum
// of the slice products of ozaki.cu, made here in one persistent kernel: for
// every 128 x 128 tile of C the MMA warp makes the levels d = s+1 .. 2 one
// after the other into two 128-column FP32 accumulators (alternating), and the
// epilogue warps fold each finished level into a running sum held in the
// other 256 TMEM columns (two 32-bit columns per value): the levels d >= d0
// exactly, as a 64-bit integer T += P_d 2^((s+1-d) beta); at level d0 - 1 the
// sum turns into FP64, S = P_(d0-1) + fl(T) 2^-((s+2-d0) beta), and the rest
// is S = P_d + 2^-beta S (the oracle's operations, so the result is bitwise
// the oracle's).  After the last level they read C once, apply the update and
// write it back.
// Operands: A's slices (rows of pitch s kp, slices 1..s) and B's (columns of
// pitch s kp, slices s..1); level d reads the first (d-1) kp elements of A's
// rows and the last (d-1) kp of B's columns.
constexpr int kOzBN = 128;
constexpr int kOzStageBytes = kStageA + kOzBN * 128;   // 32 KB: A and B boxes of 128 rows x 128 B
constexpr int kOzStages = 5;  // leaves room on every SM for a FACT base CTA beside it
constexpr int kOzThreads = 64 + 32 * kEpiWarps;        // producer, MMA, 8 epilogue warps
constexpr int kOzSmem = kOzStages * kOzStageBytes + 1024 + 512;
constexpr uint32_t kOzIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kOzBN >> 3) << 17) |
                              ((uint32_t)(kBM >> 4) << 24);  // D F32, A = B = BF16, K-major, M 128, N 128

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void tmem_ld32u(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16u(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The double of a float that holds an integer (|x| < 2^24 here, so no
// subnormals), from its bits by integer operations alone: the FP64 pipe (1/64
// of the FP32 rate) is what the level sums are short of.  Zero keeps its sign.
__device__ __forceinline__ double int_float_to_double(uint32_t u) {
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  const uint32_t hi = (u & 0x80000000u) | ((((u >> 23) & 0xffu) + 896u) << 20) | ((u >> 3) & 0xfffffu);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// fl(x) for |x| < 2^63, rounded to nearest even, by integer operations alone
// (the value __ll2double_rn gives, off the FP64 pipe).
__device__ __forceinline__ double ll_to_double_rn(long long x) {
  if (x == 0) return 0.0;
  const unsigned long long sgn = x < 0 ? 0x8000000000000000ULL : 0ULL;
  const unsigned long long a = x < 0 ? 0ULL - (unsigned long long)x : (unsigned long long)x;
  int e = 63 - __clzll((long long)a);  // a in [2^e, 2^(e+1))
  unsigned long long mant;
  if (e <= 52) {
    mant = a << (52 - e);
  } else {
    const int sh = e - 52;
    mant = a >> sh;
    const unsigned long long rem = a & ((1ULL << sh) - 1ULL), half = 1ULL << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ULL))) ++mant;
    if (mant == (1ULL << 53)) {
      mant >>= 1;
      ++e;
    }
  }
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 1023) << 52) | (mant & ((1ULL << 52) - 1ULL))));
}

// 2^e as a double for e in the normal range, else 0 or infinity by ldexp.
__device__ __forceinline__ double pow2d(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

__global__ void __launch_bounds__(kOzThreads, 1)
ozaki_fused_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m, int n,
                   int kp, int s, int beta, int d0, const int* __restrict__ E, const int* __restrict__ F,
                   double* __restrict__ C, int64_t ldc, int tiles_m, int tiles_n, int* err, int* tile_ctr) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOzStages * kOzStageBytes);
  uint64_t* empty = full + kOzStages;
  uint64_t* acc_full = empty + kOzStages;   // [2]
  uint64_t* acc_empty = acc_full + 2;       // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  TileSched sch;  // every tile, in a static or (with tile_ctr) a shared dynamic schedule
  sch.ctr = tile_ctr;
  sch.lo = 0;
  sch.hi = tiles_m * tiles_n;
  sch.slot = reinterpret_cast<volatile int*>(tmem_slot + 2);
  sch.sfull = reinterpret_cast<uint64_t*>(tmem_slot + 2 + kSchedSlots);
  sch.sempty = sch.sfull + kSchedSlots;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kpsteps = kp / 64;  // K steps of 64 BF16 per slice

  if (threadIdx.x == 0) {
    for (int q = 0; q < kOzStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kEpiWarps);
    }
    for (int q = 0; q < kSchedSlots; ++q) {
      mbar_init(&sch.sfull[q], 1);
      mbar_init(&sch.sempty[q], 1 + kEpiWarps);  // MMA thread and epilogue warps
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer: for every tile, levels s+1 .. 2, their K steps
    const uint64_t keep = policy_evict_last();
    int g = 0;
    bool ok = true;
    for (int i = 0, t; ok && sch.claim(i, &t, abort, err); ++i) {
      int tm, tn;
      tile_coords(t, tiles_m, tiles_n, 0, &tm, &tn);
      for (int d = s + 1; d >= 2 && ok; --d) {
        const int nk = (d - 1) * kpsteps;
        const int xb0 = (s - d + 1) * kp;
        for (int ks = 0; ks < nk; ++ks, ++g) {
          const int q = g % kOzStages, round = g / kOzStages;
          if (round > 0 && !mbar_wait(&empty[q], (round - 1) & 1, abort, err)) { ok = false; break; }
          uint8_t* a = smem + q * kOzStageBytes;
          uint8_t* b = a + kStageA;
          mbar_expect_tx(&full[q], kOzStageBytes);
          tma_load_2d(a, &tmA, &full[q], ks * 64, tm * kBM, keep);
          tma_load_2d(b, &tmB, &full[q], xb0 + ks * 64, tn * kOzBN, keep);
        }
      }
    }
    if (*abort) {  // wait (bounded) for the copies still in flight
      for (int q = (g > kOzStages ? g - kOzStages : 0); q < g; ++q) {
        unsigned long long t0 = now_ns();
        while (!mbar_try_wait(&full[q % kOzStages], (q / kOzStages) & 1) && now_ns() - t0 < kWaitLimitNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: level lv of this CTA into accumulator lv % 2
    int g = 0, lv = 0;
    bool ok = true;
    for (int i = 0, t; ok && sch.next(i, &t, abort, err); ++i) {
      for (int d = s + 1; d >= 2 && ok; --d, ++lv) {
        const int abuf = lv & 1, use = lv >> 1;
        if (use > 0 && !mbar_wait(&acc_empty[abuf], (use - 1) & 1, abort, err)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + (uint32_t)(abuf * kOzBN);
        const int nk = (d - 1) * kpsteps;
        for (int ks = 0; ks < nk; ++ks, ++g) {
          const int q = g % kOzStages;
          if (!mbar_wait(&full[q], (g / kOzStages) & 1, abort, err)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint8_t* a = smem + q * kOzStageBytes;
          const uint8_t* b = a + kStageA;
          const uint64_t ad = smem_desc_sw128(a), bd = smem_desc_sw128(b);
#pragma unroll
          for (int k = 0; k < 4; ++k) mma<0>(dacc, ad + 2 * k, bd + 2 * k, kOzIdesc, (ks > 0 || k > 0) ? 1u : 0u);
          mma_commit(&empty[q]);
        }
        if (ok) mma_commit(&acc_full[abuf]);
      }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: warp (lane quarter qq, column half h) owns rows
    // 32 qq .. 32 qq + 31 and columns 64 h .. 64 h + 63 of the tile; its level
    // sum is 64 doubles per lane at TMEM columns 256 + 128 h ..
    const int qq = warp & 3;
    const int half = (warp - 2) >> 2;
    const double down = pow2d(-beta);
    const double first_fp = pow2d(-(s + 2 - d0) * beta);  // weight of fl(T) at level d0 - 1
    const double all_int = pow2d(-(s - 1) * beta);        // weight of fl(T) when every level is integer
    int lv = 0;
    bool ok = true;
    for (int i = 0; ok; ++i) {
      int t = 0, have = 0;
      if (lane == 0) have = sch.next(i, &t, abort, err) ? 1 : 0;
      have = __shfl_sync(0xffffffffu, have, 0);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (!have) break;
      int tm, tn;
      tile_coords(t, tiles_m, tiles_n, 0, &tm, &tn);
      const int row = tm * kBM + qq * 32 + lane;
      const int er = row < m ? E[row] : 0;
      const uint32_t lanebase = tmem + ((uint32_t)(qq * 32) << 16);
      for (int d = s + 1; d >= 2; --d, ++lv) {
        const int abuf = lv & 1, use = lv >> 1;
        int ready = 0;
        if (lane == 0) ready = mbar_wait(&acc_full[abuf], use & 1, abort, err) ? 1 : 0;
        ready = __shfl_sync(0xffffffffu, ready, 0);
        if (!ready) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // 16 columns at a time: the level (16 words), the running sum (32
        // words) and, at the last level, 16 entries of C in flight
#pragma unroll 1
        for (int cc = 0; cc < 4; ++cc) {
          const uint32_t tacc = lanebase + (uint32_t)(abuf * kOzBN + half * 64 + cc * 16);
          const uint32_t tsum = lanebase + (uint32_t)(2 * kOzBN + half * 128 + cc * 32);
          uint32_t v[16];
          tmem_ld16u(tacc, v);
          uint32_t w[32];  // the running sum: int64 T (levels >= d0) or FP64 S, lo/hi words
          if (d < s + 1) tmem_ld32u(tsum, w);
          if (d >= d0) {
            const int sh = (s + 1 - d) * beta;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              unsigned long long T = d == s + 1 ? 0ULL : (((unsigned long long)w[2 * i + 1] << 32) | w[2 * i]);
              // |P_d| <= 2^24 converts exactly; two's complement sums wrap-free (|T| < 2^63)
              T += (unsigned long long)(long long)__float2int_rn(__uint_as_float(v[i])) << sh;
              w[2 * i] = (uint32_t)T;
              w[2 * i + 1] = (uint32_t)(T >> 32);
            }
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const double P = int_float_to_double(v[i]);  // exact: P_d is an integer below 2^24
              double S;
              if (d == d0 - 1) {
                const long long T = (long long)(((unsigned long long)w[2 * i + 1] << 32) | w[2 * i]);
                S = fma(ll_to_double_rn(T), first_fp, P);
              } else {
                S = fma(__hiloint2double((int)w[2 * i + 1], (int)w[2 * i]), down, P);
              }
              w[2 * i] = (uint32_t)__double2loint(S);
              w[2 * i + 1] = (uint32_t)__double2hiint(S);
            }
          }
          if (d > 2) {
            tmem_st32(tsum, w);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          } else if (row < m) {
            // last level: C -= 2^(E_r + F_c - 2 beta) S, C read and written once;
            // S is fl(T) 2^-((s-1) beta) when every level is integer (d0 == 2)
            const double wgt = d0 == 2 ? all_int : 1.0;
            const int col0 = tn * kOzBN + half * 64 + cc * 16;
            double* cp = C + (int64_t)row + (int64_t)col0 * ldc;
            const int cn = min(16, n - col0);
            double old[16];
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (i < cn) old[i] = cp[(int64_t)i * ldc];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              if (i >= cn) continue;
              const double S = d0 == 2 ? ll_to_double_rn((long long)(((unsigned long long)w[2 * i + 1] << 32) | w[2 * i]))
                                       : __hiloint2double((int)w[2 * i + 1], (int)w[2 * i]);
              const double sc = pow2d(er + F[col0 + i] - 2 * beta);
              cp[(int64_t)i * ldc] = fma(-(d0 == 2 ? sc * wgt : sc), S, old[i]);
            }
          }
        }
        // this warp has read its part of the accumulator: hand it back
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[abuf]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int get_encoder(EncodeTiledFn* fn) {
  static EncodeTiledFn cached = nullptr;
  if (!cached) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    HPL_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) return set_error(HPL_ERR_NOTSUP, "cuTensorMapEncodeTiled unavailable");
    cached = reinterpret_cast<EncodeTiledFn>(p);
  }
  *fn = cached;
  return HPL_OK;
}

// rows x kp (elements of 1 or 2 bytes), row pitch `pitch` elements (kp when
// 0); box = (128 B of K) x box_rows with the 128-byte swizzle, or (64 B of K)
// x box_rows with the 64-byte swizzle (sw64); out-of-range elements read as
// zero.
int make_kmajor_map(CUtensorMap* map, const void* base, int64_t rows, int64_t kp, int elem_bytes, int box_rows,
                    bool sw64 = false, int64_t pitch = 0) {
  EncodeTiledFn enc;
  HPL_TRY(get_encoder(&enc));
  if (pitch == 0) pitch = kp;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((pitch * elem_bytes) & 15) || pitch < kp)
    return set_error(HPL_ERR_NOTSUP, "tensor map: base or pitch not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch * elem_bytes)};
  cuuint32_t box[2] = {(cuuint32_t)((sw64 ? 64 : 128) / elem_bytes), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   sw64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(HPL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return HPL_OK;
}

// C (m x n FP32, column-major, ldc): boxes of 32 rows x 32 columns, no
// swizzle; reads beyond the edge return zero, writes beyond it are dropped.
int make_c_map(CUtensorMap* map, float* C, int64_t m, int64_t n, int64_t ldc) {
  EncodeTiledFn enc;
  HPL_TRY(get_encoder(&enc));
  cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)(ldc * 4)};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(HPL_ERR_CUDA, "cuTensorMapEncodeTiled (C) failed (%d)", (int)r);
  return HPL_OK;
}

template <int KIND, bool CT, bool X3 = false>
int launch_ct(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc, int m, int n, int ksteps,
              int nterm, uint32_t sched, int kpiece, int store, int tri, float* C, int64_t ldc, const int* eL,
              const int* eU, int tiles_m, int tiles_n, int grid, int* err, unsigned* amax, int amax_by,
              cudaStream_t s, int tile_lo, int tile_hi, int* tile_ctr) {
  constexpr int smem = smem_of(CT, X3);
  HPL_TRY(set_smem_attr((const void*)mxp_gemm_kernel<KIND, CT, X3>, smem));
  mxp_gemm_kernel<KIND, CT, X3><<<grid, threads_of(CT), smem, s>>>(ta, tb, tc, m, n, ksteps, nterm, sched, kpiece, store,
                                                                tri, C, ldc, eL, eU, tiles_m, tiles_n, err, amax,
                                                                amax_by, tile_lo, tile_hi, tile_ctr);
  count_launch();
  return check_launch("mxp_gemm_kernel");
}

// The SM-pair kernel: with HPLGB_MXP_PAIR=1.
bool pair_enabled() {
  const char* e = getenv("HPLGB_MXP_PAIR");
  return e && e[0] == '1';
}

template <int KIND>
int launch_pair(const CUtensorMap& ta, const void* qU, const CUtensorMap& tc, int m, int n, int kp, int ksteps,
                const int* eL, const int* eU, int num_sms, int* err, cudaStream_t s) {
  const int eb = KIND == 0 ? 2 : 1;
  CUtensorMap tb;
  HPL_TRY(make_kmajor_map(&tb, qU, n, kp, eb, kPairBN));
  const int ptiles_m = (m + 2 * kBM - 1) / (2 * kBM), tiles_n = (n + kBN - 1) / kBN;
  const int64_t nptiles = (int64_t)ptiles_m * tiles_n;
  int pairs = (int)(nptiles < num_sms / 2 ? nptiles : num_sms / 2);
  if (pairs < 1) pairs = 1;
  HPL_TRY(set_smem_attr((const void*)mxp_gemm_pair_kernel<KIND>, kPairSmem));
  mxp_gemm_pair_kernel<KIND><<<2 * pairs, kPairThreads, kPairSmem, s>>>(ta, tb, tc, m, n, ksteps, eL, eU, ptiles_m,
                                                                        tiles_n, err);
  count_launch();
  return check_launch("mxp_gemm_pair_kernel");
}

template <int KIND>
int launch_kind(int m, int n, int kp, int nterm, uint32_t sched, int kpiece, int store, int tri, const void* qL,
                const void* qU, const int* eL, const int* eU, float* C, int64_t ldc, int* err, cudaStream_t s,
                unsigned* amax = nullptr, int amax_by = 0, int64_t pitch = 0, int max_ctas = 0, int tile_lo = 0,
                int tile_hi = -1, int* tile_ctr = nullptr) {
  const int eb = KIND == 0 ? 2 : 1;
  // BF16 products of three pieces that only store C: all pieces of a K slice per stage
  const bool x3 = KIND == 0 && store && nterm == 6;
  CUtensorMap ta, tb, tc;
  HPL_TRY(make_kmajor_map(&ta, qL, m, kp, eb, kBM, x3, pitch));
  HPL_TRY(make_kmajor_map(&tb, qU, n, kp, eb, kBN, x3, pitch));
  // The TMA epilogue pays for its C slots with an operand stage; a product
  // that only stores C (store mode) keeps the fourth stage and stores from
  // registers.
  const bool ct = !store && (ldc % 4) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0 && m >= 32 && n >= 32 &&
                  !getenv("HPLGB_MXP_REG_EPILOGUE");
  if (ct) HPL_TRY(make_c_map(&tc, C, m, n, ldc));
  else memset(&tc, 0, sizeof(tc));
  const int ksteps = (kpiece * eb) / (x3 ? kX3SliceBytes : 128);
  const int tiles_m = (m + kBM - 1) / kBM, tiles_n = (n + kBN - 1) / kBN;
  static int num_sms = 0;
  if (!num_sms) {
    int dev = 0;
    HPL_CUDA(cudaGetDevice(&dev));
    HPL_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t ntiles = (int64_t)tiles_m * tiles_n;
  if (ntiles > 0x7fffffff) return set_error(HPL_ERR_NOTSUP, "mxp gemm: too many tiles");
  if (tile_hi < 0 || tile_hi > ntiles) tile_hi = (int)ntiles;
  if (tile_lo < 0) tile_lo = 0;
  if (tile_lo >= tile_hi) return HPL_OK;
  const int span = tile_hi - tile_lo;
  int grid = span < num_sms ? span : num_sms;  // persistent: one CTA per SM
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  // the whole trailing update, statically scheduled: on SM pairs
  if (ct && !x3 && nterm == 1 && tri == 0 && !tile_ctr && tile_lo == 0 && tile_hi == ntiles && max_ctas == 0 &&
      !amax_by && pitch == 0 && kpiece == kp && pair_enabled())
    return launch_pair<KIND>(ta, qU, tc, m, n, kp, ksteps, eL, eU, num_sms, err, s);
  if (ct)
    return launch_ct<KIND, true>(ta, tb, tc, m, n, ksteps, nterm, sched, kpiece, store, tri, C, ldc, eL, eU,
                                 tiles_m, tiles_n, grid, err, amax, amax_by, s, tile_lo, tile_hi, tile_ctr);
  if (KIND == 0 && x3)
    return launch_ct<KIND, false, KIND == 0>(ta, tb, tc, m, n, ksteps, nterm, sched, kpiece, store, tri, C, ldc, eL,
                                             eU, tiles_m, tiles_n, grid, err, amax, amax_by, s, tile_lo, tile_hi,
                                             tile_ctr);
  return launch_ct<KIND, false>(ta, tb, tc, m, n, ksteps, nterm, sched, kpiece, store, tri, C, ldc, eL, eU,
                                tiles_m, tiles_n, grid, err, amax, amax_by, s, tile_lo, tile_hi, tile_ctr);
}

}  // namespace

int launch_mxp_gemm(int prec, int64_t m, int64_t n, int64_t kp, const void* qL, const void* qU, const int* eL,
                    const int* eU, float* C, int64_t ldc, int* err, cudaStream_t s) {
  if (m <= 0 || n <= 0 || kp <= 0) return HPL_OK;
  const int eb = prec == 0 ? 2 : 1;
  if ((kp * eb) % 128) return set_error(HPL_ERR_NOTSUP, "mxp gemm: K pitch must be a multiple of 128 bytes");
  if (m > 0x7fffffff || n > 0x7fffffff) return set_error(HPL_ERR_NOTSUP, "mxp gemm: too large");
  if (prec == 0) return launch_kind<0>((int)m, (int)n, (int)kp, 1, 0u, (int)kp, 0, 0, qL, qU, eL, eU, C, ldc, err, s);
  return launch_kind<1>((int)m, (int)n, (int)kp, 1, 0u, (int)kp, 0, 0, qL, qU, eL, eU, C, ldc, err, s);
}

// Tiles tile_lo .. tile_hi - 1 (of ceil(m/128) ceil(n/256), in the kernel's
// order) of the trailing update of launch_mxp_gemm, on at most max_ctas CTAs
// (0: one per SM).  With tile_ctr (a zeroed int in device memory) the CTAs
// claim the tiles from that counter as they go, and several launches that
// share it (on different streams) share the tiles: the mixed-precision
// look-ahead runs the trailing update on the SMs the next panel's diagonal
// kernel leaves free and adds a launch on the rest when that kernel ends.
int mxp_update_tiles(int64_t m, int64_t n) { return (int)(((m + kBM - 1) / kBM) * ((n + kBN - 1) / kBN)); }

int launch_mxp_gemm_part(int prec, int64_t m, int64_t n, int64_t kp, const void* qL, const void* qU, const int* eL,
                         const int* eU, float* C, int64_t ldc, int* err, cudaStream_t s, int tile_lo, int tile_hi,
                         int max_ctas, int* tile_ctr) {
  if (m <= 0 || n <= 0 || kp <= 0) return HPL_OK;
  const int eb = prec == 0 ? 2 : 1;
  if ((kp * eb) % 128) return set_error(HPL_ERR_NOTSUP, "mxp gemm: K pitch must be a multiple of 128 bytes");
  if (m > 0x7fffffff || n > 0x7fffffff) return set_error(HPL_ERR_NOTSUP, "mxp gemm: too large");
  if (prec == 0)
    return launch_kind<0>((int)m, (int)n, (int)kp, 1, 0u, (int)kp, 0, 0, qL, qU, eL, eU, C, ldc, err, s, nullptr, 0, 0,
                          max_ctas, tile_lo, tile_hi, tile_ctr);
  return launch_kind<1>((int)m, (int)n, (int)kp, 1, 0u, (int)kp, 0, 0, qL, qU, eL, eU, C, ldc, err, s, nullptr, 0, 0,
                        max_ctas, tile_lo, tile_hi, tile_ctr);
}

// P = A B (store mode, FP32) for BF16 operands whose rows hold K-concatenated
// pieces: qa (m rows) and qb (n rows), each row `pitch` elements apart, of
// which the first kext (a multiple of 64) enter the product.  With operands
// that are integers of at most 8 significant bits and products whose sums
// stay below 2^24 in magnitude, every accumulation in FP32 is exact, so P
// holds the exact integer product (the slice levels of the emulated FP64
// update, ozaki.cu).  ezero: zero exponents, at least max(m, n) / 128 + 1.
int launch_level_product(int64_t m, int64_t n, int64_t kext, int64_t pitch, const void* qa, const void* qb,
                         const int* ezero, float* P, int64_t ldp, int* err, cudaStream_t s) {
  if (m <= 0 || n <= 0 || kext <= 0) return HPL_OK;
  if (kext % 64 || pitch % 64 || pitch < kext) return set_error(HPL_ERR_NOTSUP, "level product: K extent or pitch");
  if (m > 0x7fffffff || n > 0x7fffffff || pitch > 0x7fffffff) return set_error(HPL_ERR_NOTSUP, "level product: too large");
  return launch_kind<0>((int)m, (int)n, (int)kext, 1, 0u, (int)kext, 1, 0, qa, qb, ezero, ezero, P, ldp, err, s,
                        nullptr, 0, pitch);
}

// The fused emulated FP64 update (ozaki_fused_kernel): C (m x n FP64, ldc)
// -= 2^(E_r + F_c - 2 beta) sum_d 2^-((d-2) beta) P_d with the slices qa (m
// rows) and qb (n rows), row pitch s kp, kp a multiple of 64.
int ozaki_fused_footprint(int* smem, int* regs, int* threads) {
  cudaFuncAttributes fa;
  HPL_CUDA(cudaFuncGetAttributes(&fa, ozaki_fused_kernel));
  *smem = kOzSmem + (int)fa.sharedSizeBytes;
  *regs = fa.numRegs;
  *threads = kOzThreads;
  return HPL_OK;
}

int launch_ozaki_fused(int64_t m, int64_t n, int64_t kp, int s, int beta, int d0, const void* qa, const void* qb,
                       const int* E, const int* F, double* C, int64_t ldc, int* err, cudaStream_t st, int max_ctas,
                       int* tile_ctr) {
  if (m <= 0 || n <= 0 || kp <= 0) return HPL_OK;
  if (kp % 64 || s < 1 || s > 12) return set_error(HPL_ERR_NOTSUP, "fused emulated update: kp or s");
  if (m > 0x7fffffff || n > 0x7fffffff || (int64_t)s * kp > 0x7fffffff)
    return set_error(HPL_ERR_NOTSUP, "fused emulated update: too large");
  CUtensorMap ta, tb;
  HPL_TRY(make_kmajor_map(&ta, qa, m, (int64_t)s * kp, 2, kBM));
  HPL_TRY(make_kmajor_map(&tb, qb, n, (int64_t)s * kp, 2, kOzBN));
  const int tiles_m = (int)((m + kBM - 1) / kBM), tiles_n = (int)((n + kOzBN - 1) / kOzBN);
  int dev = 0, sms = 0;
  HPL_CUDA(cudaGetDevice(&dev));
  HPL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ntiles = (int64_t)tiles_m * tiles_n;
  if (ntiles > 0x7fffffff) return set_error(HPL_ERR_NOTSUP, "fused emulated update: too many tiles");
  int grid = (int)(ntiles < sms ? ntiles : sms);  // persistent: one CTA per SM
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  HPL_TRY(set_smem_attr((const void*)ozaki_fused_kernel, kOzSmem));
  ozaki_fused_kernel<<<grid, kOzThreads, kOzSmem, st>>>(ta, tb, (int)m, (int)n, (int)kp, s, beta, d0, E, F, C, ldc,
                                                        tiles_m, tiles_n, err, tile_ctr);
  count_launch();
  return check_launch("ozaki_fused_kernel");
}

// C = A B in FP32 accuracy from BF16 pieces: every operand row holds three
// BF16 pieces x = p0 + p1 + p2 (exact), each kpiece elements long.  The six
// products with piece-index sum <= 2 are accumulated in FP32 (smallest
// first); the three dropped ones are below 2^-24 |A||B|.  qL: m x 3 kpiece
// (rows of A), qU: n x 3 kpiece (columns of B); C column-major, overwritten.
// tri = 1 (A lower triangular) or 2 (B upper triangular) stops each tile's K
// loop at the triangle's edge.  With amax_by = 1 (2) the maxima of |C| over
// each 128-row tile (128-column group) of C are atomicMax-ed into amax, as
// non-negative float bit patterns (amax zeroed by the caller).
int launch_gemm_x3(int64_t m, int64_t n, int64_t kpiece, const void* qL, const void* qU, const int* ezero, float* C,
                   int64_t ldc, int tri, int* err, cudaStream_t s, unsigned* amax, int amax_by) {
  if (m <= 0 || n <= 0 || kpiece <= 0) return HPL_OK;
  if ((kpiece * 2) % 128) return set_error(HPL_ERR_NOTSUP, "x3 gemm: piece length must be a multiple of 64");
  if (m > 0x7fffffff || n > 0x7fffffff || 3 * kpiece > 0x7fffffff) return set_error(HPL_ERR_NOTSUP, "x3 gemm: too large");
  // (pa, pb) per term, 4 bits each: (1,1) (0,2) (2,0) (0,1) (1,0) (0,0)
  const uint32_t pair[6][2] = {{1, 1}, {0, 2}, {2, 0}, {0, 1}, {1, 0}, {0, 0}};
  uint32_t sched = 0;
  for (int t = 0; t < 6; ++t) sched |= (pair[t][0] | (pair[t][1] << 2)) << (4 * t);
  return launch_kind<0>((int)m, (int)n, (int)(3 * kpiece), 6, sched, (int)kpiece, 1, tri, qL, qU, ezero, ezero, C,
                        ldc, err, s, amax, amax_by);
}

}  // namespace hplgb
