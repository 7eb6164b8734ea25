// panel.cu -- FACT (Sec. I; Sec. III-A): LU with partial pivoting of a tall
// m x w panel, on the GPU.
//
// Recursive right-looking with two subdivisions (Sec. III-A: "two
// subdivisions in the recursion", base block 16, right-looking base):
//   factor the left half; apply its interchanges to the right half; U12 <-
//   L11^-1 A12 (trsm); A22 -= A21 A12 (gemm); factor the right half; apply its
//   interchanges to the left half.
// The base (w <= 16 columns) is one kernel of G cooperating CTAs.  The paper's
// CPU version splits the panel into row tiles owned by threads (Fig. 4) and
// reduces each pivot over threads then processes; here each CTA owns a
// contiguous block of rows and the per-column pivot search is a warp-shuffle
// argmax, then a CTA reduction, then a grid-wide reduction through published
// candidates.  One grid barrier per column: at the end of column j every CTA
// publishes its best candidate for column j+1 together with that row's values
// (and the owner of row j+1 publishes row j+1), so after the barrier every CTA
// knows the pivot row and the row it displaces without reading rows another
// CTA may be writing.  Candidate slots are double-buffered by column parity.
//
// The barrier is a monotone 64-bit counter in global memory with a bounded
// wait: a CTA that has waited ~2 s records DEV_TIMEOUT and returns (the host
// reads it through hpl_sync_check); nothing in this kernel can spin forever.
#include <stdlib.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace hplgb {

namespace {

constexpr int kBaseMaxW = 16;
constexpr int kPanelThreads = 256;
constexpr int kSlotStride = 2 + kBaseMaxW;   // |value|, row index, row values
constexpr int kMaxGrid = 160;                // CTAs of one base launch (one per SM at most)
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ULL;  // default limit of one wait

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier: returns false (and records DEV_TIMEOUT) if it gave up.
__device__ bool grid_barrier(unsigned long long* ctr, unsigned long long target, int* err,
                             int* s_flag, unsigned long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(ctr, 1ULL);
    unsigned long long t0 = globaltimer_ns();
    unsigned spins = 0;
    while (ld_acquire_u64(ctr) < target) {
      if (++spins > 64) __nanosleep(64);
      if ((spins & 255) == 0) {
        if (*(volatile int*)err == DEV_TIMEOUT || globaltimer_ns() - t0 > timeout_ns) {
          atomicExch(err, DEV_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    *s_flag = ok;  // the acquire loads above order this CTA's later reads after the barrier
  }
  __syncthreads();
  return *s_flag != 0;
}

struct BaseArgs {
  int64_t m;          // rows of the panel block
  int w;              // columns (<= kBaseMaxW)
  double* P;          // block, column-major
  int64_t lda;
  int32_t* ipiv;      // w entries, value = ipiv_shift + local row + 1
  int64_t ipiv_shift;
  int32_t* info;      // may be null
  int64_t info_shift;
  double* slots;      // [2][G][kSlotStride] then [2][kBaseMaxW] for row j+1
  unsigned long long* bar;
  unsigned long long bar_base;
  unsigned long long timeout_ns;  // limit of each grid-barrier wait
  int extra_arrivals;             // test knob: arrivals awaited beyond the grid (0 in use)
  int* err;
  int64_t rows_per_cta;
};

// Block-wide argmax of (v, idx): larger v wins, equal v -> smaller idx.
// Returns the winner in (*bv, *bi) for all threads.  Requires red arrays of
// kPanelThreads/32 entries.
__device__ __forceinline__ void cta_argmax(double v, int64_t idx, double* red_v, int64_t* red_i,
                                           double* bv, int64_t* bi) {
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, off);
    int64_t oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { red_v[w] = v; red_i[w] = idx; }
  __syncthreads();
  if (w == 0) {
    v = (l < kPanelThreads / 32) ? red_v[l] : -2.0;
    idx = (l < kPanelThreads / 32) ? red_i[l] : INT64_MAX;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, v, off);
      int64_t oi = __shfl_xor_sync(0xffffffffu, idx, off);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (l == 0) { red_v[0] = v; red_i[0] = idx; }
  }
  __syncthreads();
  *bv = red_v[0];
  *bi = red_i[0];
  __syncthreads();
}

__global__ void __launch_bounds__(kPanelThreads)
panel_base_kernel(BaseArgs a) {
  // This CTA's rows of the w panel columns, resident in shared memory for the
  // whole kernel: S[c * rs + r] holds P(rb + r, c) (column-major, so threads on
  // consecutive rows touch consecutive words).
  extern __shared__ double S[];
  __shared__ double prow[kBaseMaxW];
  __shared__ double jrow[kBaseMaxW];
  __shared__ double red_v[kPanelThreads / 32];
  __shared__ int64_t red_i[kPanelThreads / 32];
  __shared__ int s_flag;
  // every CTA's published candidate of the current column, and row jj (one
  // load round trip for the whole grid's candidates instead of a strided
  // search followed by a second trip for the pivot row)
  __shared__ double s_slots[kMaxGrid * kSlotStride];
  __shared__ double s_jrow[kBaseMaxW];

  const int G = gridDim.x;
  const int g = blockIdx.x;
  const int t = threadIdx.x;
  const int64_t m = a.m;
  const int w = a.w;
  const int64_t lda = a.lda;
  double* P = a.P;
  const int rs = (int)a.rows_per_cta;
  const int64_t rb = (int64_t)g * rs;
  const int64_t re = min(m, rb + rs);
  const int nloc = re > rb ? (int)(re - rb) : 0;
  double* slot_base = a.slots;
  double* jslot_base = a.slots + 2 * (int64_t)G * kSlotStride;
  unsigned long long target = a.bar_base;

  for (int c = 0; c < w; ++c)
    for (int r = t; r < nloc; r += kPanelThreads) S[c * rs + r] = P[(rb + r) + c * lda];
  __syncthreads();

  // publish this CTA's candidate for column `col` (rows >= col) and, if owned,
  // row `col` itself, into parity buffer `par`
  // (with scanned = true the thread's candidate v, idx was taken during the
  // update that produced the column)
  auto publish = [&](int col, int par, bool scanned, double v, int64_t idx) {
    if (!scanned) {
      v = -1.0;
      idx = INT64_MAX;
      const int r0 = col > rb ? (int)(col - rb) : 0;
      for (int r = r0 + t; r < nloc; r += kPanelThreads) {
        double x = fabs(S[col * rs + r]);
        if (x > v) { v = x; idx = rb + r; }  // rows ascend per thread: first maximum kept
      }
    }
    double bv;
    int64_t bi;
    cta_argmax(v, idx, red_v, red_i, &bv, &bi);
    double* slot = slot_base + ((int64_t)par * G + g) * kSlotStride;
    if (t == 0) {
      slot[0] = bv;
      slot[1] = (bi == INT64_MAX) ? -1.0 : (double)bi;
    }
    if (bi != INT64_MAX && t < w) slot[2 + t] = S[t * rs + (int)(bi - rb)];
    if (col >= rb && col < re && t < w) jslot_base[par * kBaseMaxW + t] = S[t * rs + (int)(col - rb)];
  };

  publish(0, 0, false, 0.0, 0);
  target += G;
  if (!grid_barrier(a.bar, target + a.extra_arrivals, a.err, &s_flag, a.timeout_ns)) return;

  for (int jj = 0; jj < w; ++jj) {
    const int par = jj & 1;
    {
      const double* src = slot_base + (int64_t)par * G * kSlotStride;
      const int tot = G * kSlotStride;
#pragma unroll 4
      for (int i = t; i < tot; i += kPanelThreads) s_slots[i] = __ldcg(src + i);
      if (t < w) s_jrow[t] = __ldcg(jslot_base + par * kBaseMaxW + t);
    }
    __syncthreads();
    // grid-wide argmax over the published candidates, the pivot row and the
    // interchange in this CTA's rows: all by warp 0 (w <= 16 lanes hold the
    // row values), so one CTA barrier follows instead of three
    if (t < 32) {
      double v = -2.0;
      int64_t idx = INT64_MAX;
      for (int q = t; q < G; q += 32) {
        const double* sl = s_slots + q * kSlotStride;
        double ov = sl[0];
        double oid = sl[1];
        int64_t oi = oid < 0 ? INT64_MAX : (int64_t)oid;
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
      }
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, off);
        int64_t oi = __shfl_xor_sync(0xffffffffu, idx, off);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
      }
      // every lane holds the same winner
      if (idx == INT64_MAX || idx < jj || idx >= m) { idx = jj; v = -1.0; }  // no usable candidate
      const int64_t pw = idx;
      // the pivot row's values: from the winning CTA's slot, or (no usable
      // candidate, e.g. NaN column) row jj itself
      if (t < w) {
        prow[t] = v >= 0.0 ? s_slots[(pw / rs) * kSlotStride + 2 + t] : s_jrow[t];
        jrow[t] = s_jrow[t];
      }
      __syncwarp();
      if (g == 0 && t == 0) {
        a.ipiv[jj] = (int32_t)(a.ipiv_shift + pw + 1);
        if (a.info && prow[jj] == 0.0) atomicCAS(a.info, 0, (int32_t)(a.info_shift + jj + 1));
      }
      // interchange rows jj and p within the block's w columns
      if (pw != jj && t < w) {
        if (jj >= rb && jj < re) S[t * rs + (int)(jj - rb)] = prow[t];
        if (pw >= rb && pw < re) S[t * rs + (int)(pw - rb)] = jrow[t];
      }
    }
    __syncthreads();
    const double piv = prow[jj];
    // the next column's candidate of this thread, taken as the update writes it
    double nv = -1.0;
    int64_t ni = INT64_MAX;
    const bool scan_in_update = piv != 0.0 && jj + 1 < w;
    if (piv != 0.0) {
      // multipliers by the reciprocal of the pivot (within one ulp of a
      // division), then the rank-1 update of the remaining base columns
      const double rinv = 1.0 / piv;
      const int r0 = jj + 1 > rb ? (int)(jj + 1 - rb) : 0;
      for (int r = r0 + t; r < nloc; r += kPanelThreads) {
        const double l = S[jj * rs + r] * rinv;
        S[jj * rs + r] = l;
        if (jj + 1 < w) {
          const double x = fma(-l, prow[jj + 1], S[(jj + 1) * rs + r]);
          S[(jj + 1) * rs + r] = x;
          if (fabs(x) > nv) { nv = fabs(x); ni = rb + r; }  // rows ascend per thread: first maximum kept
        }
        for (int c = jj + 2; c < w; ++c) S[c * rs + r] = fma(-l, prow[c], S[c * rs + r]);
      }
    }
    if (jj + 1 < w) {
      if (!scan_in_update) __syncthreads();  // the scan below reads other threads' rows
      publish(jj + 1, par ^ 1, scan_in_update, nv, ni);
      target += G;
      if (!grid_barrier(a.bar, target + a.extra_arrivals, a.err, &s_flag, a.timeout_ns)) return;
    }
  }
  __syncthreads();
  for (int c = 0; c < w; ++c)
    for (int r = t; r < nloc; r += kPanelThreads) P[(rb + r) + c * lda] = S[c * rs + r];
}

// Largest number of rows one CTA can hold in shared memory for a w-column base.
constexpr int kPanelSmemBytes = 200 * 1024;
inline int64_t panel_max_rows(int w) { return kPanelSmemBytes / (8 * (w > 0 ? w : 1)); }

int panel_set_smem_attr() { return set_smem_attr((const void*)panel_base_kernel, kPanelSmemBytes); }

// Launch shape of the base kernel, shared by the workspace and the no-alloc
// entry points: enough CTAs that each owns about HPLGB_PANEL_ROWS rows (256
// by default), at most one CTA per SM and at most HPLGB_PANEL_CTAS, every CTA
// resident at once (the grid barrier needs them all).  The first call on a
// device checks that a CTA with the largest shared-memory footprint fits on
// an SM; a device where it does not is reported as HPL_ERR_NOTSUP instead of
// a barrier timeout.
// Limit of each grid-barrier wait (HPLGB_WAIT_TIMEOUT_MS, default 2000 ms),
// and the test knob HPLGB_TEST_EXTRA_ARRIVAL=1, under which every barrier of
// the base kernel waits for one arrival more than its grid makes, so the
// first wait of each launch runs out and the kernel records DEV_TIMEOUT and
// returns (the failure path of the bounded waits, exercised without a fault).
// Both are read on the host at every launch.
void panel_wait_settings(unsigned long long* timeout_ns, int* extra) {
  const char* t = getenv("HPLGB_WAIT_TIMEOUT_MS");
  long long ms = t ? atoll(t) : 0;
  *timeout_ns = (ms >= 1 && ms <= 60000) ? (unsigned long long)ms * 1000000ULL : kBarrierTimeoutNs;
  const char* e = getenv("HPLGB_TEST_EXTRA_ARRIVAL");
  *extra = (e && e[0] == '1') ? 1 : 0;
}

int check_resident_once() {
  static std::mutex mu;
  static std::vector<int> checked;  // per device: 0 unknown, 1 ok
  int dev = 0;
  HPL_CUDA(cudaGetDevice(&dev));
  HPL_TRY(panel_set_smem_attr());
  std::lock_guard<std::mutex> lk(mu);
  if ((int)checked.size() <= dev) checked.resize(dev + 1, 0);
  if (!checked[dev]) {
    int per_sm = 0;
    HPL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_base_kernel, kPanelThreads,
                                                           kPanelSmemBytes));
    if (per_sm < 1) return set_error(HPL_ERR_NOTSUP, "panel kernel cannot be resident");
    checked[dev] = 1;
  }
  return HPL_OK;
}

int panel_launch_shape(int num_sms, int64_t m, int w, int64_t* G_out, int64_t* rows_out) {
  static std::mutex mu;
  static int64_t rows_per = 0, cap_env = 0;
  HPL_TRY(check_resident_once());
  {
    std::lock_guard<std::mutex> lk(mu);
    if (rows_per == 0) {
      const char* e = getenv("HPLGB_PANEL_ROWS");
      rows_per = e ? atoll(e) : 256;
      if (rows_per < 32) rows_per = 32;
      const char* c = getenv("HPLGB_PANEL_CTAS");
      cap_env = c ? atoll(c) : 0;
    }
  }
  int64_t cap = num_sms < kMaxGrid ? num_sms : kMaxGrid;
  if (cap_env >= 1 && cap_env < cap) cap = cap_env;
  int64_t G = (m + rows_per - 1) / rows_per;
  if (G > cap) G = cap;
  if (G < 1) G = 1;
  int64_t rows = (m + G - 1) / G;
  G = (m + rows - 1) / rows;
  if (rows > panel_max_rows(w))
    return set_error(HPL_ERR_NOTSUP, "panel: %lld rows per CTA exceed shared memory", (long long)rows);
  *G_out = G;
  *rows_out = rows;
  return HPL_OK;
}

int launch_panel_base(Workspace* ws, int64_t m, int w, double* P, int64_t lda, int32_t* ipiv,
                      int64_t ipiv_shift, int32_t* info, int64_t info_shift, cudaStream_t s, int max_ctas) {
  int64_t G = 0, rows = 0;
  const int sms = max_ctas > 0 && max_ctas < ws->num_sms ? max_ctas : ws->num_sms;
  HPL_TRY(panel_launch_shape(sms, m, w, &G, &rows));
  if (ws->panel_slots_bytes < (size_t)(2 * G * kSlotStride + 2 * kBaseMaxW) * sizeof(double))
    return set_error(HPL_ERR_NOTSUP, "panel: candidate slots too small");
  BaseArgs a;
  a.m = m;
  a.w = w;
  a.P = P;
  a.lda = lda;
  a.ipiv = ipiv;
  a.ipiv_shift = ipiv_shift;
  a.info = info;
  a.info_shift = info_shift;
  a.slots = ws->panel_slots;
  a.bar = ws->bar;
  a.bar_base = ws->bar_next;
  panel_wait_settings(&a.timeout_ns, &a.extra_arrivals);
  a.err = ws->dev_err;
  a.rows_per_cta = rows;
  ws->bar_next += (unsigned long long)G * (unsigned long long)w;
  panel_base_kernel<<<(unsigned)G, kPanelThreads, (size_t)w * rows * sizeof(double), s>>>(a);
  count_launch();
  return check_launch("panel_base_kernel");
}

int panel_rec(Workspace* ws, int64_t m, int64_t w, double* A, int64_t lda, int32_t* ipiv,
              int64_t ipiv_shift, int32_t* info, int64_t info_shift, int slices, cudaStream_t s,
              int max_ctas) {
  if (w <= kBaseMaxW)
    return launch_panel_base(ws, m, (int)w, A, lda, ipiv, ipiv_shift, info, info_shift, s, max_ctas);
  int64_t w1 = (w / 2 + 7) / 8 * 8;
  if (w1 >= w) w1 = w / 2;
  const int64_t w2 = w - w1;
  HPL_TRY(panel_rec(ws, m, w1, A, lda, ipiv, ipiv_shift, info, info_shift, slices, s, max_ctas));
  // left half's interchanges on the right half's columns
  HPL_TRY(launch_laswp_fused(ipiv, 0, w1, ipiv_shift, m, false, w2, A + w1 * lda, lda, ws->dev_err, s));
  HPL_TRY(launch_trsm_llnu(w1, w2, A, lda, A + w1 * lda, lda, s));
  // the recursion's Schur update: FP64 DGEMM, or the emulated FP64 product
  // (slices >= 0) where it is wide enough to feed the tensor cores
  if (slices >= 0 && w1 >= 32 && m - w1 >= 256)
    HPL_TRY(launch_ozaki_gemm(m - w1, w2, w1, A + w1, lda, A + w1 * lda, lda, A + w1 + w1 * lda, lda, slices,
                              ws->dev_err, s, max_ctas));
  else
    HPL_TRY(launch_dgemm(false, false, m - w1, w2, w1, -1.0, A + w1, lda, A + w1 * lda, lda, 1.0,
                         A + w1 + w1 * lda, lda, s));
  HPL_TRY(panel_rec(ws, m - w1, w2, A + w1 + w1 * lda, lda, ipiv + w1, ipiv_shift + w1, info,
                    info_shift + w1, slices, s, max_ctas));
  // right half's interchanges on the left half's columns
  return launch_laswp_fused(ipiv, w1, w, ipiv_shift, m, false, w1, A, lda, ws->dev_err, s);
}

}  // namespace

size_t panel_slots_bytes_for(int num_sms) {
  return (size_t)(2 * (size_t)num_sms * kSlotStride + 2 * kBaseMaxW) * sizeof(double);
}

int panel_factor(Workspace* ws, int64_t m, int64_t w, double* A, int64_t lda, int32_t* ipiv,
                 int64_t ipiv_shift, int32_t* info, int64_t info_shift, cudaStream_t s, int slices,
                 int max_ctas) {
  if (m <= 0 || w <= 0) return HPL_OK;
  if (w > m) return set_error(HPL_ERR_NOTSUP, "panel wider than tall");
  return panel_rec(ws, m, w, A, lda, ipiv, ipiv_shift, info, info_shift, slices, s, max_ctas);
}

}  // namespace hplgb

namespace hplgb {

// The base-kernel launch of the recursion, with every piece of scratch given by
// the caller instead of taken from the per-device workspace: the candidate
// slots (slots_bytes of them), the grid-barrier counter `bar` whose next base
// value the caller tracks in *bar_next, and the device error word.  Same launch
// policy (rows per CTA, at most one CTA per SM) as the workspace path.
int launch_panel_base_scratch(int num_sms, int64_t m, int w, double* P, int64_t lda, int32_t* ipiv,
                              int64_t ipiv_shift, int32_t* info, int64_t info_shift, double* slots,
                              size_t slots_bytes, unsigned long long* bar, unsigned long long* bar_next,
                              int* err, cudaStream_t s) {
  if (w > kBaseMaxW) return set_error(HPL_ERR_NOTSUP, "panel base wider than %d", kBaseMaxW);
  int64_t G = 0, rows = 0;
  HPL_TRY(panel_launch_shape(num_sms, m, w, &G, &rows));
  if (slots_bytes < (size_t)(2 * G * kSlotStride + 2 * kBaseMaxW) * sizeof(double))
    return set_error(HPL_ERR_NOTSUP, "panel: candidate slots too small");
  BaseArgs a;
  a.m = m;
  a.w = w;
  a.P = P;
  a.lda = lda;
  a.ipiv = ipiv;
  a.ipiv_shift = ipiv_shift;
  a.info = info;
  a.info_shift = info_shift;
  a.slots = slots;
  a.bar = bar;
  a.bar_base = *bar_next;
  panel_wait_settings(&a.timeout_ns, &a.extra_arrivals);
  a.err = err;
  a.rows_per_cta = rows;
  *bar_next += (unsigned long long)G * (unsigned long long)w;
  panel_base_kernel<<<(unsigned)G, kPanelThreads, (size_t)w * rows * sizeof(double), s>>>(a);
  count_launch();
  return check_launch("panel_base_kernel");
}

int panel_base_max_width() { return kBaseMaxW; }

int panel_check_resident() { return check_resident_once(); }

int panel_base_footprint(int num_sms, int64_t m, int w, int64_t* ctas, int* smem, int* regs, int* threads) {
  int64_t G = 0, rows = 0;
  HPL_TRY(panel_launch_shape(num_sms, m, w, &G, &rows));
  cudaFuncAttributes fa;
  HPL_CUDA(cudaFuncGetAttributes(&fa, panel_base_kernel));
  *ctas = G;
  *smem = (int)fa.sharedSizeBytes + (int)((size_t)w * rows * sizeof(double));
  *regs = fa.numRegs;
  *threads = kPanelThreads;
  return HPL_OK;
}

}  // namespace hplgb
