// api.cu -- the C ABI of include/hplgb.h: argument checks, workspace, the
// getrf iteration driver (Sec. I phases FACT / RS / UPDATE, Sec. III
// look-ahead), and small utilities.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"

namespace hplgb {

// ------------------------------------------------------------------ errors
static thread_local char g_errmsg[512] = "no error";
static std::atomic<long long> g_launches{0};

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_errmsg, sizeof(g_errmsg), fmt, ap);
  va_end(ap);
  return code;
}

int fault_point(const char* site) {
  const char* f = getenv("HPLGB_FAULT");
  if (f && (strcmp(f, site) == 0 || strcmp(f, "all") == 0))
    return set_error(HPL_ERR_FAULT, "injected fault at %s (HPLGB_FAULT)", site);
  return HPL_OK;
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(HPL_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return HPL_OK;
}

// ------------------------------------------------ kernel attributes, memory
static std::mutex g_attr_mutex;
static std::map<std::pair<int, const void*>, int> g_attr_set;  // (device, kernel) -> bytes

int set_smem_attr(const void* fn, int bytes) {
  int dev = 0;
  HPL_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_attr_mutex);
  auto key = std::make_pair(dev, fn);
  auto it = g_attr_set.find(key);
  if (it != g_attr_set.end() && it->second >= bytes) return HPL_OK;
  HPL_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  g_attr_set[key] = bytes;
  return HPL_OK;
}

constexpr int kMaxCountedDevices = 64;
static std::atomic<long long> g_dev_bytes[kMaxCountedDevices];

static std::atomic<long long>* dev_counter() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxCountedDevices) return nullptr;
  return &g_dev_bytes[dev];
}

int dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(HPL_ERR_ALLOC, "device allocation of %zu bytes failed", bytes);
  }
  if (auto* c = dev_counter()) c->fetch_add((long long)bytes);
  return HPL_OK;
}

void dev_free(void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  if (auto* c = dev_counter()) c->fetch_sub((long long)bytes);
}

// --------------------------------------------------------------- workspace
static std::mutex g_ws_mutex;
static std::vector<Workspace*> g_ws;

static int grow(void** p, size_t* have, size_t want) {
  if (*have >= want) return HPL_OK;
  if (*p) {
    HPL_CUDA(cudaDeviceSynchronize());  // old buffer may be in use by queued work
    dev_free(*p, *have);
    *p = nullptr;
    *have = 0;
  }
  const size_t sz = (want + want / 4 + 255) / 256 * 256;  // a multiple of every element size
  HPL_TRY(dev_alloc(p, sz));
  *have = sz;
  return HPL_OK;
}

int get_workspace(Workspace** out) {
  int dev = 0;
  HPL_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_ws_mutex);
  if ((int)g_ws.size() <= dev) g_ws.resize(dev + 1, nullptr);
  if (!g_ws[dev]) {
    HPL_TRY(fault_point("workspace"));
    Workspace* ws = new Workspace();
    ws->device = dev;
    HPL_CUDA(cudaDeviceGetAttribute(&ws->num_sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev_alloc((void**)&ws->dev_err, 64) != HPL_OK) {
      delete ws;
      return set_error(HPL_ERR_ALLOC, "cannot allocate the device error word");
    }
    HPL_CUDA(cudaMemset(ws->dev_err, 0, 64));
    ws->bar = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ws->dev_err) + 8);
    size_t sb = panel_slots_bytes_for(ws->num_sms);
    void* p = nullptr;
    size_t have = 0;
    HPL_TRY(grow(&p, &have, sb));
    ws->panel_slots = (double*)p;
    ws->panel_slots_bytes = have;
    int lo = 0, hi = 0;
    HPL_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    HPL_CUDA(cudaStreamCreateWithPriority(&ws->la_stream, cudaStreamNonBlocking, hi));
    for (auto& e : ws->ev) HPL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ws->events_ready = true;
    g_ws[dev] = ws;
  }
  *out = g_ws[dev];
  return HPL_OK;
}

int ensure_perm(Workspace* ws, size_t ints) {
  size_t have = ws->perm_ints * sizeof(int32_t);
  void* p = ws->perm;
  HPL_TRY(grow(&p, &have, ints * sizeof(int32_t)));
  ws->perm = (int32_t*)p;
  ws->perm_ints = have / sizeof(int32_t);
  return HPL_OK;
}

int ensure_scratch(Workspace* ws, size_t bytes) {
  void* p = ws->scratch;
  HPL_TRY(grow(&p, &ws->scratch_bytes, bytes));
  ws->scratch = (double*)p;
  return HPL_OK;
}

static void free_workspace(Workspace* ws) {
  if (!ws) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(ws->device);
  cudaDeviceSynchronize();
  dev_free(ws->dev_err, 64);
  dev_free(ws->panel_slots, ws->panel_slots_bytes);
  dev_free(ws->perm, ws->perm_ints * sizeof(int32_t));
  dev_free(ws->scratch, ws->scratch_bytes);
  dev_free(ws->minv, ws->minv_bytes);
  dev_free(ws->tile_ctr, ws->tile_ctr_bytes);
  if (ws->la_stream) cudaStreamDestroy(ws->la_stream);
  if (ws->events_ready)
    for (auto& e : ws->ev) cudaEventDestroy(e);
  delete ws;
  cudaSetDevice(cur);
}

// ------------------------------------------------------------ phase timers
struct PhaseTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> evs;
  std::vector<int> phase;  // phase id of the interval ending at evs[i]
  double last[5] = {0, 0, 0, 0, 0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};
static PhaseTimer g_timer;

static void timer_mark(int phase_of_previous) {
  if (!g_timer.on) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, g_timer.s);
  g_timer.evs.push_back(e);
  g_timer.phase.push_back(phase_of_previous);
}

// --------------------------------------------- trailing-update event timing
// While enabled, every trailing-update launch (the DGEMMs of hpl_getrf, the
// tcgen05 updates of hpl_mxp_getrf) is bracketed by two CUDA events on the
// stream it runs on, with its algorithmic flops and bytes.
struct GemmTiming {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<double> flops, bytes;
};
static GemmTiming g_gt;

int gemm_timing_begin(cudaStream_t s) {
  if (!g_gt.on) return HPL_OK;
  while (g_gt.pool.size() < g_gt.used + 2) {
    cudaEvent_t e;
    HPL_CUDA(cudaEventCreate(&e));
    g_gt.pool.push_back(e);
  }
  HPL_CUDA(cudaEventRecord(g_gt.pool[g_gt.used], s));
  return HPL_OK;
}

int gemm_timing_end(cudaStream_t s, double flops, double bytes) {
  if (!g_gt.on) return HPL_OK;
  HPL_CUDA(cudaEventRecord(g_gt.pool[g_gt.used + 1], s));
  g_gt.used += 2;
  g_gt.flops.push_back(flops);
  g_gt.bytes.push_back(bytes);
  return HPL_OK;
}

// The trailing update C -= A B: the FP64 DGEMM (slices < 0), or the emulated
// FP64 update from BF16 slice products (slices >= 0; 0 = chosen per k).
static int update_gemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int slices, int* err, cudaStream_t s, int max_ctas,
                       const OzakiJoin* join) {
  if (slices < 0) return launch_dgemm(false, false, m, n, k, -1.0, A, lda, B, ldb, 1.0, C, ldc, s);
  return launch_ozaki_gemm(m, n, k, A, lda, B, ldb, C, ldc, slices, err, s, max_ctas, join);
}

// U12 <- L11^-1 U12 (L11 unit lower m x m): the FP64 blocked solve
// (slices < 0), or, with the emulated update, U12 <- U12 - M U12 with
// M = I - L11^-1 (strictly lower; made once per panel by u12_inverse) as one
// emulated FP64 product, so the solve too runs on the tensor cores.  The
// product splits U12 into slices before it writes U12, so in place is safe.
static int u12_solve(int64_t m, int64_t n, const double* L, int64_t ldl, double* B, int64_t ldb, int slices,
                     const double* M, int* err, cudaStream_t s, int max_ctas = 0) {
  if (slices < 0 || !M) return launch_trsm_llnu(m, n, L, ldl, B, ldb, s);
  return launch_ozaki_gemm(m, n, m, M, m, B, ldb, B, ldb, slices, err, s, max_ctas);
}

static int timed_gemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                      int64_t ldb, double* C, int64_t ldc, int slices, int* err, cudaStream_t s, int max_ctas = 0,
                      const OzakiJoin* join = nullptr) {
  if (!g_gt.on || m <= 0 || n <= 0 || k <= 0)
    return update_gemm(m, n, k, A, lda, B, ldb, C, ldc, slices, err, s, max_ctas, join);
  HPL_TRY(gemm_timing_begin(s));
  HPL_TRY(update_gemm(m, n, k, A, lda, B, ldb, C, ldc, slices, err, s, max_ctas, join));
  const double dm = (double)m, dn = (double)n, dk = (double)k;
  return gemm_timing_end(s, 2.0 * dm * dn * dk, 8.0 * (dm * dk + dk * dn + 2.0 * dm * dn));
}

void phase_timing_begin(cudaStream_t s) {
  const char* tv = getenv("HPLGB_TIMERS");
  for (auto e : g_timer.evs) cudaEventDestroy(e);
  g_timer.evs.clear();
  g_timer.phase.clear();
  g_timer.on = tv && tv[0] == '1';
  g_timer.s = s;
  timer_mark(-1);
}

void phase_mark(int phase_of_previous) { timer_mark(phase_of_previous); }

bool phase_timing_on() { return g_timer.on; }

// ---------------------------------------------------------------- getrf
constexpr int PH_NONE = -1;
// SMs left to FACT beside the emulated update (HPLGB_LA_SMS overrides)
constexpr int kEmulatedLaSms = 32;

// ws->minv (jb x jb, leading dimension jb) <- I - L^-1 for the unit-lower
// jb x jb triangle L: identity, the blocked FP64 solve, then the negated
// strictly lower part (the unit diagonal cancels).
static int u12_inverse(int64_t jb, const double* L, int64_t ldl, Workspace* ws, cudaStream_t s) {
  const size_t bytes = (size_t)jb * jb * sizeof(double);
  if (ws->minv_bytes < bytes) {
    void* p = ws->minv;
    HPL_TRY(grow(&p, &ws->minv_bytes, bytes));
    ws->minv = (double*)p;
  }
  HPL_TRY(launch_identity_f64(jb, ws->minv, jb, s));
  HPL_TRY(launch_trsm_llnu(jb, jb, L, ldl, ws->minv, jb, s));
  return launch_i_minus_lower(jb, ws->minv, jb, s);
}

static int getrf_impl(Workspace* ws, int64_t n, int64_t nb, double* A, int64_t lda, int32_t* ipiv,
                      int32_t* info, int lookahead, int slices, cudaStream_t s) {
  const int64_t npanels = (n + nb - 1) / nb;
  const size_t pslot = perm_ints_for(nb);
  const size_t fixed = 2 * perm_ints_for(1024);
  HPL_TRY(ensure_perm(ws, fixed + (size_t)npanels * pslot));
  int32_t* perms = ws->perm + fixed;
  if (info) HPL_CUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  HPL_CUDA(cudaMemsetAsync(ws->bar, 0, sizeof(unsigned long long), s));
  ws->bar_next = 0;
  cudaStream_t la = ws->la_stream;
  cudaEvent_t ev_cols = ws->ev[1], ev_panel = ws->ev[2];
  const bool use_la = lookahead && npanels > 1 && !g_timer.on;
  // Emulated update with look-ahead.  The update's fused kernel is persistent
  // and would hold every SM, so the next panel's FACT could not start beside
  // it: the update of the remaining columns runs on num_sms - P CTAs, FACT on
  // the look-ahead stream (its base kernel and its own emulated Schur updates
  // on at most P CTAs each), and when FACT is done P more CTAs of the update
  // join on the look-ahead stream, taking tiles from the same counter.
  // P = HPLGB_LA_SMS (0: no partition, FACT after the update).  A panel whose
  // base kernel cannot be resident (per-SM shared memory, registers, threads:
  // on the P free SMs or beside the update) takes the path without partition.
  int keep = 0;
  int oz_smem = 0, oz_regs = 0, oz_thr = 0, sm_smem = 0, resv = 0;
  if (use_la && slices >= 0) {
    const char* e = getenv("HPLGB_LA_SMS");
    keep = e ? atoi(e) : kEmulatedLaSms;
    if (keep <= 0 || keep >= ws->num_sms) keep = 0;
    if (keep) {
      HPL_TRY(ozaki_fused_footprint(&oz_smem, &oz_regs, &oz_thr));
      HPL_CUDA(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ws->device));
      HPL_CUDA(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, ws->device));
      const size_t cb = (size_t)npanels * sizeof(int);
      void* p = ws->tile_ctr;
      HPL_TRY(grow(&p, &ws->tile_ctr_bytes, cb));
      ws->tile_ctr = (int*)p;
      HPL_CUDA(cudaMemsetAsync(ws->tile_ctr, 0, cb, s));
    }
  }
  // whether FACT of an m-row panel can run beside the update on num_sms - keep SMs
  auto fact_fits = [&](int64_t m) -> bool {
    int64_t G = 0;
    int sm = 0, rg = 0, th = 0;
    if (panel_base_footprint(keep, m, panel_base_max_width(), &G, &sm, &rg, &th) != HPL_OK) return false;
    auto warp_regs = [](int r, int t) { return ((r * 32 + 255) / 256 * 256) * ((t + 31) / 32); };
    const bool beside = oz_smem + resv + sm + resv <= sm_smem && oz_thr + th <= 2048 &&
                        warp_regs(oz_regs, oz_thr) + warp_regs(rg, th) <= 65536;
    int per_free = sm_smem / (sm + resv);
    if (per_free > 2048 / th) per_free = 2048 / th;
    if (per_free > 65536 / warp_regs(rg, th)) per_free = 65536 / warp_regs(rg, th);
    const int64_t cap = (int64_t)(beside ? ws->num_sms - keep : 0) + (int64_t)keep * per_free;
    return G <= cap;
  };

  // FACT of panel 0
  timer_mark(PH_NONE);
  HPL_TRY(panel_factor(ws, n, nb < n ? nb : n, A, lda, ipiv, 0, info, 0, s, slices));
  timer_mark(PH_PANEL);
  for (int64_t k = 0; k < npanels; ++k) {
    const int64_t k0 = k * nb;
    const int64_t jb = nb < n - k0 ? nb : n - k0;
    const int64_t nx = k0 + jb;                 // first trailing column/row
    const int64_t jb2 = nx < n ? (nb < n - nx ? nb : n - nx) : 0;  // next panel width
    int32_t* perm = perms + (size_t)k * pslot;
    double* L11 = A + k0 + k0 * lda;
    // emulated path: M = I - L11^-1 for this panel's U12 solves
    const double* Minv = nullptr;
    if (slices >= 0 && nx < n) {
      HPL_TRY(u12_inverse(jb, L11, lda, ws, s));
      Minv = ws->minv;
    }
    // RS: compose this panel's interchanges once
    HPL_TRY(launch_laswp_compose(ipiv, k0, k0 + jb, 0, n, false, perm, ws->dev_err, s));
    if (jb2 > 0) {
      // UPDATE of the next panel's columns first (look-ahead, Sec. III)
      double* Cn = A + nx * lda;
      HPL_TRY(launch_laswp_apply(perm, jb, jb2, Cn, lda, s));
      timer_mark(PH_LASWP);
      HPL_TRY(u12_solve(jb, jb2, L11, lda, A + k0 + nx * lda, lda, slices, Minv, ws->dev_err, s));
      timer_mark(PH_TRSM);
      HPL_TRY(timed_gemm(n - nx, jb2, jb, A + nx + k0 * lda, lda, A + k0 + nx * lda, lda,
                         A + nx + nx * lda, lda, slices, ws->dev_err, s));
      timer_mark(PH_GEMM);
      cudaStream_t ps = s;
      if (use_la) {
        HPL_CUDA(cudaEventRecord(ev_cols, s));
        HPL_CUDA(cudaStreamWaitEvent(la, ev_cols, 0));
        ps = la;
      }
      // FACT of the next panel (on the look-ahead stream when enabled)
      const int64_t rc = nx + jb2;
      const bool part = keep > 0 && rc < n && fact_fits(n - nx);
      const int la_ctas = part ? ws->num_sms - keep : 0;
      HPL_TRY(panel_factor(ws, n - nx, jb2, A + nx + nx * lda, lda, ipiv + nx, nx, info, nx, ps, slices,
                           part ? keep : 0));
      if (use_la && !part) HPL_CUDA(cudaEventRecord(ev_panel, la));
      else if (!use_la) timer_mark(PH_PANEL);
      // UPDATE of the remaining columns
      if (rc < n) {
        double* Cr = A + rc * lda;
        HPL_TRY(launch_laswp_apply(perm, jb, n - rc, Cr, lda, s));
        timer_mark(PH_LASWP);
        HPL_TRY(u12_solve(jb, n - rc, L11, lda, A + k0 + rc * lda, lda, slices, Minv, ws->dev_err, s, la_ctas));
        timer_mark(PH_TRSM);
        const OzakiJoin join{la, ws->ev[3], keep, ws->tile_ctr + k};
        HPL_TRY(timed_gemm(n - nx, n - rc, jb, A + nx + k0 * lda, lda, A + k0 + rc * lda, lda,
                           A + nx + rc * lda, lda, slices, ws->dev_err, s, la_ctas, part ? &join : nullptr));
        timer_mark(PH_GEMM);
      }
      // with the partition the look-ahead stream ends with the joining update
      if (part) HPL_CUDA(cudaEventRecord(ev_panel, la));
    }
    // RS on the columns left of the panel (LAPACK convention)
    if (k0 > 0) {
      HPL_TRY(launch_laswp_apply(perm, jb, k0, A, lda, s));
      timer_mark(PH_LASWP);
    }
    if (use_la && jb2 > 0) HPL_CUDA(cudaStreamWaitEvent(s, ev_panel, 0));
  }
  return HPL_OK;
}

}  // namespace hplgb

using namespace hplgb;

// ------------------------------------------------------------------- C ABI
extern "C" {

const char* hpl_last_error(void) { return g_errmsg; }

int64_t hpl_kernel_launches(void) { return g_launches.load(); }

void hpl_finalize(void) {
  mxp_finalize();
  ozaki_finalize();
  std::lock_guard<std::mutex> lk(g_ws_mutex);
  for (auto*& ws : g_ws) {
    free_workspace(ws);
    ws = nullptr;
  }
}

int hpl_generate(int64_t n, uint64_t seed, int dd, double* A, int64_t lda, double* b, void* stream) {
  if (n < 0) return set_error(-1, "hpl_generate: n < 0");
  if (lda < (n > 1 ? n : 1)) return set_error(-5, "hpl_generate: lda < max(1,n)");
  if (n > 0 && !A) return set_error(-4, "hpl_generate: A is NULL");
  HPL_TRY(fault_point("generate"));
  if (n == 0) return HPL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  HPL_TRY(launch_generate(n, seed, A, lda, b, s));
  if (dd) HPL_TRY(launch_dd_diag(n, A, lda, s));
  return HPL_OK;
}

static int getrf_entry(const char* name, int64_t n, int64_t nb, double* A, int64_t lda, int32_t* ipiv,
                       int32_t* info, int lookahead, int slices, void* stream) {
  if (n < 0) return set_error(-1, "%s: n < 0", name);
  if (nb < 1) return set_error(-2, "%s: nb < 1", name);
  if (n > 0 && !A) return set_error(-3, "%s: A is NULL", name);
  if (lda < (n > 1 ? n : 1)) return set_error(-4, "%s: lda < max(1,n)", name);
  if (n > 0 && !ipiv) return set_error(-5, "%s: ipiv is NULL", name);
  if (n > 0x7fffffffLL) return set_error(-1, "%s: n exceeds int32 pivots", name);
  HPL_TRY(fault_point("getrf"));
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (info) HPL_CUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
    return HPL_OK;
  }
  if (nb > n) nb = n;
  if (nb > 1024) return set_error(-2, "%s: nb > 1024 is not supported", name);
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  // phase timers (HPLGB_TIMERS=1)
  const char* tv = getenv("HPLGB_TIMERS");
  for (auto e : g_timer.evs) cudaEventDestroy(e);
  g_timer.evs.clear();
  g_timer.phase.clear();
  g_timer.on = tv && tv[0] == '1';
  g_timer.s = s;
  return getrf_impl(ws, n, nb, A, lda, ipiv, info, lookahead, slices, s);
}

int hpl_getrf(int64_t n, int64_t nb, double* A, int64_t lda, int32_t* ipiv, int32_t* info,
              int lookahead, void* stream) {
  return getrf_entry("hpl_getrf", n, nb, A, lda, ipiv, info, lookahead, -1, stream);
}

int hpl_getrf_emulated(int64_t n, int64_t nb, double* A, int64_t lda, int32_t* ipiv, int32_t* info,
                       int lookahead, int slices, void* stream) {
  if (slices < 0) return set_error(-8, "hpl_getrf_emulated: slices < 0");
  int sl = 0, beta = 0;
  if (n > 0 && !ozaki_params(nb < n ? (nb < 384 ? nb : 384) : (n < 384 ? n : 384), slices, &sl, &beta))
    return set_error(-8, "hpl_getrf_emulated: no exact slice width for %d slices", slices);
  return getrf_entry("hpl_getrf_emulated", n, nb, A, lda, ipiv, info, lookahead, slices, stream);
}

int hpl_dgemm_emulated(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int slices, void* stream) {
  if (m < 0) return set_error(-1, "hpl_dgemm_emulated: m < 0");
  if (n < 0) return set_error(-2, "hpl_dgemm_emulated: n < 0");
  if (k < 0) return set_error(-3, "hpl_dgemm_emulated: k < 0");
  if (m > 0 && k > 0 && !A) return set_error(-4, "hpl_dgemm_emulated: A is NULL");
  if (lda < (m > 1 ? m : 1)) return set_error(-5, "hpl_dgemm_emulated: lda < max(1,m)");
  if (k > 0 && n > 0 && !B) return set_error(-6, "hpl_dgemm_emulated: B is NULL");
  if (ldb < (k > 1 ? k : 1)) return set_error(-7, "hpl_dgemm_emulated: ldb < max(1,k)");
  if (m > 0 && n > 0 && !C) return set_error(-8, "hpl_dgemm_emulated: C is NULL");
  if (ldc < (m > 1 ? m : 1)) return set_error(-9, "hpl_dgemm_emulated: ldc < max(1,m)");
  if (slices < 0) return set_error(-10, "hpl_dgemm_emulated: slices < 0");
  int sl = 0, beta = 0;
  if (k > 0 && !ozaki_params(k < 384 ? k : 384, slices, &sl, &beta))
    return set_error(-10, "hpl_dgemm_emulated: no exact slice width for %d slices", slices);
  HPL_TRY(fault_point("dgemm_emulated"));
  if (m == 0 || n == 0 || k == 0) return HPL_OK;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  return launch_ozaki_gemm(m, n, k, A, lda, B, ldb, C, ldc, slices, ws->dev_err, (cudaStream_t)stream);
}

int hpl_phase_times(double* out, int64_t cap) {
  if (!out || cap <= 0) return 0;
  double acc[kNumPhases] = {0};
  if (!g_timer.evs.empty()) {
    cudaEventSynchronize(g_timer.evs.back());
    for (size_t i = 1; i < g_timer.evs.size(); ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, g_timer.evs[i - 1], g_timer.evs[i]);
      int ph = g_timer.phase[i];
      if (ph >= 1 && ph < kNumPhases) acc[ph] += ms;
      acc[0] += ms;
    }
  }
  int64_t k = cap < (int64_t)kNumPhases ? cap : (int64_t)kNumPhases;
  for (int64_t i = 0; i < k; ++i) out[i] = acc[i];
  return (int)k;
}

int hpl_getrs(char trans, int64_t n, int64_t nrhs, const double* LU, int64_t lda, const int32_t* ipiv,
              double* B, int64_t ldb, void* stream) {
  if (!(trans == 'N' || trans == 'n' || trans == 'T' || trans == 't'))
    return set_error(-1, "hpl_getrs: trans must be 'N' or 'T'");
  if (n < 0) return set_error(-2, "hpl_getrs: n < 0");
  if (nrhs < 0) return set_error(-3, "hpl_getrs: nrhs < 0");
  if (n > 0 && !LU) return set_error(-4, "hpl_getrs: LU is NULL");
  if (lda < (n > 1 ? n : 1)) return set_error(-5, "hpl_getrs: lda < max(1,n)");
  if (n > 0 && nrhs > 0 && !B) return set_error(-7, "hpl_getrs: B is NULL");
  if (ldb < (n > 1 ? n : 1)) return set_error(-8, "hpl_getrs: ldb < max(1,n)");
  HPL_TRY(fault_point("getrs"));
  if (n == 0 || nrhs == 0) return HPL_OK;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  HPL_TRY(ensure_perm(ws, 2 * perm_ints_for(1024)));
  char t = (trans == 'T' || trans == 't') ? 'T' : 'N';
  return launch_getrs(ws, t, n, nrhs, LU, lda, ipiv, B, ldb, (cudaStream_t)stream);
}

int hpl_residual(int64_t n, uint64_t seed, int dd, const double* A, int64_t lda, const double* x,
                 const double* b, double* out5, void* stream) {
  if (n < 0) return set_error(-1, "hpl_residual: n < 0");
  if (A && lda < (n > 1 ? n : 1)) return set_error(-5, "hpl_residual: lda < max(1,n)");
  if (n > 0 && !x) return set_error(-6, "hpl_residual: x is NULL");
  if (!out5) return set_error(-8, "hpl_residual: out5 is NULL");
  HPL_TRY(fault_point("residual"));
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  return launch_residual(ws, n, seed, dd, A, lda, x, b, out5, (cudaStream_t)stream);
}

int hpl_dgemm(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
              int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
              void* stream) {
  bool TA = ta == 'T' || ta == 't', TB = tb == 'T' || tb == 't';
  if (!(TA || ta == 'N' || ta == 'n')) return set_error(-1, "hpl_dgemm: bad ta");
  if (!(TB || tb == 'N' || tb == 'n')) return set_error(-2, "hpl_dgemm: bad tb");
  if (m < 0) return set_error(-3, "hpl_dgemm: m < 0");
  if (n < 0) return set_error(-4, "hpl_dgemm: n < 0");
  if (k < 0) return set_error(-5, "hpl_dgemm: k < 0");
  int64_t arows = TA ? k : m, brows = TB ? n : k;
  if (lda < (arows > 1 ? arows : 1)) return set_error(-8, "hpl_dgemm: lda too small");
  if (ldb < (brows > 1 ? brows : 1)) return set_error(-10, "hpl_dgemm: ldb too small");
  if (ldc < (m > 1 ? m : 1)) return set_error(-13, "hpl_dgemm: ldc too small");
  // operands are checked where they are read: C for a nonempty product, A and
  // B when k > 0 as well (a NULL operand would otherwise fault on the device)
  if (m > 0 && n > 0 && k > 0 && !A) return set_error(-7, "hpl_dgemm: A is NULL");
  if (m > 0 && n > 0 && k > 0 && !B) return set_error(-9, "hpl_dgemm: B is NULL");
  if (m > 0 && n > 0 && !C) return set_error(-12, "hpl_dgemm: C is NULL");
  HPL_TRY(fault_point("dgemm"));
  return launch_dgemm(TA, TB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, (cudaStream_t)stream);
}

int hpl_outer_update(int64_t m, int64_t n, int64_t k, double alpha, const double* U, int64_t ldu,
                     const double* V, int64_t ldv, double* C, int64_t ldc, void* stream) {
  if (m < 0) return set_error(-1, "hpl_outer_update: m < 0");
  if (n < 0) return set_error(-2, "hpl_outer_update: n < 0");
  if (k < 0) return set_error(-3, "hpl_outer_update: k < 0");
  if (ldu < (m > 1 ? m : 1)) return set_error(-6, "hpl_outer_update: ldu < max(1,m)");
  if (ldv < (n > 1 ? n : 1)) return set_error(-8, "hpl_outer_update: ldv < max(1,n)");
  if (ldc < (m > 1 ? m : 1)) return set_error(-10, "hpl_outer_update: ldc < max(1,m)");
  if (m > 0 && n > 0 && k > 0 && !U) return set_error(-5, "hpl_outer_update: U is NULL");
  if (m > 0 && n > 0 && k > 0 && !V) return set_error(-7, "hpl_outer_update: V is NULL");
  if (m > 0 && n > 0 && !C) return set_error(-9, "hpl_outer_update: C is NULL");
  HPL_TRY(fault_point("outer_update"));
  return launch_dgemm(false, true, m, n, k, alpha, U, ldu, V, ldv, 0.0, C, ldc, (cudaStream_t)stream);
}

int hpl_laswp(int64_t ncols, double* A, int64_t lda, int64_t k1, int64_t k2, const int32_t* ipiv,
              void* stream) {
  if (ncols < 0) return set_error(-1, "hpl_laswp: ncols < 0");
  if (k1 < 0 || k2 < k1) return set_error(-4, "hpl_laswp: bad k1/k2");
  if (lda < (k2 > 1 ? k2 : 1)) return set_error(-3, "hpl_laswp: lda < k2");
  if (ncols > 0 && k2 > k1 && !A) return set_error(-2, "hpl_laswp: A is NULL");
  if (ncols > 0 && k2 > k1 && !ipiv) return set_error(-6, "hpl_laswp: ipiv is NULL");
  HPL_TRY(fault_point("laswp"));
  if (ncols == 0 || k2 == k1) return HPL_OK;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  HPL_TRY(ensure_perm(ws, 2 * perm_ints_for(1024)));
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* perm = ws->perm + perm_ints_for(1024);
  for (int64_t a = k1; a < k2; a += 1024) {
    int64_t e = a + 1024 < k2 ? a + 1024 : k2;
    HPL_TRY(launch_laswp_compose(ipiv, a, e, 0, lda, false, perm, ws->dev_err, s));
    HPL_TRY(launch_laswp_apply(perm, e - a, ncols, A, lda, s));
  }
  return HPL_OK;
}

int hpl_trsm_llnu(int64_t m, int64_t n, const double* A, int64_t lda, double* B, int64_t ldb,
                  void* stream) {
  if (m < 0) return set_error(-1, "hpl_trsm_llnu: m < 0");
  if (n < 0) return set_error(-2, "hpl_trsm_llnu: n < 0");
  if (lda < (m > 1 ? m : 1)) return set_error(-4, "hpl_trsm_llnu: lda < max(1,m)");
  if (ldb < (m > 1 ? m : 1)) return set_error(-6, "hpl_trsm_llnu: ldb < max(1,m)");
  if (m > 0 && n > 0 && !A) return set_error(-3, "hpl_trsm_llnu: A is NULL");
  if (m > 0 && n > 0 && !B) return set_error(-5, "hpl_trsm_llnu: B is NULL");
  HPL_TRY(fault_point("trsm"));
  return launch_trsm_llnu(m, n, A, lda, B, ldb, (cudaStream_t)stream);
}

int hpl_panel_getrf(int64_t m, int64_t w, double* A, int64_t lda, int32_t* ipiv, int32_t* info,
                    void* stream) {
  if (m < 0) return set_error(-1, "hpl_panel_getrf: m < 0");
  if (w < 0 || w > m) return set_error(-2, "hpl_panel_getrf: need 0 <= w <= m");
  if (w > 1024) return set_error(-2, "hpl_panel_getrf: w > 1024 is not supported");
  if (lda < (m > 1 ? m : 1)) return set_error(-4, "hpl_panel_getrf: lda < max(1,m)");
  if (m > 0 && w > 0 && !A) return set_error(-3, "hpl_panel_getrf: A is NULL");
  if (m > 0 && w > 0 && !ipiv) return set_error(-5, "hpl_panel_getrf: ipiv is NULL");
  HPL_TRY(fault_point("panel"));
  if (m == 0 || w == 0) return HPL_OK;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  HPL_TRY(ensure_perm(ws, 2 * perm_ints_for(1024)));
  cudaStream_t s = (cudaStream_t)stream;
  if (info) HPL_CUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  HPL_CUDA(cudaMemsetAsync(ws->bar, 0, sizeof(unsigned long long), s));
  ws->bar_next = 0;
  return panel_factor(ws, m, w, A, lda, ipiv, 0, info, 0, s);
}

int hpl_set_gemm_timing(int on) {
  g_gt.on = on != 0;
  g_gt.used = 0;
  g_gt.flops.clear();
  g_gt.bytes.clear();
  return HPL_OK;
}

int hpl_gemm_timing(double* out4) {
  if (!out4) return set_error(-1, "hpl_gemm_timing: out4 is NULL");
  double ms = 0, fl = 0, by = 0;
  for (size_t i = 0; i + 1 < g_gt.used; i += 2) {
    HPL_CUDA(cudaEventSynchronize(g_gt.pool[i + 1]));
    float t = 0;
    HPL_CUDA(cudaEventElapsedTime(&t, g_gt.pool[i], g_gt.pool[i + 1]));
    ms += t;
    fl += g_gt.flops[i / 2];
    by += g_gt.bytes[i / 2];
  }
  out4[0] = (double)(g_gt.used / 2);
  out4[1] = ms;
  out4[2] = fl;
  out4[3] = by;
  return HPL_OK;
}

int hpl_sync_check(void* stream) {
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  HPL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  HPL_CUDA(cudaStreamSynchronize(ws->la_stream));
  int e = 0;
  HPL_CUDA(cudaMemcpy(&e, ws->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != DEV_OK) {
    HPL_CUDA(cudaMemset(ws->dev_err, 0, sizeof(int)));
    if (e == DEV_TIMEOUT) return set_error(HPL_ERR_TIMEOUT, "a bounded grid-wide wait expired");
    if (e == DEV_BADPIV) return set_error(HPL_ERR_CUDA, "an interchange named a row outside the matrix");
    return set_error(HPL_ERR_CUDA, "device error word %d", e);
  }
  return HPL_OK;
}

int hpl_fp64_dmma_peak(int64_t iters, double* gflops, void* stream) {
  if (iters < 1) return set_error(-1, "hpl_fp64_dmma_peak: iters < 1");
  if (!gflops) return set_error(-2, "hpl_fp64_dmma_peak: gflops is NULL");
  return launch_fp64_dmma_peak(iters, gflops, (cudaStream_t)stream);
}

int hpl_fp64_mixed_peak(int64_t iters, int dfma_tiles, int split_warps, double* gflops, void* stream) {
  if (iters < 1) return set_error(-1, "hpl_fp64_mixed_peak: iters < 1");
  if (dfma_tiles < 0 || dfma_tiles > 64) return set_error(-2, "hpl_fp64_mixed_peak: dfma_tiles outside [0, 64]");
  if (!gflops) return set_error(-4, "hpl_fp64_mixed_peak: gflops is NULL");
  return launch_fp64_mixed_peak(iters, dfma_tiles, split_warps, gflops, (cudaStream_t)stream);
}

int64_t hpl_workspace_bytes(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxCountedDevices) return -1;
  return (int64_t)g_dev_bytes[dev].load();
}

int hpl_fp64_peak(int64_t iters, double* gflops, void* stream) {
  if (iters < 1) return set_error(-1, "hpl_fp64_peak: iters < 1");
  if (!gflops) return set_error(-2, "hpl_fp64_peak: gflops is NULL");
  return launch_fp64_peak(iters, gflops, (cudaStream_t)stream);
}

}  // extern "C"
