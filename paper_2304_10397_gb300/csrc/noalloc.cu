// noalloc.cu -- hpl_panel_getrf_noalloc: the panel factorization (FACT) with
// all of its scratch in one fixed, statically allocated device array, for
// callers that cannot allocate device memory when they call the library: a
// process that hands the whole GPU memory to its own pool allocator at start-up,
// or a latency-bound loop that must never enter the driver's allocator.  The
// caller still owns and passes the panel, the pivots and info.
//
// The array below is part of the library image: every GPU that loads the
// library holds kNoAllocScratchBytes (64 KiB) of it until the process exits.
// In host code `g_noalloc_scratch` names a host-side stand-in, not device
// memory, so the kernels are given the device address that
// cudaGetSymbolAddress returns, looked up once per device (with that device
// current) by the first call made on it.  Make that first call outside any
// stream capture.  Every call shares the array: the barrier counter and the
// error word are cleared at the start of each call (asynchronously, on the
// caller's stream), and two calls whose work overlaps on the GPU race on the
// array, so calls must be ordered (one stream, or synchronized).
#include <mutex>

#include "common.cuh"

namespace hplgb {

int launch_panel_base_scratch(int num_sms, int64_t m, int w, double* P, int64_t lda, int32_t* ipiv,
                              int64_t ipiv_shift, int32_t* info, int64_t info_shift, double* slots,
                              size_t slots_bytes, unsigned long long* bar, unsigned long long* bar_next,
                              int* err, cudaStream_t s);
int panel_check_resident();

namespace {

// Layout: [0, 8) grid-barrier counter, [8, 12) error word, [256, 256 + kSlotsBytes)
// pivot-candidate slots for up to kMaxCtas CTAs, then the composed permutation
// (for up to kMaxWidth interchanges).
constexpr int kMaxCtas = 160;
constexpr int kMaxWidth = 1024;
constexpr size_t kSlotsBytes = (size_t)(2 * kMaxCtas * (2 + 16) + 2 * 16) * sizeof(double);  // 46336
constexpr size_t kPermOffset = 256 + ((kSlotsBytes + 255) / 256) * 256;
constexpr size_t kNoAllocScratchBytes = 64 * 1024;
static_assert(kPermOffset + (size_t)(4 * kMaxWidth + 4) * sizeof(int32_t) <= kNoAllocScratchBytes,
              "no-alloc scratch too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct Scratch {
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch
  int num_sms = 0;
};
constexpr int kMaxDevices = 64;
Scratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

struct Ctx {
  int num_sms;
  double* slots;
  unsigned long long* bar;
  unsigned long long bar_next;
  int* err;
  int32_t* perm;
};

// A bounded wait that expired gives info = -1; an interchange that named a
// row outside the panel (only possible if the panel's memory was changed
// under the call) gives info = -2.
__global__ void fold_error_into_info(const int* err, int32_t* info) {
  const int e = *err;
  if (e == DEV_TIMEOUT) *info = -1;
  else if (e != 0) *info = -2;
}

int rec(Ctx* c, int64_t m, int64_t w, double* A, int64_t lda, int32_t* ipiv, int64_t ipiv_shift, int32_t* info,
        int64_t info_shift, cudaStream_t s) {
  if (w <= panel_base_max_width())
    return launch_panel_base_scratch(c->num_sms, m, (int)w, A, lda, ipiv, ipiv_shift, info, info_shift, c->slots,
                                     kSlotsBytes, c->bar, &c->bar_next, c->err, s);
  int64_t w1 = (w / 2 + 7) / 8 * 8;
  if (w1 >= w) w1 = w / 2;
  const int64_t w2 = w - w1;
  HPL_TRY(rec(c, m, w1, A, lda, ipiv, ipiv_shift, info, info_shift, s));
  HPL_TRY(launch_laswp_compose(ipiv, 0, w1, ipiv_shift, m, false, c->perm, c->err, s));
  HPL_TRY(launch_laswp_apply(c->perm, w1, w2, A + w1 * lda, lda, s));
  HPL_TRY(launch_trsm_llnu(w1, w2, A, lda, A + w1 * lda, lda, s));
  HPL_TRY(launch_dgemm(false, false, m - w1, w2, w1, -1.0, A + w1, lda, A + w1 * lda, lda, 1.0,
                       A + w1 + w1 * lda, lda, s));
  HPL_TRY(rec(c, m - w1, w2, A + w1 + w1 * lda, lda, ipiv + w1, ipiv_shift + w1, info, info_shift + w1, s));
  HPL_TRY(launch_laswp_compose(ipiv, w1, w, ipiv_shift, m, false, c->perm, c->err, s));
  return launch_laswp_apply(c->perm, w2, w1, A, lda, s);
}

}  // namespace

}  // namespace hplgb

using namespace hplgb;

extern "C" int hpl_panel_getrf_noalloc(int64_t m, int64_t w, double* A, int64_t lda, int32_t* ipiv,
                                       int32_t* info, void* stream) {
  if (m < 0) return set_error(-1, "hpl_panel_getrf_noalloc: m < 0");
  if (w < 0 || w > m) return set_error(-2, "hpl_panel_getrf_noalloc: need 0 <= w <= m");
  if (w > kMaxWidth)
    return set_error(-2, "hpl_panel_getrf_noalloc: w = %lld exceeds the fixed scratch (at most %d columns)",
                     (long long)w, kMaxWidth);
  if (lda < (m > 1 ? m : 1)) return set_error(-4, "hpl_panel_getrf_noalloc: lda < max(1,m)");
  if (m > 0 && w > 0 && (!A || !ipiv)) return set_error(-3, "hpl_panel_getrf_noalloc: A or ipiv is NULL");
  if (!info) return set_error(-6, "hpl_panel_getrf_noalloc: info is required");
  HPL_TRY(fault_point("panel_noalloc"));
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  HPL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(HPL_ERR_NOTSUP, "hpl_panel_getrf_noalloc: device index");
  Scratch sc;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    if (!g_scratch[dev].base) {  // set-up, once per device, with that device current
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return set_error(HPL_ERR_CUDA, "cudaGetSymbolAddress(no-alloc scratch): %s", cudaGetErrorString(e));
      int sms = 0;
      HPL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      // every CTA of the base kernel must be resident at once (grid barrier)
      HPL_TRY(panel_check_resident());
      g_scratch[dev].base = static_cast<unsigned char*>(p);
      g_scratch[dev].num_sms = sms < kMaxCtas ? sms : kMaxCtas;
    }
    sc = g_scratch[dev];
  }
  // state that must start at zero: barrier counter, error word, info
  HPL_CUDA(cudaMemsetAsync(sc.base, 0, 16, s));
  HPL_CUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  if (m == 0 || w == 0) return HPL_OK;
  Ctx c;
  c.num_sms = sc.num_sms;
  c.bar = reinterpret_cast<unsigned long long*>(sc.base);
  c.err = reinterpret_cast<int*>(sc.base + 8);
  c.slots = reinterpret_cast<double*>(sc.base + 256);
  c.perm = reinterpret_cast<int32_t*>(sc.base + kPermOffset);
  c.bar_next = 0;
  HPL_TRY(rec(&c, m, w, A, lda, ipiv, 0, info, 0, s));
  fold_error_into_info<<<1, 1, 0, s>>>(c.err, info);
  count_launch();
  return check_launch("fold_error_into_info");
}
