// peak.cu -- FP64 pipe throughput probes.  The roofline of the FP64 kernels is
// the FP64 pipe; these measure what it delivers on the running GPU, under the
// clocks of the moment, so that fractions of peak are taken against a number
// measured beside them, and so that the choice between the two FP64 paths
// sm_103a exposes (DFMA from registers, mma.sync m8n8k4 f64 "DMMA") rests on
// a measurement.
//
//   dfma:  each thread updates a 4x4 register tile acc[i][j] += a[i] b[j]
//          (the inner step of the trailing-update DGEMM): 16 independent
//          FMA chains per thread, 8 warps per SM quadrant.
//   dmma:  four independent m8n8k4 f64 chains per warp.
//   mixed: both in one kernel, either within every warp (r DFMA tiles per
//          DMMA step) or split by warp (even warps DFMA, odd warps DMMA).
#include "common.cuh"

namespace hplgb {

namespace {

// 2 * 16 flop per thread per tile step
__device__ __forceinline__ void dfma_tile(double (&acc)[4][4], const double (&a)[4], const double (&b)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
}

// 2 * 8 * 8 * 4 flop per warp per chain step (four chains)
__device__ __forceinline__ void dmma_step(double (&c)[4][2], double a, double b) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c[i][0]), "+d"(c[i][1])
                 : "d"(a), "d"(b));
}

// MODE 0: DFMA only (r tile steps per iteration); 1: DMMA only; 2: per
// iteration one DMMA step and r DFMA tile steps in every warp; 3: even warps
// run the DFMA loop, odd warps the DMMA loop.  Each mode holds only the
// registers it uses, so that the occupancy of a mode is its own.
template <int MODE>
__global__ void __launch_bounds__(256) fp64_probe_kernel(int iters, int r, double* sink) {
  constexpr bool kDfma = MODE != 1, kDmma = MODE != 0;
  double acc[4][4], a[4], b[4], c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[i] = 1.0 + 1e-9 * (threadIdx.x + i);
    b[i] = 1.0 - 1e-9 * (threadIdx.x + 2 * i);
    c[i][0] = i;
    c[i][1] = i + 1;
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 1e-3 * (i * 4 + j);
  }
  const int warp = threadIdx.x >> 5;
  const bool do_dfma = kDfma && (MODE != 3 || (warp & 1) == 0);
  const bool do_dmma = kDmma && (MODE != 3 || (warp & 1) == 1);
  const double ma = threadIdx.x * 1e-6, mb = 1e-7;
  for (int it = 0; it < iters; ++it) {
    if (kDmma && do_dmma) dmma_step(c, ma, mb);
    if (kDfma && do_dfma)
      for (int q = 0; q < r; ++q) dfma_tile(acc, a, b);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (kDmma) s += c[i][0] + c[i][1];
    if (kDfma)
#pragma unroll
      for (int j = 0; j < 4; ++j) s += acc[i][j];
  }
  if (s == 1234.5678) *sink = s;  // never true for these inputs; keeps the chains live
}

// Runs the probe (4 warm-up launches, best of 5 timed) as one full wave of
// CTAs (every SM holds as many as fit, so no partial second wave dilutes the
// rate) and returns GFLOP/s of the flops it performed.
template <int MODE>
int run_probe_mode(int64_t iters, int r, double* gflops, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  HPL_CUDA(cudaGetDevice(&dev));
  HPL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HPL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_probe_kernel<MODE>, 256, 0));
  if (per_sm < 1) return set_error(HPL_ERR_NOTSUP, "fp64 probe cannot be resident");
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  double* sink = reinterpret_cast<double*>(reinterpret_cast<char*>(ws->dev_err) + 16);
  cudaEvent_t e0, e1;
  HPL_CUDA(cudaEventCreate(&e0));
  HPL_CUDA(cudaEventCreate(&e1));
  const int blocks = sms * per_sm, threads = 256;
  const int it = (int)(iters > 0x40000000 ? 0x40000000 : iters);
  for (int w = 0; w < 4; ++w) {
    fp64_probe_kernel<MODE><<<blocks, threads, 0, s>>>(it, r, sink);
    count_launch();
  }
  HPL_TRY(check_launch("fp64_probe_kernel"));
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    HPL_CUDA(cudaEventRecord(e0, s));
    fp64_probe_kernel<MODE><<<blocks, threads, 0, s>>>(it, r, sink);
    count_launch();
    HPL_CUDA(cudaEventRecord(e1, s));
    HPL_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    HPL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HPL_TRY(check_launch("fp64_probe_kernel"));
  const double warps = (double)blocks * (threads / 32);
  const double dfma_per_warp = 2.0 * 16 * 32 * r;   // flop per iteration
  const double dmma_per_warp = 2.0 * 8 * 8 * 4 * 4;
  double fl = 0.0;
  if (MODE == 0) fl = warps * dfma_per_warp;
  if (MODE == 1) fl = warps * dmma_per_warp;
  if (MODE == 2) fl = warps * (dfma_per_warp + dmma_per_warp);
  if (MODE == 3) fl = 0.5 * warps * (dfma_per_warp + dmma_per_warp);
  *gflops = fl * (double)it / (best * 1e-3) / 1e9;
  return HPL_OK;
}

int run_probe(int mode, int64_t iters, int r, double* gflops, cudaStream_t s) {
  switch (mode) {
    case 0: return run_probe_mode<0>(iters, r, gflops, s);
    case 1: return run_probe_mode<1>(iters, r, gflops, s);
    case 2: return run_probe_mode<2>(iters, r, gflops, s);
    default: return run_probe_mode<3>(iters, r, gflops, s);
  }
}

}  // namespace

int launch_fp64_peak(int64_t iters, double* gflops, cudaStream_t s) { return run_probe(0, iters, 1, gflops, s); }

int launch_fp64_dmma_peak(int64_t iters, double* gflops, cudaStream_t s) { return run_probe(1, iters, 0, gflops, s); }

int launch_fp64_mixed_peak(int64_t iters, int dfma_tiles, int split_warps, double* gflops, cudaStream_t s) {
  return run_probe(split_warps ? 3 : 2, iters, dfma_tiles, gflops, s);
}

}  // namespace hplgb
