// peak.cu -- FP64 FMA throughput probe.  The roofline of the FP64 kernels is
// the DFMA pipe; this measures what it delivers on the running GPU, under the
// clocks of the moment, so that fractions of peak are taken against a number
// measured beside them.
#include "common.cuh"

namespace hplgb {

namespace {

constexpr int kAcc = 8;

__global__ void __launch_bounds__(256) dfma_peak_kernel(int iters, double b, double c, double* sink) {
  double acc[kAcc];
#pragma unroll
  for (int i = 0; i < kAcc; ++i) acc[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kAcc; ++i) acc[i] = fma(acc[i], b, c);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < kAcc; ++i) s += acc[i];
  if (s == 1234.5678) *sink = s;  // never true for these inputs; keeps the chains live
}

// Four independent FP64 mma.sync m8n8k4 chains per warp (the FP64 tensor
// path that sm_103a exposes to PTX): 2*8*8*4 flop per instruction.
__global__ void __launch_bounds__(256) dmma_peak_kernel(int iters, double* sink) {
  double a = threadIdx.x * 1e-6, b = 1e-7;
  double c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) { c[i][0] = i; c[i][1] = i + 1; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[i][0]), "+d"(c[i][1])
                   : "d"(a), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
  if (s == 1234.5678) *sink = s;
}

}  // namespace

int launch_fp64_dmma_peak(int64_t iters, double* gflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  HPL_CUDA(cudaGetDevice(&dev));
  HPL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  double* sink = reinterpret_cast<double*>(reinterpret_cast<char*>(ws->dev_err) + 16);
  cudaEvent_t e0, e1;
  HPL_CUDA(cudaEventCreate(&e0));
  HPL_CUDA(cudaEventCreate(&e1));
  const int blocks = sms * 4, threads = 256;
  const int it = (int)(iters > 0x40000000 ? 0x40000000 : iters);
  for (int w = 0; w < 4; ++w) {
    dmma_peak_kernel<<<blocks, threads, 0, s>>>(it, sink);
    count_launch();
  }
  HPL_TRY(check_launch("dmma_peak_kernel"));
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    HPL_CUDA(cudaEventRecord(e0, s));
    dmma_peak_kernel<<<blocks, threads, 0, s>>>(it, sink);
    count_launch();
    HPL_CUDA(cudaEventRecord(e1, s));
    HPL_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    HPL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  double flops = 2.0 * 8 * 8 * 4 * 4 * (double)it * blocks * (threads / 32);
  *gflops = flops / (best * 1e-3) / 1e9;
  return HPL_OK;
}

int launch_fp64_peak(int64_t iters, double* gflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  HPL_CUDA(cudaGetDevice(&dev));
  HPL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* sink = nullptr;
  Workspace* ws = nullptr;
  HPL_TRY(get_workspace(&ws));
  sink = reinterpret_cast<double*>(reinterpret_cast<char*>(ws->dev_err) + 16);
  cudaEvent_t e0, e1;
  HPL_CUDA(cudaEventCreate(&e0));
  HPL_CUDA(cudaEventCreate(&e1));
  const int blocks = sms * 4, threads = 256;
  const int it = (int)(iters > 0x40000000 ? 0x40000000 : iters);
  // warm-up long enough for the clocks to settle (~0.1 s)
  for (int w = 0; w < 4; ++w) {
    dfma_peak_kernel<<<blocks, threads, 0, s>>>(it, 1.0000001, 1e-9, sink);
    count_launch();
  }
  HPL_TRY(check_launch("dfma_peak_kernel"));
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    HPL_CUDA(cudaEventRecord(e0, s));
    dfma_peak_kernel<<<blocks, threads, 0, s>>>(it, 1.0000001, 1e-9, sink);
    count_launch();
    HPL_TRY(check_launch("dfma_peak_kernel"));
    HPL_CUDA(cudaEventRecord(e1, s));
    HPL_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    HPL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  double flops = 2.0 * kAcc * (double)it * blocks * threads;
  *gflops = flops / (best * 1e-3) / 1e9;
  return HPL_OK;
}

}  // namespace hplgb
