// k_peaks.cu -- throughput probes of the arithmetic units the inversion's kernels use, for
// the benchmark's roofline denominators: FP64 FMA (DFMA), FP64 mma.sync (DMMA, m8n8k4) and
// FP32 FMA (FFMA).  Each probe runs independent chains (no memory traffic in the timed
// loop) on every SM, several resident blocks per SM, and is timed with CUDA events on its
// own stream after a warm-up launch.
#include <stdio.h>

#include "gj_internal.cuh"

namespace gj {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) out[0] = s;  // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(kProbeThreads) ffma_probe_kernel(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) out[0] = s;
}

// One m8n8k4 FP64 MMA per warp per chain step: 2 * 8 * 8 * 4 = 512 FLOP.
__global__ void __launch_bounds__(kProbeThreads) dmma_probe_kernel(double* out, int iters, double a0, double b0) {
  double acc[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = 1e-3 * (threadIdx.x + c);
  const double a = a0 * (1.0 + 1e-6 * threadIdx.x), b = b0;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(a), "d"(b));
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
  if (s == 12345.678) out[0] = s;
}

template <class F>
gj_status time_probe(F launch, double flop, int reps, double* gflops) {
  cudaStream_t s;
  GJ_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch(s);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, s);
    launch(s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return cuda_fail(e, "peak probe");
  *gflops = flop / (best * 1e-3) / 1e9;
  return GJ_OK;
}

}  // namespace
}  // namespace gj

using namespace gj;

extern "C" gj_status gj_measure_peaks(gj_peaks* out) {
  set_last_error("");
  if (!out) return GJ_ERR_ARG;
  int dev = 0, sms = 0;
  GJ_CUDA(cudaGetDevice(&dev));
  GJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* scratch = nullptr;
  GJ_CUDA(cudaMalloc(&scratch, 64));
  const int blocks = sms * 4;
  const double threads = (double)blocks * kProbeThreads;
  gj_status st = GJ_OK;
  {
    const int it = 4096;
    st = time_probe([&](cudaStream_t s) { dfma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(scratch, it, 0.999, 1e-3); },
                    2.0 * kChains * it * threads, 5, &out->fp64_fma_gflops);
  }
  if (st == GJ_OK) {
    const int it = 2048;
    st = time_probe([&](cudaStream_t s) { dmma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(scratch, it, 0.999, 1e-3); },
                    512.0 * 4 * it * (threads / 32.0), 5, &out->fp64_mma_gflops);
  }
  if (st == GJ_OK) {
    const int it = 16384;
    st = time_probe(
        [&](cudaStream_t s) {
          ffma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(reinterpret_cast<float*>(scratch), it, 0.999f, 1e-3f);
        },
        2.0 * kChains * it * threads, 5, &out->fp32_fma_gflops);
  }
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  out->sm_count = sms;
  out->max_clock_mhz = clk_khz / 1000.0;
  cudaFree(scratch);
  return st;
}
