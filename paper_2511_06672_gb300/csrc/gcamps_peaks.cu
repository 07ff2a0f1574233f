// Arithmetic peaks of the GPU the library runs on, measured with CUDA events: the denominators of the
// engine's roofline (its exact class evaluations are FP64, its screen and estimates FP32).  Each probe is a
// grid of independent multiply-add chains long enough (hundreds of milliseconds) that launch overheads
// vanish; flops are counted as 2 per fused multiply-add.

#include <cuda_runtime.h>

#include "gcamps.h"

namespace {

constexpr int kPeakThreads = 256;

// 8 independent FP64 chains per thread
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma64(double* sink, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = 1e-3 * (threadIdx.x + u);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(a[u], b, c);
  }
  double t = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) t += a[u];
  if (t == 1.2345) sink[0] = t;   // keeps the chains live
}

// 16 independent FP32 chains per thread
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma32(float* sink, int iters, float b, float c) {
  float a[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) a[u] = 1e-3f * (threadIdx.x + u);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) a[u] = fmaf(a[u], b, c);
  }
  float t = 0;
#pragma unroll
  for (int u = 0; u < 16; ++u) t += a[u];
  if (t == 1.2345f) sink[0] = t;
}

// FP64 tensor-core MMA (m8n8k4, 512 flops per warp instruction), 4 independent accumulators per warp
__global__ void __launch_bounds__(kPeakThreads) k_peak_dmma(double* sink, int iters) {
  const double a = 1e-3 * (threadIdx.x & 31), b = 0.5;
  double c[4][2];
#pragma unroll
  for (int u = 0; u < 4; ++u) c[u][0] = c[u][1] = 1e-6 * u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[u][0]), "+d"(c[u][1])
                   : "d"(a), "d"(b));
  }
  double t = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) t += c[u][0] + c[u][1];
  if (t == 1.2345) sink[0] = t;
}

template <typename F>
float time_ms(F launch) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();   // warm-up
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

}  // namespace

extern "C" int gcamps_measure_peaks(double* tflops, int count) {
  if (!tflops || count < 3) return GCAMPS_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GCAMPS_ECUDA;
  double* sink = nullptr;
  if (cudaMalloc(&sink, 64) != cudaSuccess) return GCAMPS_ENOMEM;
  const int blocks = sms * 8;
  const double threads = (double)blocks * kPeakThreads;
  const int it64 = 1 << 15, it32 = 1 << 19, itmma = 1 << 16;
  const float ms64 = time_ms([&] { k_peak_fma64<<<blocks, kPeakThreads>>>(sink, it64, 0.999999, 1e-7); });
  const float ms32 = time_ms([&] {
    k_peak_fma32<<<blocks, kPeakThreads>>>(reinterpret_cast<float*>(sink), it32, 0.999999f, 1e-7f);
  });
  const float msmma = time_ms([&] { k_peak_dmma<<<blocks, kPeakThreads>>>(sink, itmma); });
  const cudaError_t ce = cudaGetLastError();
  cudaFree(sink);
  if (ce != cudaSuccess || ms64 <= 0.f || ms32 <= 0.f || msmma <= 0.f) return GCAMPS_ECUDA;
  tflops[0] = 2.0 * 8 * it64 * threads / (ms64 * 1e-3) / 1e12;
  tflops[1] = 2.0 * 16 * it32 * threads / (ms32 * 1e-3) / 1e12;
  tflops[2] = 512.0 * 4 * itmma * (threads / 32) / (msmma * 1e-3) / 1e12;
  return GCAMPS_OK;
}
