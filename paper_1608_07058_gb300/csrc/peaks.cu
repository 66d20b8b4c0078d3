// Pipe-throughput microbenchmarks for the roofline of the simulation kernels: FP64 FMA,
// FP32 FMA and the special-function unit (base-2 logarithm), each as 8 independent
// dependency chains per thread over a grid of 8 CTAs of 256 threads per SM, sized to run
// about 20 ms.  The results feed only the benchmark's report.
#include <cstdint>

#include <cuda_runtime.h>

#include "matleap.h"
#include "ml_internal.h"

namespace mlk {
namespace {

__device__ double g_peak_sink;  // written only if a result is impossible (keeps the work)

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_peak_fma(int iters, T seed, T mul, T add) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], mul, add);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == T(-1)) g_peak_sink = (double)s;
}

// x <- log2(x) + 2 converges to 4 and stays finite; one special-function op per step.
__global__ void __launch_bounds__(kThreads) k_peak_lg2(int iters, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = __log2f(a[c]) + 2.0f;
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.f) g_peak_sink = (double)s;
}

// Runs `launch(iters)` sized to ~20 ms from a short probe; returns ops per second.
template <class F>
int time_ops(F launch, double ops_per_iter, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
             double* out) {
  int iters = 256;
  float ms = 0.f;
  for (int round = 0; round < 3; ++round) {
    cudaEventRecord(e0, s);
    launch(iters);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return set_error(ML_ERR_CUDA, cudaGetErrorString(e));
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ML_ERR_CUDA, cudaGetErrorString(e));
    cudaEventElapsedTime(&ms, e0, e1);
    if (round < 2) {
      const double scale = 20.0 / (ms > 1e-3f ? ms : 1e-3f);
      const double next = iters * scale;
      iters = (int)(next < 1 << 28 ? (next > 256 ? next : 256) : 1 << 28);
    }
  }
  *out = ops_per_iter * iters / (ms * 1e-3);
  return ML_OK;
}

}  // namespace
}  // namespace mlk

extern "C" int ml_measure_pipe_peaks(double* out3, void* stream) {
  using namespace mlk;
  if (!out3) return set_error(ML_ERR_ARG, "out3 is NULL");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(ML_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = sms * 8;
  const double lanes = (double)grid * kThreads * kChains;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = time_ops([&](int it) { k_peak_fma<double><<<grid, kThreads, 0, s>>>(it, 1.0, 0.999999, 1e-7); },
                    2.0 * lanes, s, e0, e1, &out3[0]);
  if (rc == ML_OK)
    rc = time_ops([&](int it) { k_peak_fma<float><<<grid, kThreads, 0, s>>>(it, 1.0f, 0.999999f, 1e-7f); },
                  2.0 * lanes, s, e0, e1, &out3[1]);
  if (rc == ML_OK)
    rc = time_ops([&](int it) { k_peak_lg2<<<grid, kThreads, 0, s>>>(it, 3.0f); }, lanes, s, e0,
                  e1, &out3[2]);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}
