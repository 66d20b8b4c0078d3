// Accuracy metric of the paper's Section 3 (Table 1): the Kullback-Leibler divergence of
// a method's marginal distributions from those of exact SSA, per time point and species,
// averaged over all of them.  Binned, half-count-smoothed empirical distributions (the
// paper does not say how it forms them): bins of integer width w = ceil((hi - lo + 1) /
// max_bins) on the pooled range of both samples, 1/2 added to every bin.  Compiled without
// FMA contraction; the counts are exact integers and the FP64 sums take a fixed lane
// order, so the results are bit-reproducible.
#include <cstdint>

#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "matleap.h"
#include "ml_internal.h"

namespace mlk {
namespace {

constexpr int kKlThreads = 256;
constexpr int kKlMaxBins = 4096;

__device__ __forceinline__ long long warp_min(long long v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const long long o = __shfl_xor_sync(0xffffffffu, v, d);
    v = o < v ? o : v;
  }
  return v;
}

__device__ __forceinline__ long long warp_max(long long v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const long long o = __shfl_xor_sync(0xffffffffu, v, d);
    v = o > v ? o : v;
  }
  return v;
}

// Sum in the canonical order: lane l adds elements l, l + 32, ... in increasing index
// (an empty lane holds 0), then lanes combine pairwise at xor distances 16, 8, 4, 2, 1.
// Called by one full warp; every lane returns the sum.
template <class F>
__device__ __forceinline__ double lane_tree(int n, int lane, F elem) {
  double v = 0.0;
  for (int j = lane; j < n; j += 32) v = (j < 32) ? elem(j) : v + elem(j);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v = v + __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// One CTA per (time point k, species s).  X layout [n][K][N].
__global__ void __launch_bounds__(kKlThreads) k_kl(int64_t n_ref, const int64_t* __restrict__ Xr,
                                                  int64_t n_test, const int64_t* __restrict__ Xt,
                                                  int K, int N, int max_bins,
                                                  double* __restrict__ kl) {
  __shared__ unsigned int ca[kKlMaxBins], cb[kKlMaxBins];
  __shared__ long long red_lo[kKlThreads / 32], red_hi[kKlThreads / 32];
  const int ks = blockIdx.x;  // k * N + s
  const long long stride = (long long)K * N;
  const int64_t* a = Xr + ks;
  const int64_t* b = Xt + ks;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // pooled range (exact integer reductions)
  long long lo = a[0], hi = a[0];
  for (long long i = threadIdx.x; i < n_ref; i += blockDim.x) {
    const long long v = a[i * stride];
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
  for (long long i = threadIdx.x; i < n_test; i += blockDim.x) {
    const long long v = b[i * stride];
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  if (lane == 0) {
    red_lo[warp] = lo;
    red_hi[warp] = hi;
  }
  for (int j = threadIdx.x; j < kKlMaxBins; j += blockDim.x) ca[j] = cb[j] = 0u;
  __syncthreads();
  lo = red_lo[0];
  hi = red_hi[0];
  for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
    lo = red_lo[q] < lo ? red_lo[q] : lo;
    hi = red_hi[q] > hi ? red_hi[q] : hi;
  }
  // bin width w = ceil((d + 1) / max_bins) = floor(d / max_bins) + 1 with d = hi - lo, in
  // unsigned arithmetic so that any pair of int64 values gives a bin index < max_bins
  const unsigned long long d = (unsigned long long)hi - (unsigned long long)lo;
  const unsigned long long w = d / (unsigned long long)max_bins + 1ull;
  const int nbins = (int)(d / w + 1ull);

  for (long long i = threadIdx.x; i < n_ref; i += blockDim.x)
    atomicAdd(&ca[((unsigned long long)a[i * stride] - (unsigned long long)lo) / w], 1u);
  for (long long i = threadIdx.x; i < n_test; i += blockDim.x)
    atomicAdd(&cb[((unsigned long long)b[i * stride] - (unsigned long long)lo) / w], 1u);
  __syncthreads();

  if (warp == 0) {
    const double da = (double)n_ref + 0.5 * (double)nbins;
    const double db = (double)n_test + 0.5 * (double)nbins;
    const double sum = lane_tree(nbins, lane, [&](int j) {
      const double p = ((double)ca[j] + 0.5) / da;
      const double q = ((double)cb[j] + 0.5) / db;
      return p * (refmath::log_ref(p) - refmath::log_ref(q));
    });
    if (lane == 0) kl[ks] = sum;
  }
}

// Mean over the K x N divergences in the canonical lane order (one warp).
__global__ void k_kl_mean(int n, const double* __restrict__ kl, double* __restrict__ mean) {
  const double s = lane_tree(n, threadIdx.x & 31, [&](int j) { return kl[j]; });
  if (threadIdx.x == 0) *mean = s / (double)n;
}

}  // namespace
}  // namespace mlk

extern "C" int ml_kl_divergence(int64_t n_ref, const int64_t* X_ref, int64_t n_test,
                                const int64_t* X_test, int32_t K, int32_t N, int32_t max_bins,
                                double* kl_out, double* kl_mean_out, void* stream) {
  using namespace mlk;
  if (n_ref < 1 || n_test < 1 || n_ref >= (1LL << 31) || n_test >= (1LL << 31))
    return set_error(ML_ERR_ARG, "need 1 <= n_ref, n_test < 2^31");
  if (K < 1 || N < 1 || (int64_t)K * N > 0x7fffffffLL)
    return set_error(ML_ERR_ARG, "need K >= 1, N >= 1 and K * N < 2^31");
  if (max_bins < 1 || max_bins > kKlMaxBins)
    return set_error(ML_ERR_ARG, "need 1 <= max_bins <= 4096");
  if (!is_device_pointer(X_ref) || !is_device_pointer(X_test) || !is_device_pointer(kl_out))
    return set_error(ML_ERR_ARG, "X_ref, X_test and kl_out must be device memory");
  if (kl_mean_out && !is_device_pointer(kl_mean_out))
    return set_error(ML_ERR_ARG, "kl_mean_out must be device memory");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_kl<<<(unsigned)(K * N), kKlThreads, 0, s>>>(n_ref, X_ref, n_test, X_test, K, N, max_bins,
                                                 kl_out);
  if (kl_mean_out) k_kl_mean<<<1, 32, 0, s>>>(K * N, kl_out, kl_mean_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ML_OK : set_error(ML_ERR_CUDA, cudaGetErrorString(e));
}
