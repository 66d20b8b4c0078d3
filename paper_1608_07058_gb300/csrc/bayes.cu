// The Bayesian step after a simulation (paper Section 1): per-trajectory draws from the
// conjugate posterior Gamma(alpha_j + r_j, beta_j + G_j) of every rate constant, and
// systematic resampling of particles from log-weights.  Compiled without FMA contraction:
// the FP64 arithmetic follows a fixed operation order and reproduces an independent
// implementation of the same definitions bit for bit.
#include <cstdint>

#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "matleap.h"
#include "ml_internal.h"

namespace mlk {
namespace {

constexpr int kGammaMaxTrials = 64;

// Gamma(shape, rate) by Marsaglia & Tsang (2000): d = a - 1/3, c = 1/sqrt(9d); normal z by
// the Marsaglia polar method; v = (1 + c z)^3; accept iff log u < z^2/2 + d - d v + d log v;
// shape < 1 draws Gamma(shape + 1) and multiplies by U^(1/shape).  Counter (id, 0x80000000 +
// stream, 0, block): block 2t the polar pair of trial t, block 2t+1 the acceptance uniform
// (words 0, 1) and the boost uniform (words 2, 3).
__device__ double gamma_draw(double shape, double rate, uint32_t k0, uint32_t k1, uint32_t id,
                             uint32_t stream, uint32_t& flags) {
  if (!(shape > 0.0) || !(rate > 0.0)) return __longlong_as_double(0x7ff8000000000000LL);
  const bool boost = shape < 1.0;
  const double a = boost ? shape + 1.0 : shape;
  const double d = a - 1.0 / 3.0;
  const double c = 1.0 / sqrt(9.0 * d);
  const uint32_t cstep = 0x80000000u + stream;
  for (uint32_t t = 0; t < (uint32_t)kGammaMaxTrials; ++t) {
    const Words4 w = philox_block(k0, k1, id, cstep, 0u, 2u * t);
    const double v1 = 2.0 * u01_f64(w.w0, w.w1) - 1.0;
    const double v2 = 2.0 * u01_f64(w.w2, w.w3) - 1.0;
    const double s = v1 * v1 + v2 * v2;
    if (!(s < 1.0) || s == 0.0) continue;
    const double z = v1 * sqrt((-2.0 * refmath::log_ref(s)) / s);
    const double base = 1.0 + c * z;
    if (!(base > 0.0)) continue;
    const double v = (base * base) * base;
    const Words4 w2 = philox_block(k0, k1, id, cstep, 0u, 2u * t + 1u);
    const double u = u01_f64(w2.w0, w2.w1);
    if (refmath::log_ref(u) < ((0.5 * (z * z) + d) - d * v) + d * refmath::log_ref(v)) {
      double x = d * v;
      if (boost) {
        const double ub = u01_f64(w2.w2, w2.w3);
        x = x * refmath::exp_ref(refmath::log_ref(ub) / shape);
      }
      return x / rate;
    }
  }
  flags |= 1u;
  return shape / rate;
}

// One thread per (trajectory, reaction).
__global__ void k_posterior(int64_t n, int32_t M, const double* __restrict__ alpha,
                            int32_t alpha_per, const double* __restrict__ beta, int32_t beta_per,
                            const int64_t* __restrict__ r, const double* __restrict__ G,
                            uint64_t seed, uint64_t id_base, double* __restrict__ theta,
                            uint32_t* __restrict__ status) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * (long long)M) return;
  const long long i = e / M;
  const int j = (int)(e - i * M);
  const double al = alpha_per ? alpha[e] : alpha[j];
  const double be = beta_per ? beta[e] : beta[j];
  uint32_t flags = 0;
  theta[e] = gamma_draw(al + (double)r[e], be + G[e], (uint32_t)seed, (uint32_t)(seed >> 32),
                        (uint32_t)(id_base + (unsigned long long)i), (uint32_t)j, flags);
  if (status && flags) atomicOr(status + i, flags);
}

// ---- systematic resampling ----------------------------------------------------------
constexpr int kScanBlock = 1024;

// Per-block maximum of the log-weights (NaN never compares greater).
__global__ void k_block_max(int64_t n, const double* __restrict__ logw, double* __restrict__ out) {
  __shared__ double sm[32];
  double m = __longlong_as_double((long long)0xfff0000000000000ULL);  // -inf
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (logw[i] > m) m = logw[i];
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const double o = __shfl_xor_sync(0xffffffffu, m, d);
    m = o > m ? o : m;
  }
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : __longlong_as_double((long long)0xfff0000000000000ULL);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, m, d);
      m = o > m ? o : m;
    }
    if (threadIdx.x == 0) out[blockIdx.x] = m;
  }
}

__global__ void k_final_max(int nb, double* __restrict__ bmax) {  // one warp
  double m = __longlong_as_double((long long)0xfff0000000000000ULL);
  for (int i = threadIdx.x; i < nb; i += 32)
    if (bmax[i] > m) m = bmax[i];
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const double o = __shfl_xor_sync(0xffffffffu, m, d);
    m = o > m ? o : m;
  }
  __syncwarp();
  if (threadIdx.x == 0) bmax[0] = m;
}

// Quantized weights q_i = floor(exp(logw_i - max) 2^40) (0 for NaN) and their inclusive
// prefix within each block of kScanBlock; block totals to bsum.
__global__ void k_quantize_scan(int64_t n, const double* __restrict__ logw,
                                const double* __restrict__ mx_ptr, uint64_t* __restrict__ incl,
                                uint64_t* __restrict__ bsum) {
  __shared__ uint64_t sm[kScanBlock];
  const double mx = mx_ptr[0];
  const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
  uint64_t q = 0;
  if (i < n) {
    const double l = logw[i];
    const double wgt = l == l ? refmath::exp_ref(l - mx) : 0.0;
    q = (uint64_t)floor(wgt * 1099511627776.0);  // 2^40
  }
  sm[threadIdx.x] = q;
  __syncthreads();
  for (int d = 1; d < kScanBlock; d <<= 1) {  // Hillis-Steele inclusive scan (exact integers)
    const uint64_t add = threadIdx.x >= (unsigned)d ? sm[threadIdx.x - d] : 0;
    __syncthreads();
    sm[threadIdx.x] += add;
    __syncthreads();
  }
  if (i < n) incl[i] = sm[threadIdx.x];
  if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = sm[kScanBlock - 1];
}

// Exclusive prefix of the block totals, one CTA walking the totals in chunks.
__global__ void k_scan_blocks(int nb, uint64_t* __restrict__ bsum) {
  __shared__ uint64_t sm[kScanBlock];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += kScanBlock) {
    const int i = base + threadIdx.x;
    const uint64_t v = i < nb ? bsum[i] : 0;
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int d = 1; d < kScanBlock; d <<= 1) {
      const uint64_t add = threadIdx.x >= (unsigned)d ? sm[threadIdx.x - d] : 0;
      __syncthreads();
      sm[threadIdx.x] += add;
      __syncthreads();
    }
    const uint64_t c = carry;
    if (i < nb) bsum[i] = c + sm[threadIdx.x] - v;  // exclusive
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry = c + sm[kScanBlock - 1];
    __syncthreads();
  }
}

__global__ void k_add_offsets(int64_t n, uint64_t* __restrict__ incl,
                              const uint64_t* __restrict__ boff) {
  const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) incl[i] += boff[blockIdx.x];
}

// Ancestor k: the first i whose inclusive prefix exceeds (k Q + floor(u Q)) / n.
__global__ void k_ancestors(int64_t n, const uint64_t* __restrict__ incl,
                            const double* __restrict__ mx_ptr, uint64_t seed, uint64_t id_base,
                            int64_t* __restrict__ anc) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double mx = mx_ptr[0];
  const uint64_t Q = incl[n - 1];
  if (!(mx > __longlong_as_double((long long)0xfff0000000000000ULL)) ||
      mx == __longlong_as_double(0x7ff0000000000000LL) || Q == 0) {
    anc[k] = -1;
    return;
  }
  const Words4 w = philox_block((uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)id_base,
                                0xC0000000u, 0u, 0u);
  const double u = u01_f64(w.w0, w.w1);
  const unsigned __int128 uQ = (unsigned __int128)(uint64_t)floor(u * (double)Q);
  const uint64_t target =
      (uint64_t)(((unsigned __int128)k * Q + uQ) / (unsigned __int128)(uint64_t)n);
  long long lo = 0, hi = n - 1;  // first index with incl > target (exists: target < Q)
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (incl[mid] > target) hi = mid;
    else lo = mid + 1;
  }
  anc[k] = lo;
}

size_t resample_ws(int64_t n) {
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  return 256 + (size_t)n * 8 + (size_t)nb * 8 + 256;
}

}  // namespace
}  // namespace mlk

extern "C" {

int ml_posterior_sample(int64_t n, int32_t M, const double* alpha, int32_t alpha_per_traj,
                        const double* beta, int32_t beta_per_traj, const int64_t* r,
                        const double* G, uint64_t seed, uint64_t traj_id_base, double* theta_out,
                        uint32_t* status_out, void* stream) {
  using namespace mlk;
  if (n < 0 || M < 1 || M > 4096) return set_error(ML_ERR_ARG, "need n >= 0 and 1 <= M <= 4096");
  if (traj_id_base > 0xffffffffULL || (uint64_t)n > 0x100000000ULL - traj_id_base)
    return set_error(ML_ERR_ARG, "trajectory ids must stay below 2^32");
  if (n == 0) return ML_OK;
  const void* req[] = {alpha, beta, r, G, theta_out};
  for (const void* p : req)
    if (!is_device_pointer(p)) return set_error(ML_ERR_ARG, "alpha, beta, r, G and theta_out must be device memory");
  if (status_out && !is_device_pointer(status_out)) return set_error(ML_ERR_ARG, "status_out must be device memory");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (status_out) {
    cudaError_t e = cudaMemsetAsync(status_out, 0, (size_t)n * 4, s);
    if (e != cudaSuccess) return set_error(ML_ERR_CUDA, cudaGetErrorString(e));
  }
  const long long total = n * (long long)M;
  const int block = 256;
  const long long grid = (total + block - 1) / block;
  if (grid > 0x7fffffffLL) return set_error(ML_ERR_ARG, "n * M too large for one launch");
  k_posterior<<<(unsigned)grid, block, 0, s>>>(n, M, alpha, alpha_per_traj, beta, beta_per_traj,
                                                r, G, seed, traj_id_base, theta_out, status_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ML_OK : set_error(ML_ERR_CUDA, cudaGetErrorString(e));
}

size_t ml_resample_workspace_bytes(int64_t n) { return n < 1 ? 0 : mlk::resample_ws(n); }

int ml_resample_systematic(int64_t n, const double* logw, uint64_t seed, uint64_t id_base,
                           int64_t* ancestors, void* workspace, size_t workspace_bytes,
                           void* stream) {
  using namespace mlk;
  // q_i <= 2^40, so the 64-bit prefix sums stay exact for n < 2^24.
  if (n < 1 || n >= (1LL << 24)) return set_error(ML_ERR_ARG, "need 1 <= n < 2^24");
  if (!is_device_pointer(logw) || !is_device_pointer(ancestors) || !is_device_pointer(workspace))
    return set_error(ML_ERR_ARG, "logw, ancestors and workspace must be device memory");
  if (workspace_bytes < resample_ws(n))
    return set_error(ML_ERR_ARG, "workspace smaller than ml_resample_workspace_bytes(n)");
  if (reinterpret_cast<uintptr_t>(workspace) % 16)
    return set_error(ML_ERR_ARG, "workspace must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  double* mx = reinterpret_cast<double*>(ws);                 // [0, 256): maxima
  uint64_t* incl = reinterpret_cast<uint64_t*>(ws + 256);     // n inclusive prefixes
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  uint64_t* bsum = incl + n;                                  // nb block totals
  const int red_blocks = (int)(nb < 32 ? nb : 32);
  k_block_max<<<red_blocks, 256, 0, s>>>(n, logw, mx);
  k_final_max<<<1, 32, 0, s>>>(red_blocks, mx);
  k_quantize_scan<<<(unsigned)nb, kScanBlock, 0, s>>>(n, logw, mx, incl, bsum);
  k_scan_blocks<<<1, kScanBlock, 0, s>>>((int)nb, bsum);
  k_add_offsets<<<(unsigned)nb, kScanBlock, 0, s>>>(n, incl, bsum);
  k_ancestors<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, incl, mx, seed, id_base, ancestors);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ML_OK : set_error(ML_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
