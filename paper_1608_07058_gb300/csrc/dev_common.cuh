// Device building blocks: counter-based random numbers, the FP64 elementary functions
// of the reference-precision path, and bulk staging of model tables into shared memory.
#pragma once
#ifndef __CUDACC_RTC__  // runtime compilation (model-specialized kernels) brings its own types
#include <cstdint>

#include <cuda_runtime.h>
#endif

namespace mlk {

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC11): ten rounds, each two 32x32->64
// products of counter words 0 and 2 with fixed multipliers, xored into the other words
// with the key, the key bumped by two Weyl constants between rounds.
// Counter = (trajectory id, step, stream, block), key = (seed lo, seed hi).
// ---------------------------------------------------------------------------------
struct Words4 {
  uint32_t w0, w1, w2, w3;
};

__device__ __forceinline__ Words4 philox_block(uint32_t k0, uint32_t k1, uint32_t id,
                                               uint32_t step, uint32_t stream,
                                               uint32_t block) {
  uint32_t c0 = id, c1 = step, c2 = stream, c3 = block;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo_a = 0xD2511F53u * c0;
    const uint32_t hi_a = __umulhi(0xD2511F53u, c0);
    const uint32_t lo_b = 0xCD9E8D57u * c2;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi_b ^ c1 ^ k0;
    const uint32_t n2 = hi_a ^ c3 ^ k1;
    c0 = n0;
    c1 = lo_b;
    c2 = n2;
    c3 = lo_a;
  }
  return Words4{c0, c1, c2, c3};
}

// FP64 uniform in (0,1) from two words: 52 bits n, u = (n + 1/2) 2^-52 (exact).
__device__ __forceinline__ double u01_f64(uint32_t hi, uint32_t lo) {
  const double n = (double)(hi >> 6) * 67108864.0 + (double)(lo >> 6);
  return (n + 0.5) * 0x1p-52;
}

// FP32 uniform in (0,1) from one word: 23 bits n, u = (n + 1/2) 2^-23 (exact).
__device__ __forceinline__ float u01_f32(uint32_t w) {
  return ((float)(w >> 9) + 0.5f) * 0x1p-23f;
}

// ---------------------------------------------------------------------------------
// FP64 elementary functions of the reference path (Cody & Waite 1980 style): additive
// reduction by k ln2 with ln2 split in a 32-bit head and a tail, then a polynomial.
// Only +,-,*,/ (the reference translation unit is compiled without FMA contraction),
// so the results are fixed by the operation order below.
// ---------------------------------------------------------------------------------
namespace refmath {
constexpr double kLn2Head = 0x1.62e42fee00000p-1;   // 32 leading bits of ln 2
constexpr double kLn2Tail = 0x1.a39ef35793c76p-33;  // ln 2 - kLn2Head
constexpr double kInvLn2 = 0x1.71547652b82fep+0;
constexpr double kSqrt2 = 0x1.6a09e667f3bcdp+0;
constexpr double kHalfLog2Pi = 0x1.d67f1c864beb5p-1;

// exp(x) on [-708, 709]: x = k ln2 + r, Taylor series of e^r to r^13 by Horner.
__device__ __forceinline__ double exp_ref(double x) {
  if (x != x) return x;
  if (x < -708.0) return 0.0;
  if (x > 709.0) return __longlong_as_double(0x7ff0000000000000LL);
  const double kd = floor(x * kInvLn2 + 0.5);
  const double r = (x - kd * kLn2Head) - kd * kLn2Tail;
  double p = 1.0 / 6227020800.0;
  p = p * r + 1.0 / 479001600.0;
  p = p * r + 1.0 / 39916800.0;
  p = p * r + 1.0 / 3628800.0;
  p = p * r + 1.0 / 362880.0;
  p = p * r + 1.0 / 40320.0;
  p = p * r + 1.0 / 5040.0;
  p = p * r + 1.0 / 720.0;
  p = p * r + 1.0 / 120.0;
  p = p * r + 1.0 / 24.0;
  p = p * r + 1.0 / 6.0;
  p = p * r + 0.5;
  p = p * r + 1.0;
  p = p * r + 1.0;
  const long long k = (long long)kd;
  return p * __longlong_as_double((k + 1023LL) << 52);
}

// log(x) for positive normal x: x = 2^e m, m in [sqrt(1/2), sqrt(2)); with f = m - 1 and
// s = f/(2+f), log m = 2 atanh s = 2s (1 + z/3 + ... + z^11/23), z = s^2.
__device__ __forceinline__ double log_ref(double x) {
  if (x != x || x < 0.0) return __longlong_as_double(0x7ff8000000000000LL);
  if (x == 0.0) return __longlong_as_double((long long)0xfff0000000000000ULL);
  if (x == __longlong_as_double(0x7ff0000000000000LL)) return x;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7ffULL) - 1023;
  double m = __longlong_as_double(
      (long long)((bits & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL));
  if (m > kSqrt2) {
    m = m * 0.5;
    e = e + 1;
  }
  const double f = m - 1.0;
  const double s = f / (2.0 + f);
  const double z = s * s;
  double q = 1.0 / 23.0;
  q = q * z + 1.0 / 21.0;
  q = q * z + 1.0 / 19.0;
  q = q * z + 1.0 / 17.0;
  q = q * z + 1.0 / 15.0;
  q = q * z + 1.0 / 13.0;
  q = q * z + 1.0 / 11.0;
  q = q * z + 1.0 / 9.0;
  q = q * z + 1.0 / 7.0;
  q = q * z + 1.0 / 5.0;
  q = q * z + 1.0 / 3.0;
  const double two_s = s + s;
  const double logm = two_s + (two_s * z) * q;
  const double ed = (double)e;
  return ed * kLn2Head + (ed * kLn2Tail + logm);
}

// log k!: exact product then log below 16; Stirling series of log Gamma(k+1) from 16.
__device__ __forceinline__ double log_factorial_ref(long long k) {
  if (k < 2) return 0.0;
  if (k < 16) {
    double f = 1.0;
    for (long long i = 2; i <= k; ++i) f = f * (double)i;
    return log_ref(f);
  }
  const double z = (double)k + 1.0;
  const double w = 1.0 / z;
  const double w2 = w * w;
  double ser = 1.0 / 1188.0;
  ser = ser * w2 - 1.0 / 1680.0;
  ser = ser * w2 + 1.0 / 1260.0;
  ser = ser * w2 - 1.0 / 360.0;
  ser = ser * w2 + 1.0 / 12.0;
  ser = ser * w;
  return (((z - 0.5) * log_ref(z) - z) + kHalfLog2Pi) + ser;
}
}  // namespace refmath

// ---------------------------------------------------------------------------------
// Persistent form: the next trajectory to run.  The k-th claim on the work queue is
// trajectory order[k] when the caller gave an order (meant to be a permutation of
// 0..n-1, longest first), else trajectory k.  Entries outside [0, n) are passed over, so a
// malformed order cannot index out of bounds (trajectories it leaves out are not run).
// Returns n_traj when the queue is exhausted.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ long long queue_claim(unsigned long long* queue, const int64_t* order,
                                                 long long n_traj) {
  for (;;) {
    const long long k = (long long)atomicAdd(queue, 1ULL);
    if (k >= n_traj) return n_traj;
    if (!order) return k;
    const long long i = __ldg(order + k);
    if (i >= 0 && i < n_traj) return i;
  }
}

// ---------------------------------------------------------------------------------
// Model staging: one bulk asynchronous copy (TMA engine, cp.async.bulk) of the model
// tables from global to shared memory, completed on an mbarrier.  The wait is bounded
// (poll_limit polls per thread); if it runs out the CTA waits again, bounded, for its copy
// in flight, then copies the tables with plain loads and reports it.
// bytes must be a multiple of 16 and both addresses 16-byte aligned.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ bool stage_model_bulk(void* smem_dst, const void* gmem_src,
                                                 uint32_t bytes, uint64_t* mbar,
                                                 int poll_limit) {
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(mbar);
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem_dst);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile(
        "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "l"(gmem_src), "r"(bytes), "r"(bar)
        : "memory");
  }
  // every thread waits on phase 0, at most poll_limit polls
  uint32_t done = 0;
  for (int it = 0; it < poll_limit && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar)
        : "memory");
  }
  const int ok = __syncthreads_and((int)done);
  if (!ok) {
    // The copy may still be in flight: wait again (bounded) before overwriting.
    for (int it = 0; it < (1 << 22) && !done; ++it) {
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(bar)
          : "memory");
    }
    __syncthreads();
    const uint4* src = reinterpret_cast<const uint4*>(gmem_src);
    uint4* d = reinterpret_cast<uint4*>(smem_dst);
    for (uint32_t k = threadIdx.x; k < bytes / 16; k += blockDim.x) d[k] = src[k];
    __syncthreads();
  }
  return ok != 0;
}

}  // namespace mlk
