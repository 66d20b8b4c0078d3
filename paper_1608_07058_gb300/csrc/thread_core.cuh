// One trajectory per thread: the adaptive explicit-implicit tau-leaping loop for small
// networks (N <= 8 species, M <= 16 reactions), templated on the table capacities
// (NM, MM) and on the arithmetic (P = PrecRef: FP64, fixed operation order, bitwise
// reproducible; P = PrecFast: FP32 propensities, step sizes, Poisson means and G
// increments, FP64 time and G totals, and an FP64 implicit Newton solve -- or, on
// request, an FP32 solve for the increment).  All per-trajectory arrays are indexed with
// compile-time indices only so that they live in registers.
//
// Steps (paper Section 2, with the published methods it names):
//   propensities a_j = theta_j g_j(x), a0                       (Section 1)
//   critical reactions: a_j > 0 and min_s floor(x_s/|nu_js|) < n_c
//   tau_ex: Cao 2006 bound on mean and variance of each reactant's change
//   partial-equilibrium pairs, tau_im without them, implicit iff tau_im >> tau_ex
//   tau2 ~ Exp(a0c); SSA burst if min(tau1, tau2) < ssa_factor / a0
//   explicit Poisson leap or implicit Newton leap (Rathinam 2003); one critical firing
//   negativity check (halve tau1 and retry); commit x, r, G (trapezoid) and t.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

#include "dev_common.cuh"
#include "ml_internal.h"
#include "matleap.h"

namespace mlk {

// Canonical sum over reactions for a0 and a0c: element j on lane j (j < 32); lanes
// combined pairwise at xor distances 16, 8, 4, 2, 1; lane 0's value.  Written for one
// thread holding all elements (MM <= 32), with empty lanes holding 0.
template <int MM, class R>
__device__ __forceinline__ R lane_tree_sum(const R (&v)[MM]) {
  static_assert(MM <= 32, "thread variant holds at most 32 reactions");
  R lane[32];
#pragma unroll
  for (int l = 0; l < 32; ++l) lane[l] = (l < MM) ? v[l] : R(0);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
#pragma unroll
    for (int l = 0; l < d; ++l) lane[l] = lane[l] + lane[l + d];
  }
  return lane[0];
}

// Sum over reactions: the canonical lane tree in reference precision (bitwise parity with
// the CPU reference); fast precision may add in any order and adds sequentially (the tree
// over 32 lanes costs 31 additions, most of them of zeros that IEEE arithmetic cannot
// drop).
template <int MM, class R, bool kRef>
__device__ __forceinline__ R reaction_sum(const R (&v)[MM]) {
  if (kRef) return lane_tree_sum<MM, R>(v);
  R s = v[0];
#pragma unroll
  for (int j = 1; j < MM; ++j) s = s + v[j];
  return s;
}

// C(v, m) for m = 1, 2, 3 on a real argument, in this operation order.
template <class R>
__device__ __forceinline__ R comb_factor(R v, int m) {
  if (m == 1) return v;
  if (m == 2) return (v * (v - R(1))) * R(0.5);
  return ((v * (v - R(1))) * (v - R(2))) / R(6);
}

// d/dv C(v, m): 1, v - 1/2, (3 v^2 - 6 v + 2) / 6, in this operation order.
template <class T>
__device__ __forceinline__ T comb_factor_deriv(T v, int m) {
  if (m == 1) return T(1);
  if (m == 2) return v - T(0.5);
  return ((T(3) * (v * v) - T(6) * v) + T(2)) / T(6);
}

// C(x + z, m) - C(x, m) written as z times a polynomial, so that no two large nearby
// values are subtracted: m = 2: z (2x + z - 1) / 2; m = 3 with u = x + z:
// z (u^2 + u x + x^2 - 3 (u + x) + 2) / 6.
template <class R>
__device__ __forceinline__ R comb_diff(R xv, R z, int m) {
  if (m == 1) return z;
  if (m == 2) return (z * ((R(2) * xv + z) - R(1))) * R(0.5);
  const R u = xv + z;
  return (z * (((u * u + u * xv) + xv * xv) - R(3) * (u + xv) + R(2))) / R(6);
}

// Double-float (hi + lo FP32 pair) arithmetic for the fast-precision reaction pick: sums
// by TwoSum (Knuth) renormalized with Fast2Sum, about 46 significant bits, all on the
// FP32 pipe.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_norm(float s, float e) {
  const float hi = s + e;
  return DF{hi, e - (hi - s)};
}
__device__ __forceinline__ DF df_add(DF a, float b) {
  const float s = a.hi + b;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b - bb);
  return df_norm(s, err + a.lo);
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb);
  return df_norm(s, err + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
__device__ __forceinline__ bool df_lt(DF a, DF b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
// u * t for a 48-bit uniform u = (w_hi>>8) 2^-24 + ((w_lo>>8) + 1/2) 2^-48 in (0, 1).
__device__ __forceinline__ DF df_uniform_times(DF t, uint32_t w_hi, uint32_t w_lo) {
  const float uh = (float)(w_hi >> 8) * 0x1p-24f;
  const float ul = ((float)(w_lo >> 8) + 0.5f) * 0x1p-48f;
  const float p = uh * t.hi;
  const float e = fmaf(uh, t.hi, -p);
  return df_norm(p, e + (uh * t.lo + ul * t.hi));
}

// Compensated (Kahan) FP32 accumulation: the sum is s - c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Highest-order-reaction factor h_s (Cao 2006) from the species' flags and count.
template <class R>
__device__ __forceinline__ R hor_factor(uint8_t f, long long x) {
  const R xd = (R)x;
  R h = R(0);
  if (f & kHorO1) h = h < R(1) ? R(1) : h;
  if (f & kHorO2M1) h = h < R(2) ? R(2) : h;
  if (f & kHorO2M2) {
    const R v = x >= 2 ? R(2) + R(1) / (xd - R(1)) : R(2);
    h = h < v ? v : h;
  }
  if (f & kHorO3M1) h = h < R(3) ? R(3) : h;
  if (f & kHorO3M2) {
    const R v = x >= 2 ? R(1.5) * (R(2) + R(1) / (xd - R(1))) : R(3);
    h = h < v ? v : h;
  }
  if (f & kHorO3M3) {
    const R v = x >= 3 ? (R(3) + R(1) / (xd - R(1))) + R(2) / (xd - R(2)) : R(3);
    h = h < v ? v : h;
  }
  return h;
}

struct PrecRef {
  using R = double;
  static constexpr bool kRef = true;
  __device__ static __forceinline__ R u(const Words4& w, int k) {
    return k == 0 ? u01_f64(w.w0, w.w1) : u01_f64(w.w2, w.w3);
  }
  __device__ static __forceinline__ R log(R x) { return refmath::log_ref(x); }
  __device__ static __forceinline__ R exp(R x) { return refmath::exp_ref(x); }
  __device__ static __forceinline__ R lfact(long long k) {
    return refmath::log_factorial_ref(k);
  }
  __device__ static __forceinline__ R sqrt(R x) { return ::sqrt(x); }
  __device__ static __forceinline__ R log1p(R x) { return ::log1p(x); }  // unused
  __device__ static __forceinline__ R inf() {
    return __longlong_as_double(0x7ff0000000000000LL);
  }
};

struct PrecFast {
  using R = float;
  static constexpr bool kRef = false;
  __device__ static __forceinline__ R u(const Words4& w, int k) {
    return k == 0 ? u01_f32(w.w0) : u01_f32(w.w2);
  }
  // accurate logf: the waiting times -log(u)/a0 need relative accuracy for u near 1,
  // where the hardware approximation's absolute error would bias the clock
  __device__ static __forceinline__ R log(R x) { return logf(x); }
  __device__ static __forceinline__ R exp(R x) { return __expf(x); }
  __device__ static __forceinline__ R lfact(long long k) {
    return lgammaf((float)k + 1.0f);
  }
  __device__ static __forceinline__ R sqrt(R x) { return sqrtf(x); }
  __device__ static __forceinline__ R log1p(R x) { return log1pf(x); }
  __device__ static __forceinline__ R inf() { return __int_as_float(0x7f800000); }
};

// FP64 PTRS with library functions, used by the fast path for very large means where
// FP32 cannot hold the integer count exactly.
struct PrecWide {
  using R = double;
  static constexpr bool kRef = false;
  __device__ static __forceinline__ R u(const Words4& w, int k) {
    return k == 0 ? u01_f64(w.w0, w.w1) : u01_f64(w.w2, w.w3);
  }
  __device__ static __forceinline__ R log(R x) { return ::log(x); }
  __device__ static __forceinline__ R exp(R x) { return ::exp(x); }
  __device__ static __forceinline__ R lfact(long long k) { return ::lgamma((double)k + 1.0); }
  __device__ static __forceinline__ R sqrt(R x) { return ::sqrt(x); }
  __device__ static __forceinline__ R log1p(R x) { return ::log1p(x); }
  __device__ static __forceinline__ R inf() {
    return __longlong_as_double(0x7ff0000000000000LL);
  }
};

constexpr int kPtrsMaxTrials = 256;

// PTRS: Hoermann (1993), transformed rejection with squeeze, for mean mu >= 10.  Trial b
// uses block b of the stream: U from the first uniform, V from the second.
struct PoissonDraw {
  long long k;
  uint32_t flags;  // ML_ST_PTRS_CAP when the trial cap was hit
};

template <class P>
__device__ __noinline__ PoissonDraw poisson_ptrs(typename P::R mu, uint32_t k0, uint32_t k1,
                                                 uint32_t id, uint32_t step, uint32_t stream) {
  using R = typename P::R;
  const R slam = P::sqrt(mu);
  const R loglam = P::log(mu);
  const R b = R(0.931) + R(2.53) * slam;
  const R a = R(-0.059) + R(0.02483) * b;
  const R inv_alpha = R(1.1239) + R(1.1328) / (b - R(3.4));
  const R v_r = R(0.9277) - R(3.6224) / (b - R(2));
  for (uint32_t trial = 0; trial < (uint32_t)kPtrsMaxTrials; ++trial) {
    const Words4 w = philox_block(k0, k1, id, step, stream, trial);
    const R U = P::u(w, 0) - R(0.5);
    const R V = P::u(w, 1);
    const R us = R(0.5) - fabs(U);
    const R kd = floor((((R(2) * a) / us + b) * U + mu) + R(0.43));
    if (us >= R(0.07) && V <= v_r) return PoissonDraw{(long long)kd, 0u};
    if (kd < R(0) || (us < R(0.013) && V > us)) continue;
    const R lhs = (P::log(V) + P::log(inv_alpha)) - P::log(a / (us * us) + b);
    R rhs;
    if (P::kRef || kd < R(10)) {
      rhs = (-mu + kd * loglam) - P::lfact((long long)kd);
    } else {
      // log of the Poisson pmf without cancellation: with z = k + 1 and Stirling's series
      // for log Gamma(z), -mu + k log mu - log k! =
      //   (z - mu) + (z - 1) log1p((mu - z)/z) - log(z)/2 - log(2 pi)/2 - 1/(12 z) + 1/(360 z^3)
      const R z = kd + R(1);
      const R iz = R(1) / z;
      rhs = ((z - mu) + (z - R(1)) * P::log1p((mu - z) * iz)) - R(0.5) * P::log(z) -
            R(0.91893853320467274178) - iz * (R(1) / R(12) - (iz * iz) * (R(1) / R(360)));
    }
    if (lhs <= rhs) return PoissonDraw{(long long)kd, 0u};
  }
  return PoissonDraw{(long long)floor(mu + R(0.5)), ML_ST_PTRS_CAP};
}

// Poisson(mu): 0 for mu <= 0 (no draw); inversion by sequential search below 10; PTRS.
template <class P>
__device__ __forceinline__ PoissonDraw poisson_sample(typename P::R mu, uint32_t k0, uint32_t k1,
                                                   uint32_t id, uint32_t step, uint32_t stream) {
  using R = typename P::R;
  if (!(mu > R(0))) return PoissonDraw{0, 0u};
  if (mu < R(10)) {
    const Words4 w = philox_block(k0, k1, id, step, stream, 0);
    const R u = P::u(w, 0);
    R p = P::exp(-mu);
    R F = p;
    long long k = 0;
    while (u > F) {
      k = k + 1;
      p = p * (mu / (R)k);
      if (p == R(0)) break;
      F = F + p;
    }
    return PoissonDraw{k, 0u};
  }
  return (!P::kRef && mu > R(4.0e6)) ? poisson_ptrs<PrecWide>((double)mu, k0, k1, id, step, stream)
                                     : poisson_ptrs<P>(mu, k0, k1, id, step, stream);
}

template <class P>
__device__ __forceinline__ long long poisson_draw(typename P::R mu, uint32_t k0, uint32_t k1,
                                                  uint32_t id, uint32_t step, uint32_t stream,
                                                  uint32_t& status) {
  const PoissonDraw d = poisson_sample<P>(mu, k0, k1, id, step, stream);
  status |= d.flags;
  return d.k;
}

// MDL: the model tables' type -- the shared-memory ThreadModel staged at kernel start, or
// a type with the same members known at compile time.
template <int NM, int MM, class P, class MDL = ThreadModel<NM, MM>>
struct ThreadTraj {
  using R = typename P::R;
  using Model = MDL;

  // g_j at an integer state (0 when some x_s < m_js), product in increasing s.
  __device__ static __forceinline__ R g_int(const Model& md, int j, const long long (&x)[NM]) {
    R v = R(1);
    bool zero = false;
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      const int m = md.ord[j][s];
      if (m != 0) {
        if (x[s] < m) zero = true;
        else v = v * comb_factor<R>((R)x[s], m);
      }
    }
    return zero ? R(0) : v;
  }

  // Fast precision: g_j from an FP32 copy of the state (exact while counts stay below
  // 2^24, where it equals g_int; above, FP32 rounds the count as g_int's conversion does).
  __device__ static __forceinline__ float g_flt(const Model& md, int j, const float (&xf)[NM]) {
    float v = 1.f;
    bool zero = false;
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      const int m = md.ord[j][s];
      if (m != 0) {
        if (xf[s] < (float)m) zero = true;
        else v = v * comb_factor<float>(xf[s], m);
      }
    }
    return zero ? 0.f : v;
  }

  // g_j at a real state (implicit solve), FP64 always.
  __device__ static __forceinline__ double g_real(const Model& md, int j,
                                                  const double (&y)[NM]) {
    double v = 1.0;
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      const int m = md.ord[j][s];
      if (m != 0) v = v * comb_factor<double>(y[s], m);
    }
    return v;
  }

  // exact d g_j / d y_q: the product with species q's factor replaced by its derivative
  template <class T>
  __device__ static __forceinline__ T g_real_deriv(const Model& md, int j, const T (&y)[NM],
                                                   int q) {
    T v = T(1);
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      const int m = md.ord[j][s];
      if (m != 0) v = v * (s == q ? comb_factor_deriv<T>(y[s], m) : comb_factor<T>(y[s], m));
    }
    return v;
  }

  __device__ static __forceinline__ void eval_props(const Model& md, const long long (&x)[NM],
                                                    const R (&th)[MM], R (&g)[MM], R (&a)[MM]) {
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      g[j] = g_int(md, j, x);
      a[j] = th[j] * g[j];
    }
  }

  // Cao 2006 step size over reactions in `use`: per reactant species,
  // mu = sum nu a, var = sum nu^2 a (increasing j, nonzero nu), bound = max(eps x/h, 1),
  // tau_s = min(bound/|mu|, bound^2/var); the minimum over species.
  __device__ static __forceinline__ R tau_select(const Model& md, const R (&a)[MM],
                                                 const long long (&x)[NM], uint32_t use, R eps) {
    R tau = P::inf();
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      if (md.isreact[s]) {
        R mu = R(0), var = R(0);
#pragma unroll
        for (int j = 0; j < MM; ++j) {
          const int v = md.nu[j][s];
          if (((use >> j) & 1u) && v != 0) {
            mu = mu + (R)v * a[j];
            var = var + (R)(v * v) * a[j];
          }
        }
        const R h = hor_factor<R>(md.hor[s], x[s]);
        R bound = (eps * (R)x[s]) / h;
        if (bound < R(1)) bound = R(1);
        const R t1 = bound / fabs(mu);
        const R t2 = (bound * bound) / var;
        const R ts = t1 < t2 ? t1 : t2;
        if (ts < tau) tau = ts;
      }
    }
    return tau;
  }

  // Implicit leap (Rathinam 2003): solve y = c + tau sum_j nu_j a_j(y) over the
  // non-critical reactions by Newton's method: residual, iterate and stopping test in
  // FP64; the Jacobian (forward differences or exact) assembled and factorized by Gaussian
  // elimination with partial pivoting and column-oriented back substitution in the
  // working precision R (FP64 in reference precision; FP32 in fast precision, where an
  // approximate Jacobian changes only the rate of convergence, not the FP64 root).
  // Returns 0 converged, 1 not converged, 2 singular.
  __device__ static __forceinline__ int implicit_solve(const Model& md, const R (&th)[MM],
                                       const long long (&x)[NM], uint32_t nc,
                                       const long long (&Pk)[MM], const R (&a)[MM],
                                       double tau, double tol, int maxit, double fd_h,
                                       bool analytic, double (&y)[NM]) {
    double c[NM];
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      double acc = (double)x[s];
#pragma unroll
      for (int j = 0; j < MM; ++j) {
        const int v = md.nu[j][s];
        if (((nc >> j) & 1u) && v != 0)
          acc = acc + (double)v * ((double)Pk[j] - (double)a[j] * tau);
      }
      c[s] = acc;
      y[s] = (double)x[s];
    }
    const R taur = (R)tau;
    for (int it = 0; it < maxit; ++it) {
      double ay[MM];
#pragma unroll
      for (int j = 0; j < MM; ++j) ay[j] = (double)th[j] * g_real(md, j, y);
      R A[NM][NM], b[NM];
#pragma unroll
      for (int s = 0; s < NM; ++s) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < MM; ++j) {
          const int v = md.nu[j][s];
          if (((nc >> j) & 1u) && v != 0) acc = acc + (double)v * ay[j];
        }
        b[s] = (R)(-((y[s] - c[s]) - tau * acc));
      }
      R yr[NM];
#pragma unroll
      for (int s = 0; s < NM; ++s) yr[s] = (R)y[s];
#pragma unroll
      for (int q = 0; q < NM; ++q) {
        R Dq[MM];
        if (analytic) {
#pragma unroll
          for (int j = 0; j < MM; ++j)
            Dq[j] = (((nc >> j) & 1u) && md.ord[j][q] != 0)
                        ? th[j] * g_real_deriv<R>(md, j, yr, q)
                        : R(0);
        } else {
          const double aq = fabs(y[q]);
          const double h = fd_h * (aq > 1.0 ? aq : 1.0);
          double yq[NM];
#pragma unroll
          for (int s = 0; s < NM; ++s) yq[s] = y[s];
          yq[q] = y[q] + h;
          const double he = yq[q] - y[q];
#pragma unroll
          for (int j = 0; j < MM; ++j)
            Dq[j] = (((nc >> j) & 1u) && md.ord[j][q] != 0)
                        ? (R)(((double)th[j] * g_real(md, j, yq) - ay[j]) / he)
                        : R(0);
        }
#pragma unroll
        for (int s = 0; s < NM; ++s) {
          R acc = R(0);
#pragma unroll
          for (int j = 0; j < MM; ++j) {
            const int v = md.nu[j][s];
            if (((nc >> j) & 1u) && v != 0 && md.ord[j][q] != 0) acc = acc + (R)v * Dq[j];
          }
          A[s][q] = (s == q ? R(1) : R(0)) - taur * acc;
        }
      }
      // elimination with partial pivoting (row swaps by compile-time selects)
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        int piv = k;
        R best = fabs(A[k][k]);
#pragma unroll
        for (int i = k + 1; i < NM; ++i) {
          if (fabs(A[i][k]) > best) {
            best = fabs(A[i][k]);
            piv = i;
          }
        }
        if (best == R(0)) return 2;
#pragma unroll
        for (int i = k + 1; i < NM; ++i) {
          if (i == piv) {
#pragma unroll
            for (int cc = 0; cc < NM; ++cc) {
              const R tmp = A[k][cc];
              A[k][cc] = A[i][cc];
              A[i][cc] = tmp;
            }
            const R tb = b[k];
            b[k] = b[i];
            b[i] = tb;
          }
        }
#pragma unroll
        for (int i = k + 1; i < NM; ++i) {
          const R l = A[i][k] / A[k][k];
#pragma unroll
          for (int cc = k + 1; cc < NM; ++cc) A[i][cc] = A[i][cc] - l * A[k][cc];
          b[i] = b[i] - l * b[k];
        }
      }
      R d[NM];
#pragma unroll
      for (int i = NM - 1; i >= 0; --i) {
        d[i] = b[i] / A[i][i];
#pragma unroll
        for (int rr = 0; rr < i; ++rr) b[rr] = b[rr] - A[rr][i] * d[i];
      }
      double dmax = 0.0, ymax = 0.0;
#pragma unroll
      for (int s = 0; s < NM; ++s) {
        const double ds = (double)d[s];
        y[s] = y[s] + ds;
        if (fabs(ds) > dmax) dmax = fabs(ds);
        if (fabs(y[s]) > ymax) ymax = fabs(y[s]);
      }
      if (dmax <= tol * (ymax > 1.0 ? ymax : 1.0)) return 0;
    }
    return 1;
  }

  // g_j(x + z) - g_j(x) over the reactant species in increasing s, by the recursion
  // D <- f(u) D + (f(u) - f(x)) B, B <- f(x) B with f = C(., m_js), u = x + z.
  __device__ static __forceinline__ R g_diff(const Model& md, int j, const R (&xf)[NM],
                                             const R (&z)[NM]) {
    R D = R(0), B = R(1);
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      const int m = md.ord[j][s];
      if (m != 0) {
        D = comb_factor<R>(xf[s] + z[s], m) * D + comb_diff<R>(xf[s], z[s], m) * B;
        B = comb_factor<R>(xf[s], m) * B;
      }
    }
    return D;
  }

  // Fast precision: the implicit leap for the increment z = y - x, entirely in FP32.  The
  // equation z = c + tau sum_j nu_j theta_j (g_j(x + z) - g_j(x)), c_s = sum_j nu_js P_j
  // (an exact integer sum), has no cancellation between propensities of size a tau: the
  // differences of the binomial factors are polynomials in z.  So FP32 keeps the firing
  // counts K_j = P_j + round(tau theta_j (g_j(x + z) - g_j(x))) within rounding of the
  // FP64 solution (on dimerisation states one leap in about 200 differs by one firing,
  // with no preferred sign).  The stopping test uses max(tol, 1e-6) (FP32 cannot resolve
  // 1e-10).  On success K holds the counts.  The Jacobian is always the exact one (the paper's symbolic Jacobian): in
  // this FP32 solve it only sets the rate of convergence, the exact derivative is the
  // cheaper to evaluate, and leaving out the forward-difference variant keeps the
  // generic 8 x 16 build compact.  Returns 0 converged, 1 not converged, 2 singular.
  __device__ static __forceinline__ int implicit_solve_fast(const Model& md, const R (&th)[MM],
                                            const long long (&x)[NM], uint32_t nc,
                                            long long (&K)[MM], R tau,
                                            double tol, int maxit) {
    R xf[NM], z[NM], c[NM];
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      xf[s] = (R)x[s];
      z[s] = R(0);
      long long cs = 0;
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if ((nc >> j) & 1u) cs += (long long)md.nu[j][s] * K[j];
      c[s] = (R)cs;
    }
    const R tolr = tol > 1e-6 ? (R)tol : R(1e-6);
    for (int it = 0; it < maxit; ++it) {
      R dg[MM];
#pragma unroll
      for (int j = 0; j < MM; ++j) dg[j] = ((nc >> j) & 1u) ? g_diff(md, j, xf, z) : R(0);
      R A[NM][NM], b[NM], yr[NM];
#pragma unroll
      for (int s = 0; s < NM; ++s) {
        R acc = R(0);
#pragma unroll
        for (int j = 0; j < MM; ++j) {
          const int v = md.nu[j][s];
          if (((nc >> j) & 1u) && v != 0) acc = acc + (R)v * (th[j] * dg[j]);
        }
        b[s] = -((z[s] - c[s]) - tau * acc);
        yr[s] = xf[s] + z[s];
      }
#pragma unroll
      for (int q = 0; q < NM; ++q) {
        R Dq[MM];
#pragma unroll
        for (int j = 0; j < MM; ++j)
          Dq[j] = (((nc >> j) & 1u) && md.ord[j][q] != 0)
                      ? th[j] * g_real_deriv<R>(md, j, yr, q)
                      : R(0);
#pragma unroll
        for (int s = 0; s < NM; ++s) {
          R acc = R(0);
#pragma unroll
          for (int j = 0; j < MM; ++j) {
            const int v = md.nu[j][s];
            if (((nc >> j) & 1u) && v != 0 && md.ord[j][q] != 0) acc = acc + (R)v * Dq[j];
          }
          A[s][q] = (s == q ? R(1) : R(0)) - tau * acc;
        }
      }
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        int piv = k;
        R best = fabs(A[k][k]);
#pragma unroll
        for (int i = k + 1; i < NM; ++i) {
          if (fabs(A[i][k]) > best) {
            best = fabs(A[i][k]);
            piv = i;
          }
        }
        if (!(best > R(0))) return 2;
#pragma unroll
        for (int i = k + 1; i < NM; ++i) {
          if (i == piv) {
#pragma unroll
            for (int cc = 0; cc < NM; ++cc) {
              const R tmp = A[k][cc];
              A[k][cc] = A[i][cc];
              A[i][cc] = tmp;
            }
            const R tb = b[k];
            b[k] = b[i];
            b[i] = tb;
          }
        }
#pragma unroll
        for (int i = k + 1; i < NM; ++i) {
          const R l = A[i][k] / A[k][k];
#pragma unroll
          for (int cc = k + 1; cc < NM; ++cc) A[i][cc] = A[i][cc] - l * A[k][cc];
          b[i] = b[i] - l * b[k];
        }
      }
      R d[NM];
#pragma unroll
      for (int i = NM - 1; i >= 0; --i) {
        d[i] = b[i] / A[i][i];
#pragma unroll
        for (int rr = 0; rr < i; ++rr) b[rr] = b[rr] - A[rr][i] * d[i];
      }
      R dmax = R(0), ymax = R(0);
#pragma unroll
      for (int s = 0; s < NM; ++s) {
        z[s] = z[s] + d[s];
        if (fabs(d[s]) > dmax) dmax = fabs(d[s]);
        const R ys = fabs(xf[s] + z[s]);
        if (ys > ymax) ymax = ys;
      }
      if (!(dmax == dmax)) return 1;
      if (dmax <= tolr * (ymax > R(1) ? ymax : R(1))) {
#pragma unroll
        for (int j = 0; j < MM; ++j) {
          if ((nc >> j) & 1u) {
            const R d = tau * (th[j] * g_diff(md, j, xf, z));
            if (!(d < R(kLeapLimit))) {  // beyond the leap limit (or NaN): saturate
              K[j] = kCountLimit;
            } else {
              const long long kj = K[j] + llroundf(d);
              K[j] = kj > 0 ? kj : 0;
            }
          }
        }
        return 0;
      }
    }
    return 1;
  }

  // Inverse-CDF pick of a reaction with probability v_j / sum v, from the second uniform
  // of block w (words 2, 3).  Reference: sequential prefix sums in index order (the
  // canonical order), target u * sum with the lane-tree sum.  Fast: see pick_fast.
  // Rounding that leaves no hit picks the last positive entry.
  __device__ static __forceinline__ int pick_reaction(const R (&v)[MM], const Words4& w) {
    if (!P::kRef) return pick_fast(v, w);
    int pk = -1, last = -1;
    const R target = P::u(w, 1) * lane_tree_sum<MM, R>(v);
    R acc = R(0);
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      if (v[j] > R(0)) last = j;
      acc = acc + v[j];
      if (pk < 0 && target < acc) pk = j;
    }
    return pk < 0 ? last : pk;
  }

  // Fast precision pick with a 48-bit uniform u = (w2>>8) 2^-24 + ((w3>>8) + 1/2) 2^-48.
  // First in FP32: prefix sums P_j and the target (w2>>8) 2^-24 P_{M-1}.  Against exact
  // arithmetic each P_j is off by less than M 2^-24 P_{M-1} and the target by less than
  // (M + 1) 2^-24 P_{M-1}, so when the target is farther than (M + 2) 2^-23 P_{M-1} from
  // every P_j the FP32 search selects the reaction the exact one does.  Otherwise (about
  // 2 M (M + 2) 2^-23 of the picks, ~1e-5) the double-float search decides, which keeps
  // reactions many decades below the total at their exact share.
  __device__ static __forceinline__ int pick_fast(const R (&v)[MM], const Words4& w) {
    float pre[MM];
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      acc = acc + (float)v[j];
      pre[j] = acc;
    }
    const float target = (float)(w.w2 >> 8) * 0x1p-24f * acc;
    const float margin = (float)(MM + 2) * 0x1p-23f * acc;
    int pk = 0;
    bool clear = true;
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      pk += pre[j] <= target ? 1 : 0;
      clear = clear && fabsf(pre[j] - target) > margin;
    }
    if (clear && pk < MM) return pk;
    return pick_df(v, w);
  }

  // The same search over double-float (TwoSum) prefix sums of the FP32 values with the
  // full 48-bit uniform; rarely taken, so kept out of line.
  __device__ static __noinline__ int pick_df(const R (&v)[MM], const Words4& w) {
    int pk = -1, last = -1;
    DF pre[MM];
    DF acc{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      if (v[j] > R(0)) last = j;
      acc = df_add(acc, (float)v[j]);
      pre[j] = acc;
    }
    const DF target = df_uniform_times(acc, w.w2, w.w3);
#pragma unroll
    for (int j = 0; j < MM; ++j)
      if (pk < 0 && df_lt(target, pre[j])) pk = j;
    return pk < 0 ? last : pk;
  }

};


// Inputs and outputs of one implicit leap of the fast kernels, passed to the non-inlined
// solve through local memory so that the leap loop's arrays stay in registers.
template <int NM, int MM>
struct ImplicitIo {
  long long x[NM];
  long long K[MM];  // in: Poisson draws P_j (and the critical firing); out: firing counts
  float th[MM];
};

// Fast precision, FP64 implicit leap (Rathinam 2003): FP64 propensities a_j(x) =
// theta_j g_j(x) from the FP32 rate constants, Newton's method from y = x with the FP64
// residual F(y) = y - c - tau sum_j nu_j a_j(y), Jacobian (forward differences or exact),
// partial pivoting and stopping test max |dy| <= tol max(1, max |y|), then
// K_j = max(0, round((a_j(y) tau + P_j) - a_j(x) tau)) for the non-critical reactions.
// Unlike the reference solve it need not reproduce a fixed operation order, so it divides
// once per species and pivot (reciprocals of the difference steps and pivots) instead of
// once per Jacobian entry and eliminated element: FP64 division is a long instruction
// sequence on this GPU.  Not inlined: its FP64 working set stays out of the register
// allocation of the leap loop.  Returns 0 converged, 1 not converged, 2 singular.
template <int NM, int MM, class MDL>
__device__ __noinline__ int implicit_leap_wide(const MDL& md,
                                               ImplicitIo<NM, MM>& io, uint32_t nc,
                                               double tau, double tol, int maxit, double fd_h,
                                               bool analytic) {
  using TR = ThreadTraj<NM, MM, PrecRef, MDL>;
  double th[MM], ax[MM], y[NM], c[NM];
#pragma unroll
  for (int j = 0; j < MM; ++j) {
    th[j] = (double)io.th[j];
    ax[j] = th[j] * TR::g_int(md, j, io.x);
  }
#pragma unroll
  for (int s = 0; s < NM; ++s) {
    double acc = (double)io.x[s];
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      const int v = md.nu[j][s];
      if (((nc >> j) & 1u) && v != 0) acc += (double)v * ((double)io.K[j] - ax[j] * tau);
    }
    c[s] = acc;
    y[s] = (double)io.x[s];
  }
  int rc = 1;
  for (int it = 0; it < maxit && rc == 1; ++it) {
    double ay[MM];
#pragma unroll
    for (int j = 0; j < MM; ++j) ay[j] = ((nc >> j) & 1u) ? th[j] * TR::g_real(md, j, y) : 0.0;
    double A[NM][NM], b[NM];
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < MM; ++j) {
        const int v = md.nu[j][s];
        if (v != 0) acc += (double)v * ay[j];
      }
      b[s] = -((y[s] - c[s]) - tau * acc);
    }
#pragma unroll
    for (int q = 0; q < NM; ++q) {
      double Dq[MM];
      if (analytic) {
#pragma unroll
        for (int j = 0; j < MM; ++j)
          Dq[j] = (((nc >> j) & 1u) && md.ord[j][q] != 0)
                      ? th[j] * TR::template g_real_deriv<double>(md, j, y, q)
                      : 0.0;
      } else {
        const double aq = fabs(y[q]);
        double yq[NM];
#pragma unroll
        for (int s = 0; s < NM; ++s) yq[s] = y[s];
        yq[q] = y[q] + fd_h * (aq > 1.0 ? aq : 1.0);
        const double inv_h = 1.0 / (yq[q] - y[q]);
#pragma unroll
        for (int j = 0; j < MM; ++j)
          Dq[j] = (((nc >> j) & 1u) && md.ord[j][q] != 0)
                      ? (th[j] * TR::g_real(md, j, yq) - ay[j]) * inv_h
                      : 0.0;
      }
#pragma unroll
      for (int s = 0; s < NM; ++s) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < MM; ++j) {
          const int v = md.nu[j][s];
          if (v != 0 && md.ord[j][q] != 0) acc += (double)v * Dq[j];
        }
        A[s][q] = (s == q ? 1.0 : 0.0) - tau * acc;
      }
    }
    double inv_piv[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      int piv = k;
      double best = fabs(A[k][k]);
#pragma unroll
      for (int i = k + 1; i < NM; ++i) {
        if (fabs(A[i][k]) > best) {
          best = fabs(A[i][k]);
          piv = i;
        }
      }
      if (!(best > 0.0)) {
        rc = 2;
        break;
      }
#pragma unroll
      for (int i = k + 1; i < NM; ++i) {
        if (i == piv) {
#pragma unroll
          for (int cc = 0; cc < NM; ++cc) {
            const double tmp = A[k][cc];
            A[k][cc] = A[i][cc];
            A[i][cc] = tmp;
          }
          const double tb = b[k];
          b[k] = b[i];
          b[i] = tb;
        }
      }
      inv_piv[k] = 1.0 / A[k][k];
#pragma unroll
      for (int i = k + 1; i < NM; ++i) {
        const double l = A[i][k] * inv_piv[k];
#pragma unroll
        for (int cc = k + 1; cc < NM; ++cc) A[i][cc] -= l * A[k][cc];
        b[i] -= l * b[k];
      }
    }
    if (rc == 2) break;
    double dmax = 0.0, ymax = 0.0;
#pragma unroll
    for (int i = NM - 1; i >= 0; --i) {
      const double d = b[i] * inv_piv[i];
#pragma unroll
      for (int rr = 0; rr < i; ++rr) b[rr] -= A[rr][i] * d;
      y[i] += d;
      dmax = fabs(d) > dmax ? fabs(d) : dmax;
    }
#pragma unroll
    for (int s = 0; s < NM; ++s) ymax = fabs(y[s]) > ymax ? fabs(y[s]) : ymax;
    if (!(dmax == dmax)) break;
    if (dmax <= tol * (ymax > 1.0 ? ymax : 1.0)) rc = 0;
  }
  if (rc == 0) {
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      if ((nc >> j) & 1u) {
        const double v = (th[j] * TR::g_real(md, j, y) * tau + (double)io.K[j]) - ax[j] * tau;
        const double rv = round(v);
        io.K[j] = !(rv < 0x1p62) ? kCountLimit : (rv > 0.0 ? (long long)rv : 0);
      }
    }
  }
  return rc;
}

// Fast precision, FP32 implicit leap for the increment z = y - x (ThreadTraj::
// implicit_solve_fast), also not inlined.
template <int NM, int MM, class MDL>
__device__ __noinline__ int implicit_leap_fp32(const MDL& md,
                                               ImplicitIo<NM, MM>& io, uint32_t nc, float tau,
                                               double tol, int maxit) {
  using TF = ThreadTraj<NM, MM, PrecFast, MDL>;
  float th[MM];
  long long x[NM], K[MM];
#pragma unroll
  for (int j = 0; j < MM; ++j) {
    th[j] = io.th[j];
    K[j] = io.K[j];
  }
#pragma unroll
  for (int s = 0; s < NM; ++s) x[s] = io.x[s];
  const int rc = TF::implicit_solve_fast(md, th, x, nc, K, tau, tol, maxit);
#pragma unroll
  for (int j = 0; j < MM; ++j) io.K[j] = K[j];
  return rc;
}

// One trajectory per thread, driven as a per-lane state machine so that a warp does not
// hold lanes in one phase while others run a long phase: a step of the machine is either
// one leap evaluation (propensities, critical set, step sizes, leap or burst decision) or
// a bounded slice of the SSA burst.  The drivers below (round-based, pool, sequential)
// only decide which lane runs which step when; each lane performs exactly the arithmetic
// of the sequential algorithm, so results do not depend on the schedule.  MDL: the model
// tables read at run time (ThreadModel in shared memory) or compiled in (specialized
// kernels).
// kGrid: time-grid output compiled in.  Without it the grid code is absent, so the
// kernels that serve calls without a grid are exactly the plain simulation.
template <int NM, int MM, class P, bool kGrid = false, class MDL = ThreadModel<NM, MM>>
struct ThreadLane {
  using R = typename P::R;
  using TT = ThreadTraj<NM, MM, P, MDL>;
  using Model = MDL;
  enum : int { kIdle = 0, kEval = 1, kSsa = 2, kDone = 3 };

  long long i;
  uint32_t id, status, step;
  int reject_run, mode;
  int kobs;  // next unrecorded grid point
  double t, T;
  R th[MM];
  long long x[NM];
  long long r[MM];
  double G[MM];
  long long cnt[4];
  R g[MM], a[MM];
  // SSA burst
  int b, n_max;
  R a0;

  __device__ __forceinline__ void start(const Model& md, const SimArgs& A, long long idx) {
    i = idx;
    id = (uint32_t)(A.id_base + (unsigned long long)idx);
    status = 0;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      double v = 0.0;
      if (j < A.M) v = A.theta ? A.theta[idx * A.M + j] : md.rates[j];
      if (!(v >= 0.0)) bad = true;
      th[j] = (R)v;
    }
    const int64_t* x0 = A.x0_per ? A.x0 + idx * A.N : A.x0;
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      x[s] = s < A.N ? x0[s] : 0;
      if (x[s] < 0) bad = true;
    }
    T = A.T_per ? A.T[idx] : A.T[0];
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      r[j] = 0;
      G[j] = 0.0;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) cnt[c] = 0;
    t = 0.0;
    step = 0;
    reject_run = 0;
    if (kGrid) kobs = 0;
    if (kGrid && A.K_obs > 0 && !grid_ok(A)) bad = true;
    if (bad) {
      status |= ML_ST_BAD_INPUT;
      t = T;
    }
    if (T != T) t = 0.0;  // NaN horizon: finishes at once
    mode = kEval;
    if (kGrid && A.K_obs > 0) record(A, t, true);  // grid points at t = 0 see x0
  }

  // Time-grid output.  The path is right-continuous and piecewise constant (it changes
  // at SSA firings and at the ends of leaps), so X(t_k) is the state after every change
  // at a time <= t_k.  Writes the current state to each pending point with t_k < tcut
  // (strict) or t_k <= tcut (inclusive).
  __device__ __forceinline__ void record(const SimArgs& A, double tcut, bool inclusive) {
    while (kobs < A.K_obs) {
      const double tk = __ldg(A.t_obs + kobs);
      if (inclusive ? !(tk <= tcut) : !(tk < tcut)) break;
      int64_t* o = A.X_obs + ((long long)i * A.K_obs + kobs) * A.N;
#pragma unroll
      for (int s = 0; s < NM; ++s)
        if (s < A.N) o[s] = x[s];
      ++kobs;
    }
  }

  // A leap ends exactly at the next grid point, as it does at T.
  __device__ __forceinline__ double stop_time(const SimArgs& A) const {
    if (kobs < A.K_obs) {
      const double tk = __ldg(A.t_obs + kobs);
      if (tk < T) return tk;
    }
    return T;
  }

  __device__ static bool grid_ok(const SimArgs& A) {
    double prev = 0.0;
    for (int k = 0; k < A.K_obs; ++k) {
      const double tk = __ldg(A.t_obs + k);
      if (!(tk >= prev) || !(tk <= 1.0e300)) return false;
      prev = tk;
    }
    return true;
  }

  __device__ __forceinline__ void finish(const SimArgs& A, bool staged) {
    // grid points past the end (beyond T, after a step-limit stop, or all of a rejected
    // grid) see the final state
    if (kGrid) {
      for (; kobs < A.K_obs; ++kobs) {
        int64_t* o = A.X_obs + ((long long)i * A.K_obs + kobs) * A.N;
#pragma unroll
        for (int s = 0; s < NM; ++s)
          if (s < A.N) o[s] = x[s];
      }
    }
#pragma unroll
    for (int s = 0; s < NM; ++s)
      if (s < A.N) A.X[i * A.N + s] = x[s];
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      if (j < A.M) {
        A.r[i * A.M + j] = r[j];
        A.G[i * A.M + j] = G[j];
      }
    }
    A.status[i] = status | (staged ? 0u : ML_ST_STAGE_TIMEOUT);
    if (A.counters) {
#pragma unroll
      for (int c = 0; c < 4; ++c) A.counters[i * 4 + c] = cnt[c];
    }
    mode = kIdle;
  }

  // The lane state as 32-bit words of a shared-memory record (pool driver): word k of
  // slot q at rec[k * kPoolSlots + q], the mode first.  g, a and a0 are not kept: a
  // loaded lane recomputes them from x and theta before use.
  static constexpr int kRWords = (int)(sizeof(R) / 4);
  static constexpr int kWords = lane_record_words(NM, MM, kRWords == 2);
  template <int S>
  __device__ __forceinline__ void save(uint32_t* rec, int q) const {
    int k = 0;
    auto put = [&](uint32_t v) { rec[(k++) * S + q] = v; };
    auto put64 = [&](unsigned long long v) {
      put((uint32_t)v);
      put((uint32_t)(v >> 32));
    };
    put((uint32_t)mode);
    put(id);
    put(status);
    put(step);
    put((uint32_t)reject_run);
    put((uint32_t)b);
    put((uint32_t)n_max);
    put64((unsigned long long)i);
    put64((unsigned long long)__double_as_longlong(t));
    put64((unsigned long long)__double_as_longlong(T));
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      if constexpr (kRWords == 2) put64((unsigned long long)__double_as_longlong((double)th[j]));
      else put(__float_as_uint((float)th[j]));
    }
#pragma unroll
    for (int s2 = 0; s2 < NM; ++s2) put64((unsigned long long)x[s2]);
#pragma unroll
    for (int j = 0; j < MM; ++j) put64((unsigned long long)r[j]);
#pragma unroll
    for (int j = 0; j < MM; ++j) put64((unsigned long long)__double_as_longlong(G[j]));
#pragma unroll
    for (int c = 0; c < 4; ++c) put64((unsigned long long)cnt[c]);
  }
  template <int S>
  __device__ __forceinline__ void load(const uint32_t* rec, int q) {
    int k = 0;
    auto get = [&]() { return rec[(k++) * S + q]; };
    auto get64 = [&]() {
      const unsigned long long lo = get();
      return lo | ((unsigned long long)get() << 32);
    };
    mode = (int)get();
    id = get();
    status = get();
    step = get();
    reject_run = (int)get();
    b = (int)get();
    n_max = (int)get();
    i = (long long)get64();
    t = __longlong_as_double((long long)get64());
    T = __longlong_as_double((long long)get64());
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      if constexpr (kRWords == 2) th[j] = (R)__longlong_as_double((long long)get64());
      else th[j] = (R)__uint_as_float(get());
    }
#pragma unroll
    for (int s2 = 0; s2 < NM; ++s2) x[s2] = (long long)get64();
#pragma unroll
    for (int j = 0; j < MM; ++j) r[j] = (long long)get64();
#pragma unroll
    for (int j = 0; j < MM; ++j) G[j] = __longlong_as_double((long long)get64());
#pragma unroll
    for (int c = 0; c < 4; ++c) cnt[c] = (long long)get64();
  }

  __device__ __forceinline__ void begin_burst(int n) {
    mode = kSsa;
    b = 0;
    n_max = n;
  }

  __device__ __forceinline__ void end_burst() {
    step++;
    reject_run = 0;
    mode = kEval;
  }

  // Up to n_slice firings of the SSA burst (Gillespie 1977 direct method) at outer step
  // `step`, firing index b; g, a, a0 are current for b == 0 (or recomputed with fresh).
  // Fast precision accumulates the slice's G increments in FP32 and its elapsed time in
  // compensated FP32 and folds them into the FP64 totals at the end of the slice (every
  // driver runs slices of kSsaPerRound firings, so all fold at the same firings).  The firing counts of the slice are kept in
  // 32-bit registers and added to r once at the end.  The random block of the next
  // firing is generated while the current one is processed: it depends only on the
  // counter, so the two dependency chains overlap.
  __device__ __forceinline__ void ssa_slice(const Model& md, const SimArgs& A, int n_slice,
                                            bool fresh = false) {
    const uint32_t k0 = (uint32_t)A.seed, k1 = (uint32_t)(A.seed >> 32);
    const uint32_t Mr = (uint32_t)A.M;
    const double rem = T - t;
    const float remf = (float)rem;
    float el = 0.f, elc = 0.f;
    float Gs[MM];
    int rc[MM];
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      Gs[j] = 0.f;
      rc[j] = 0;
    }
    // fast precision: an FP32 copy of the state, updated with the FP32 net changes, so
    // that the propensities need no 64-bit conversions; synchronized at every slice start
    float xf[NM];
#pragma unroll
    for (int s = 0; s < NM; ++s) xf[s] = P::kRef ? 0.f : (float)x[s];
    const int b_first = b;
    bool to_horizon = false, burst_over = false;
    Words4 w = philox_block(k0, k1, id, step, Mr + 2u, (uint32_t)b);
    for (int k = 0; k < n_slice; ++k) {
      if (b > 0 || (fresh && k == 0)) {  // the state changed at the previous firing
        if (P::kRef) {
          TT::eval_props(md, x, th, g, a);
        } else {
#pragma unroll
          for (int j = 0; j < MM; ++j) {
            g[j] = (R)TT::g_flt(md, j, xf);
            a[j] = th[j] * g[j];
          }
        }
        a0 = reaction_sum<MM, R, P::kRef>(a);
      }
      if (a0 == R(0)) {
        to_horizon = burst_over = true;
        break;
      }
      const Words4 w_next = philox_block(k0, k1, id, step, Mr + 2u, (uint32_t)b + 1u);
      if (P::kRef) {
        const R dt = -P::log(P::u(w, 0)) / a0;
        const double tn = t + (double)dt;
        if (tn > T) {
          to_horizon = burst_over = true;
          break;
        }
#pragma unroll
        for (int j = 0; j < MM; ++j) G[j] = G[j] + (double)g[j] * (double)dt;
        if (kGrid && A.K_obs > 0) record(A, tn, false);  // points before the firing: old state
        t = tn;
      } else {
        const float dt = __fdividef(-P::log(P::u(w, 0)), a0);  // about 2 ulp
        if ((el - elc) + dt > remf) {
          to_horizon = burst_over = true;
          break;
        }
        // a slice holds at most kSsaPerRound firings: its G sums of that many positive
        // terms are within 8 FP32 roundings; the elapsed time is summed compensated
#pragma unroll
        for (int j = 0; j < MM; ++j) Gs[j] = fmaf((float)g[j], dt, Gs[j]);
        kahan_add(el, elc, dt);
        if (kGrid && A.K_obs > 0) record(A, t + ((double)el - (double)elc), false);
      }
      const int pick = TT::pick_reaction(a, w);
      if constexpr (Model::kCompiled) {
        // compile-time net changes: one predicated update per nonzero entry
#pragma unroll
        for (int j = 0; j < MM; ++j) {
#pragma unroll
          for (int s = 0; s < NM; ++s) {
            if (md.nu[j][s] != 0 && j == pick) {
              x[s] += md.nu[j][s];
              if (!P::kRef) xf[s] += md.nuf[j][s];
            }
          }
        }
      } else {
#pragma unroll
        for (int s = 0; s < NM; ++s) {
          x[s] += md.nu[pick][s];
          if (!P::kRef) xf[s] += md.nuf[pick][s];
        }
      }
#pragma unroll
      for (int j = 0; j < MM; ++j) rc[j] += (j == pick) ? 1 : 0;
      if (kGrid && A.K_obs > 0)  // a point at the firing time: new state
        record(A, P::kRef ? t : t + ((double)el - (double)elc), true);
      w = w_next;
      if (++b >= n_max) {
        burst_over = true;
        break;
      }
    }
#pragma unroll
    for (int j = 0; j < MM; ++j) r[j] += rc[j];
    cnt[2] += b - b_first;
    if (P::kRef) {
      if (to_horizon) {
        const double rm = T - t;
#pragma unroll
        for (int j = 0; j < MM; ++j) G[j] = G[j] + (double)g[j] * rm;
        t = T;
      }
    } else {
      const double elapsed = (double)el - (double)elc;
      // one FP64 addition per reaction and slice
#pragma unroll
      for (int j = 0; j < MM; ++j) G[j] = G[j] + (double)Gs[j];
      if (to_horizon) {
        const double left = rem - elapsed > 0.0 ? rem - elapsed : 0.0;
#pragma unroll
        for (int j = 0; j < MM; ++j) G[j] = G[j] + (double)g[j] * left;
        t = T;
      } else {
        t = t + elapsed;
      }
    }
    if (burst_over) end_burst();
  }

  // One outer step: either a committed leap (stays in kEval), the start of an SSA burst,
  // or the end of the trajectory.
  __device__ __forceinline__ void eval_phase(const Model& md, const SimArgs& A) {
    const uint32_t k0 = (uint32_t)A.seed, k1 = (uint32_t)(A.seed >> 32);
    const uint32_t Mr = (uint32_t)A.M;  // stream numbering uses the real M
    if (!(t < T)) {
      mode = kDone;
      return;
    }
    if ((long long)step >= A.max_steps) {
      status |= ML_ST_STEP_LIMIT;
      mode = kDone;
      return;
    }
    {
      bool big = false;
#pragma unroll
      for (int s = 0; s < NM; ++s) big = big || x[s] > kCountLimit;
#pragma unroll
      for (int j = 0; j < MM; ++j) big = big || r[j] > kCountLimit;
      if (big) {
        status |= ML_ST_OVERFLOW;
        mode = kDone;
        return;
      }
    }
    TT::eval_props(md, x, th, g, a);
    a0 = reaction_sum<MM, R, P::kRef>(a);
    if (a0 == R(0)) {
      const double rm = T - t;
#pragma unroll
      for (int j = 0; j < MM; ++j) G[j] = G[j] + (double)g[j] * rm;
      t = T;
      mode = kDone;
      return;
    }
    int burst = 0;
    const R eps = (R)A.eps;
    if (A.mode == ML_MODE_SSA_ONLY) {
      burst = A.n_ssa_ex;
    } else {
      // critical reactions: a_j > 0 and min over consumed species of floor(x_s/|nu_js|)
      // below n_c, i.e. some consumed species has x_s < n_c |nu_js| (no division needed)
      uint32_t nc = 0;
      R ac[MM];
#pragma unroll
      for (int j = 0; j < MM; ++j) {
        bool crit = false;
        if (a[j] > R(0)) {
#pragma unroll
          for (int s = 0; s < NM; ++s) {
            const int v = md.nu[j][s];
            if (v < 0 && x[s] < (long long)A.n_c * (long long)(-v)) crit = true;
          }
        }
        if (!crit) nc |= 1u << j;
        ac[j] = crit ? a[j] : R(0);
      }
      const R a0c = reaction_sum<MM, R, P::kRef>(ac);
      const R tau_ex = TT::tau_select(md, a, x, nc, eps);
      // partial equilibrium and the implicit step size
      bool implicit = false;
      R tau1 = tau_ex;
      if (A.mode == ML_MODE_ADAPTIVE && md.n_pairs > 0) {
        uint32_t pe = 0;
#pragma unroll
        for (int j = 0; j < MM; ++j) {
          const int k = md.partner[j];
          if (k >= 0 && ((nc >> j) & 1u) && ((nc >> k) & 1u)) {
            R ak = R(0);
#pragma unroll
            for (int kk = 0; kk < MM; ++kk)
              if (kk == k) ak = a[kk];
            const R lo = a[j] < ak ? a[j] : ak;
            if (fabs(a[j] - ak) <= (R)A.pe_delta * lo) pe |= (1u << j) | (1u << k);
          }
        }
        if (pe != 0) {
          const R tau_im = TT::tau_select(md, a, x, nc & ~pe, eps);
          if (tau_im > (R)A.stiff_ratio * tau_ex) {
            implicit = true;
            tau1 = tau_im;
          }
        }
      }
      // attempt loop: tau2, SSA switch, leap, negativity check
      for (;;) {
        if (reject_run >= A.max_reject) {
          status |= ML_ST_REJECT_LIMIT;
          burst = A.n_ssa_ex;
          break;
        }
        R tau2 = P::inf();
        if (a0c > R(0)) {
          const Words4 w = philox_block(k0, k1, id, step, Mr, 0u);
          tau2 = -P::log(P::u(w, 0)) / a0c;
        }
        const R tmin = tau1 < tau2 ? tau1 : tau2;
        if (tmin < (R)A.ssa_factor / a0) {
          burst = implicit ? A.n_ssa_im : A.n_ssa_ex;
          break;
        }
        const double stop = kGrid ? stop_time(A) : T;
        const double rm = stop - t;
        R tau = tau1;
        if (tau2 < tau) tau = tau2;
        bool at_horizon = false;
        if ((R)rm <= tau) {
          tau = (R)rm;
          at_horizon = true;
        }
        const bool crit_fire = (tau2 <= tau1) && (tau2 <= (R)rm);
        {
          bool over = false;
#pragma unroll
          for (int j = 0; j < MM; ++j)
            over = over || (((nc >> j) & 1u) && a[j] * tau > (R)kLeapLimit);
          if (over) {
            status |= ML_ST_OVERFLOW;
            mode = kDone;
            return;
          }
        }
        long long K[MM];
#pragma unroll
        for (int j = 0; j < MM; ++j) K[j] = 0;
        if (crit_fire) {
          const Words4 w = philox_block(k0, k1, id, step, Mr + 1u, 0u);
          const int pick = TT::pick_reaction(ac, Words4{0u, 0u, w.w0, w.w1});
#pragma unroll
          for (int j = 0; j < MM; ++j) K[j] = (j == pick) ? 1 : 0;
        }
        const bool implicit_step = implicit && tau > tau_ex;
        // Poisson firings of the non-critical reactions (explicit counts, or the noise
        // term P_j of the implicit equation)
#pragma unroll
        for (int j = 0; j < MM; ++j)
          if ((nc >> j) & 1u)
            K[j] = poisson_draw<P>(a[j] * tau, k0, k1, id, step, (uint32_t)j, status);
        if (implicit_step) {
          int rc;
          if constexpr (P::kRef) {
            double y[NM];
            const double taud = (double)tau;
            rc = TT::implicit_solve(md, th, x, nc, K, a, taud, A.newton_tol, A.newton_maxit,
                                    A.fd_h, A.jacobian == ML_JAC_ANALYTIC, y);
            if (rc == 0) {
#pragma unroll
              for (int j = 0; j < MM; ++j) {
                if ((nc >> j) & 1u) {
                  const double ayj = (double)th[j] * TT::g_real(md, j, y);
                  const double v = (ayj * taud + (double)K[j]) - (double)a[j] * taud;
                  const double rv = round(v);
                  K[j] = !(rv < 0x1p62) ? kCountLimit : (rv > 0.0 ? (long long)rv : 0);
                }
              }
            }
          } else {
            ImplicitIo<NM, MM> io;
#pragma unroll
            for (int s = 0; s < NM; ++s) io.x[s] = x[s];
#pragma unroll
            for (int j = 0; j < MM; ++j) {
              io.K[j] = K[j];
              io.th[j] = (float)th[j];
            }
            rc = A.newton_fp32
                     ? implicit_leap_fp32<NM, MM>(md, io, nc, (float)tau, A.newton_tol,
                                                  A.newton_maxit)
                     : implicit_leap_wide<NM, MM>(md, io, nc, (double)tau, A.newton_tol,
                                                  A.newton_maxit, A.fd_h,
                                                  A.jacobian == ML_JAC_ANALYTIC);
#pragma unroll
            for (int j = 0; j < MM; ++j) K[j] = io.K[j];
          }
          if (rc != 0) {
            status |= ML_ST_NEWTON_FAIL;
            implicit = false;
            tau1 = tau_ex;
            step++;
            continue;
          }
        }
        if (implicit_step) {
          bool over = false;
#pragma unroll
          for (int j = 0; j < MM; ++j) over = over || (((nc >> j) & 1u) && K[j] > kLeapLimitInt);
          if (over) {
            status |= ML_ST_OVERFLOW;
            mode = kDone;
            return;
          }
        }
        long long xn[NM];
        bool negative = false;
#pragma unroll
        for (int s = 0; s < NM; ++s) {
          long long v = x[s];
#pragma unroll
          for (int j = 0; j < MM; ++j) v += (long long)md.nu[j][s] * K[j];
          xn[s] = v;
          if (v < 0) negative = true;
        }
        if (negative) {
          tau1 = tau1 * R(0.5);
          step++;
          reject_run++;
          cnt[3] += 1;
          continue;
        }
        const double half = (double)tau * 0.5;
        const R half_r = tau * R(0.5);
#pragma unroll
        for (int j = 0; j < MM; ++j) {
          const R gn = TT::g_int(md, j, xn);
          r[j] += K[j];
          if (P::kRef) G[j] = G[j] + half * ((double)g[j] + (double)gn);
          else G[j] = G[j] + (double)(half_r * (g[j] + gn));  // FP32 increment
        }
#pragma unroll
        for (int s = 0; s < NM; ++s) x[s] = xn[s];
        t = at_horizon ? stop : t + (double)tau;
        if (kGrid && A.K_obs > 0) record(A, t, true);
        cnt[implicit_step ? 1 : 0] += 1;
        step++;
        reject_run = 0;
        break;
      }
    }
    if (burst > 0) begin_burst(burst);
  }
};

#ifndef ML_THREAD_MIN_BLOCKS
#define ML_THREAD_MIN_BLOCKS 1
#endif
#if ML_THREAD_MIN_BLOCKS == 2
// the occupancy build: at most 128 threads per CTA, about 168 registers, 3 CTAs per SM
#define ML_THREAD_BOUNDS __launch_bounds__(128, 3)
#else
#define ML_THREAD_BOUNDS __launch_bounds__(256, 1)
#endif

// Warp schedule: in every round a lane that needs a leap evaluation performs one, and a
// lane inside an SSA burst performs up to kSsaPerRound firings (about the cost of one
// evaluation), so lanes in different phases progress together instead of a whole burst
// holding the warp.  (Running only one phase per round, the evaluations once at least 4
// or 8 lanes need one, measured 2.6 and 1.8 times slower on the gene-expression batch.)
constexpr int kSsaPerRound = 8;

// Round-based driver: plain form (queue null): thread i runs trajectory i.  Persistent
// form: lanes claim trajectory indices from the device queue (in the caller's order, if
// any) and refill as soon as their trajectory ends.
template <int NM, int MM, class P, class MDL>
__device__ __forceinline__ void run_rounds(const MDL& md, bool staged, const SimArgs& args) {
  using Lane = ThreadLane<NM, MM, P, false, MDL>;
  Lane L;
  L.mode = Lane::kIdle;
  const long long first = args.queue ? queue_claim(args.queue, args.order, args.n_traj)
                                     : (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (first < args.n_traj) L.start(md, args, first);
  for (;;) {
    if (L.mode == Lane::kDone) {
      L.finish(args, staged);
      if (args.queue) {
        const long long nxt = queue_claim(args.queue, args.order, args.n_traj);
        if (nxt < args.n_traj) L.start(md, args, nxt);
      }
    }
    if (!__any_sync(0xffffffffu, L.mode != Lane::kIdle)) break;
    if (L.mode == Lane::kEval) {
      L.eval_phase(md, args);
    } else if (L.mode == Lane::kSsa) {
      L.ssa_slice(md, args, kSsaPerRound);
    }
  }
}

// Pool driver: every warp keeps kPoolSlots trajectories (two per lane) in shared memory
// and in each round runs one phase for 32 of them: SSA slices while at least 32 (or more
// than the evaluations waiting) are inside a burst, else leap evaluations.  A lane loads
// the chosen trajectory's state, runs the phase and stores it back, so the lanes of a
// warp execute the same phase instead of taking turns between the evaluation and the SSA
// code (the round-based driver's lanes diverge there).  A finished trajectory is written
// out and its slot refilled from the work queue at once.  Persistent form only.

// Position of the (n+1)-th set bit of m (n < popcount(m)).
__device__ __forceinline__ int nth_set_bit(unsigned long long m, int n) {
  const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
  const int clo = __popc(lo);
  uint32_t v = n < clo ? lo : hi;
  int k = n < clo ? n : n - clo;
  for (; k > 0; --k) v &= v - 1u;
  return (n < clo ? 0 : 32) + __ffs((int)v) - 1;
}

template <int NM, int MM, class P, class MDL>
__device__ __forceinline__ void run_pool(const MDL& md, bool staged, const SimArgs& args,
                                         uint32_t* pool_words) {
  using Lane = ThreadLane<NM, MM, P, false, MDL>;
  const int lane = threadIdx.x & 31;
  uint32_t* rec = pool_words + (size_t)(threadIdx.x >> 5) * Lane::kWords * kPoolSlots;
#pragma unroll 1
  for (int h = lane; h < kPoolSlots; h += 32) {
    Lane L;
    L.mode = Lane::kIdle;
    const long long idx = queue_claim(args.queue, args.order, args.n_traj);
    if (idx < args.n_traj) L.start(md, args, idx);
    L.template save<kPoolSlots>(rec, h);
  }
  __syncwarp();
  // the search for ready slots starts at a rotating position, so that no slot waits
  // while others are served round after round
  int rot = 0;
  for (;;) {
    const uint32_t m_lo = rec[lane], m_hi = rec[32 + lane];  // mode words
    const unsigned long long ms =
        (unsigned long long)__ballot_sync(0xffffffffu, m_lo == (uint32_t)Lane::kSsa) |
        ((unsigned long long)__ballot_sync(0xffffffffu, m_hi == (uint32_t)Lane::kSsa) << 32);
    const unsigned long long me =
        (unsigned long long)__ballot_sync(0xffffffffu, m_lo == (uint32_t)Lane::kEval) |
        ((unsigned long long)__ballot_sync(0xffffffffu, m_hi == (uint32_t)Lane::kEval) << 32);
    const int ns = __popcll(ms), ne = __popcll(me);
    if (ns + ne == 0) break;
    const bool ssa = ns >= 32 || (ne < 32 && ns >= ne);
    const int n_run = ssa ? ns : ne;
    const unsigned long long m = ssa ? ms : me;
    const int r0 = rot;
    rot = (rot + 29) & (kPoolSlots - 1);
    const unsigned long long mr = r0 ? (m >> r0) | (m << (kPoolSlots - r0)) : m;
    if (lane < n_run) {
      const int q = (nth_set_bit(mr, lane) + r0) & (kPoolSlots - 1);
      Lane L;
      L.template load<kPoolSlots>(rec, q);
      if (ssa) L.ssa_slice(md, args, kSsaPerRound, true);
      else L.eval_phase(md, args);
      if (L.mode == Lane::kDone) {
        L.finish(args, staged);
        const long long nxt = queue_claim(args.queue, args.order, args.n_traj);
        if (nxt < args.n_traj) L.start(md, args, nxt);
      }
      L.template save<kPoolSlots>(rec, q);
    }
    __syncwarp();
  }
}

// Sequential per-lane driver over the same lane state machine: each thread runs its
// trajectory to the end before claiming the next one.  It has less scheduling overhead
// and suits leap-dominated workloads; the autotuner picks between the drivers.  Its kGrid
// build serves every thread-shape call with time-grid output (the drivers give identical
// results).
template <int NM, int MM, class P, bool kGrid, class MDL>
__device__ __forceinline__ void run_sequential(const MDL& md, bool staged, const SimArgs& args) {
  using Lane = ThreadLane<NM, MM, P, kGrid, MDL>;
  Lane L;
  long long i = args.queue ? queue_claim(args.queue, args.order, args.n_traj)
                           : (long long)blockIdx.x * blockDim.x + threadIdx.x;
  while (i < args.n_traj) {
    L.start(md, args, i);
    while (L.mode != Lane::kDone) {
      if (L.mode == Lane::kEval) L.eval_phase(md, args);
      else L.ssa_slice(md, args, kSsaPerRound);
    }
    L.finish(args, staged);
    if (!args.queue) break;
    i = queue_claim(args.queue, args.order, args.n_traj);
  }
}

// Kernels over the run-time tables: stage the model once per CTA into shared memory (one
// bulk copy), then run a driver.
template <int NM, int MM, class P>
__global__ void ML_THREAD_BOUNDS k_thread(const ThreadModel<NM, MM>* __restrict__ gmd,
                                          const SimArgs args) {
  __shared__ ThreadModel<NM, MM> smd;
  __shared__ uint64_t mbar;
  const bool staged = stage_model_bulk(&smd, gmd, (uint32_t)thread_model_bytes<NM, MM>(), &mbar,
                                       args.stage_polls);
  run_rounds<NM, MM, P>(smd, staged, args);
}

template <int NM, int MM, class P>
__global__ void ML_THREAD_BOUNDS k_thread_pool(const ThreadModel<NM, MM>* __restrict__ gmd,
                                               const SimArgs args) {
  __shared__ ThreadModel<NM, MM> smd;
  __shared__ uint64_t mbar;
  extern __shared__ uint32_t pool_words[];
  const bool staged = stage_model_bulk(&smd, gmd, (uint32_t)thread_model_bytes<NM, MM>(), &mbar,
                                       args.stage_polls);
  run_pool<NM, MM, P>(smd, staged, args, pool_words);
}

template <int NM, int MM, class P, bool kGrid = false>
__global__ void ML_THREAD_BOUNDS k_thread_seq(const ThreadModel<NM, MM>* __restrict__ gmd,
                                              const SimArgs args) {
  __shared__ ThreadModel<NM, MM> smd;
  __shared__ uint64_t mbar;
  const bool staged = stage_model_bulk(&smd, gmd, (uint32_t)thread_model_bytes<NM, MM>(), &mbar,
                                       args.stage_polls);
  run_sequential<NM, MM, P, kGrid>(smd, staged, args);
}

}  // namespace mlk
