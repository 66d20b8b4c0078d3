// One trajectory per warp: the same adaptive tau-leaping step for networks too large for
// one thread (up to 64 species and 128 reactions).  Lane l owns reactions l, l+32, l+64,
// l+96 (propensities, Poisson draws, r and G in registers) and species l, l+32 (the
// mean/variance sums of the step-size bound, the state update and one row of the
// implicit Jacobian).  The state x, the propensities a, the firings K and the Newton
// system live in a per-warp slab of shared memory.
//
// Reference precision keeps the canonical operation order of the CPU reference: a0 and
// a0c by the lane tree (lane l sums reactions l, l+32, ... in order, then xor distances
// 16..1), per-species sums sequential in reaction index, sequential prefix sums for the
// SSA and critical picks, and the Newton system assembled, eliminated and back-
// substituted element by element in the same order.  Fast precision uses any order.
#pragma once
#include <cstdint>

#include "thread_core.cuh"

namespace mlk {

constexpr int kRPL = kWarpMaxM / 32;  // reactions per lane
constexpr int kSPL = kWarpMaxN / 32;  // species per lane

// Per-warp shared-memory slab; offsets depend on the model size, on the working precision
// R (rbytes = sizeof(R): propensities) and on the arithmetic of the Newton system
// (lbytes: the matrix, right-hand side and derivatives; FP64 unless fast precision asks
// for an FP32 factorization); the iterate and its propensities are FP64.
struct WarpSlab {
  long long* x;   // [N] state
  long long* xn;  // [N] proposed state
  long long* K;   // [M] firings of the current leap (Poisson draws before the solve)
  double* y;      // [N] Newton iterate
  double* ay;     // [M] propensities at y
  void* b;        // [N] right-hand side / update (Newton type)
  void* D;        // [M][3] Jacobian entries by reactant slot (Newton type)
  void* J;        // [N][N] Newton matrix (Newton type)
  void* a;        // [M] propensities (R)
  void* ac;       // [M] critical propensities (R)
};

__host__ __device__ inline size_t warp_slab_bytes(int N, int M, int rbytes, int lbytes) {
  size_t b = 0;
  b += 8 * (size_t)N * 2;                      // x, xn
  b += 8 * (size_t)M;                          // K
  b += 8 * (size_t)N;                          // y
  b += 8 * (size_t)M;                          // ay
  b += (size_t)lbytes * N;                     // b
  b += (size_t)lbytes * 3 * M;                 // D
  b += (size_t)lbytes * (size_t)N * (size_t)N; // J
  b += (size_t)rbytes * M * 2;                 // a, ac
  return (b + 15) / 16 * 16;
}

__device__ inline WarpSlab carve_slab(char* p, int N, int M, int rbytes, int lbytes) {
  WarpSlab s;
  s.x = reinterpret_cast<long long*>(p);
  p += 8 * N;
  s.xn = reinterpret_cast<long long*>(p);
  p += 8 * N;
  s.K = reinterpret_cast<long long*>(p);
  p += 8 * M;
  s.y = reinterpret_cast<double*>(p);
  p += 8 * N;
  s.ay = reinterpret_cast<double*>(p);
  p += 8 * M;
  s.b = p;
  p += (size_t)lbytes * N;
  s.D = p;
  p += (size_t)lbytes * 3 * M;
  s.J = p;
  p += (size_t)lbytes * (size_t)N * N;
  s.a = p;
  p += (size_t)rbytes * M;
  s.ac = p;
  return s;
}

template <class P>
struct WarpTraj {
  using R = typename P::R;

  // Canonical lane-tree sum of one value per owned reaction.
  __device__ static __forceinline__ R tree_sum(const R (&v)[kRPL], int lane, int M) {
    R s = R(0);
#pragma unroll
    for (int q = 0; q < kRPL; ++q) {
      const int j = lane + 32 * q;
      if (j < M) s = (q == 0) ? v[q] : s + v[q];
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) s = s + __shfl_xor_sync(0xffffffffu, s, d);
    return s;
  }

  __device__ static __forceinline__ R g_int(const WarpModel& md, int j, const long long* x) {
    R v = R(1);
    bool zero = false;
    const int nr = md.nreact[j];
    for (int k = 0; k < nr; ++k) {
      const int s = md.rsp[j][k], m = md.rmul[j][k];
      const long long xs = x[s];
      if (xs < m) zero = true;
      else v = v * comb_factor<R>((R)xs, m);
    }
    return zero ? R(0) : v;
  }

  // Fast precision: g_j from the FP32 copy of the state kept during SSA bursts.
  __device__ static __forceinline__ float g_flt(const WarpModel& md, int j, const float* xf) {
    float v = 1.f;
    bool zero = false;
    const int nr = md.nreact[j];
    for (int k = 0; k < nr; ++k) {
      const int s = md.rsp[j][k], m = md.rmul[j][k];
      const float xs = xf[s];
      if (xs < (float)m) zero = true;
      else v = v * comb_factor<float>(xs, m);
    }
    return zero ? 0.f : v;
  }

  // g_j on a real state; if `sub` >= 0 species `sub` takes the value `ysub`.
  __device__ static __forceinline__ double g_real(const WarpModel& md, int j, const double* y,
                                                  int sub, double ysub) {
    double v = 1.0;
    const int nr = md.nreact[j];
    for (int k = 0; k < nr; ++k) {
      const int s = md.rsp[j][k];
      v = v * comb_factor<double>(s == sub ? ysub : y[s], md.rmul[j][k]);
    }
    return v;
  }

  __device__ static __forceinline__ bool bit(const uint32_t (&m)[kRPL], int j) {
    return (m[j >> 5] >> (j & 31)) & 1u;
  }

  // Cao 2006 step size over reactions in `use` (all lanes return the same value).
  __device__ static R tau_select(const WarpModel& md, const R* a, const long long* x,
                                 const uint32_t (&use)[kRPL], R eps, int lane) {
    R tau = P::inf();
#pragma unroll
    for (int q = 0; q < kSPL; ++q) {
      const int s = lane + 32 * q;
      if (s < md.N && md.isreact[s]) {
        R mu = R(0), var = R(0);
        for (int e = md.sp_ptr[s]; e < md.sp_ptr[s + 1]; ++e) {
          const int j = md.sp_j[e];
          if (bit(use, j)) {
            const int v = md.sp_nu[e];
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
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      const R o = __shfl_xor_sync(0xffffffffu, tau, d);
      tau = o < tau ? o : tau;
    }
    return tau;
  }

  // Inverse-CDF pick of a reaction with probability v_j / sum v (v in shared memory,
  // owned values in vl) from the second uniform of block w.  Reference: sequential prefix
  // in index order with target u * (lane-tree sum), the canonical order.  Fast: double-
  // float prefix sums of the FP32 values over lane-major order with a 48-bit uniform, so
  // reactions many decades below the total keep their exact share without FP64 work.
  // Rounding that leaves no hit picks the last positive entry.  All lanes return the
  // same index.
  __device__ static int pick(const R* v, const R (&vl)[kRPL], const Words4& w, int M,
                             int lane) {
    if (P::kRef) {
      const R target = P::u(w, 1) * tree_sum(vl, lane, M);
      R acc = R(0);
      int pk = -1, last = -1;
      for (int j = 0; j < M; ++j) {
        const R vj = v[j];
        if (vj > R(0)) last = j;
        acc = acc + vj;
        if (target < acc) {
          pk = j;
          break;
        }
      }
      return pk < 0 ? last : pk;
    } else {
      DF S{0.f, 0.f};
#pragma unroll
      for (int q = 0; q < kRPL; ++q)
        if (lane + 32 * q < M) S = df_add(S, (float)vl[q]);
      DF E = S;  // inclusive scan over lanes
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const DF o{__shfl_up_sync(0xffffffffu, E.hi, d), __shfl_up_sync(0xffffffffu, E.lo, d)};
        if (lane >= d) E = df_add(E, o);
      }
      const DF tot{__shfl_sync(0xffffffffu, E.hi, 31), __shfl_sync(0xffffffffu, E.lo, 31)};
      const DF target = df_uniform_times(tot, w.w2, w.w3);
      DF Ex{__shfl_up_sync(0xffffffffu, E.hi, 1), __shfl_up_sync(0xffffffffu, E.lo, 1)};
      if (lane == 0) Ex = DF{0.f, 0.f};
      const unsigned hit = __ballot_sync(0xffffffffu, df_lt(target, E) && S.hi > 0.f);
      int src;
      if (hit) src = __ffs(hit) - 1;
      else {
        const unsigned pos = __ballot_sync(0xffffffffu, S.hi > 0.f);
        src = pos ? 31 - __clz(pos) : 0;
      }
      int pk = -1, last = -1;
      if (lane == src) {
        DF acc = Ex;
#pragma unroll
        for (int q = 0; q < kRPL; ++q) {
          const int j = lane + 32 * q;
          if (j < M && vl[q] > R(0)) {
            last = j;
            acc = df_add(acc, (float)vl[q]);
            if (pk < 0 && df_lt(target, acc)) pk = j;
          }
        }
        if (pk < 0) pk = last;
      }
      return __shfl_sync(0xffffffffu, pk, src);
    }
  }

  // Fast precision: one FP32 inclusive scan of the lanes' sums of their (at most kRPL)
  // values gives the total (a0) and the pick together.  The target (w2>>8) 2^-24 a0 and
  // every prefix carry less than (M + 2) 2^-23 a0 of rounding against exact arithmetic,
  // so when the target is farther than that from every prefix at the chosen lane the
  // FP32 pick is the exact one; otherwise the double-float pick decides.  All lanes
  // return the same total and index.
  // Returns the total; S = the lane's own sum, E = the inclusive prefix at the lane.
  __device__ static float scan_total(const R (&vl)[kRPL], int M, int lane, float& S,
                                     float& E) {
    S = 0.f;
#pragma unroll
    for (int q = 0; q < kRPL; ++q)
      if (lane + 32 * q < M) S = S + (float)vl[q];
    E = S;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const float o = __shfl_up_sync(0xffffffffu, E, d);
      if (lane >= d) E = E + o;
    }
    return __shfl_sync(0xffffffffu, E, 31);
  }
  __device__ static int pick_scanned(const R* v, const R (&vl)[kRPL], const Words4& w,
                                     int M, int lane, float S, float E, float tot) {
    const float target = (float)(w.w2 >> 8) * 0x1p-24f * tot;
    const float margin = (float)(M + 2) * 0x1p-23f * tot;
    const unsigned hit = __ballot_sync(0xffffffffu, target < E && S > 0.f);
    const int src = hit ? __ffs(hit) - 1 : 31;
    const float Ex = __shfl_up_sync(0xffffffffu, E, 1);
    int pk = -1;
    bool clear = hit != 0;
    if (lane == src) {
      float acc = lane == 0 ? 0.f : Ex;
      clear = clear && fabsf(target - acc) > margin;
#pragma unroll
      for (int q = 0; q < kRPL; ++q) {
        const int j = lane + 32 * q;
        if (j < M) {
          acc = acc + (float)vl[q];
          clear = clear && fabsf(target - acc) > margin;
          if (pk < 0 && target < acc && vl[q] > R(0)) pk = j;
        }
      }
      clear = clear && pk >= 0;
    }
    pk = __shfl_sync(0xffffffffu, pk, src);
    if (__shfl_sync(0xffffffffu, (int)clear, src)) return pk;
    return pick(v, vl, w, M, lane);
  }

  // Implicit solve on the per-warp slab: residual, iterate and stopping test in FP64;
  // Jacobian, elimination and back substitution in L (FP64, or FP32 when fast precision
  // asks for an FP32 factorization).  Returns 0 converged, 1 not converged, 2 singular.
  template <class L>
  __device__ static int implicit_solve(const WarpModel& md, const WarpSlab& sl,
                                       const R (&th)[kRPL], const uint32_t (&nc)[kRPL],
                                       const R* a, double tau, double tol, int maxit,
                                       double fd_h, bool analytic, int lane) {
    const int N = md.N, M = md.M;
    L* const Jm = static_cast<L*>(sl.J);
    L* const bv = static_cast<L*>(sl.b);
    L* const Dm = static_cast<L*>(sl.D);
    const L taur = (L)tau;
    double c[kSPL];
#pragma unroll
    for (int q = 0; q < kSPL; ++q) {
      const int s = lane + 32 * q;
      c[q] = 0.0;
      if (s < N) {
        double acc = (double)sl.x[s];
        for (int e = md.sp_ptr[s]; e < md.sp_ptr[s + 1]; ++e) {
          const int j = md.sp_j[e];
          if (bit(nc, j))
            acc = acc + (double)md.sp_nu[e] * ((double)sl.K[j] - (double)a[j] * tau);
        }
        c[q] = acc;
        sl.y[s] = (double)sl.x[s];
      }
    }
    __syncwarp();
    for (int it = 0; it < maxit; ++it) {
#pragma unroll
      for (int q = 0; q < kRPL; ++q) {
        const int j = lane + 32 * q;
        if (j < M) sl.ay[j] = (double)th[q] * g_real(md, j, sl.y, -1, 0.0);
      }
      __syncwarp();
      // right-hand side and Jacobian entries
#pragma unroll
      for (int q = 0; q < kSPL; ++q) {
        const int s = lane + 32 * q;
        if (s < N) {
          double acc = 0.0;
          for (int e = md.sp_ptr[s]; e < md.sp_ptr[s + 1]; ++e) {
            const int j = md.sp_j[e];
            if (bit(nc, j)) acc = acc + (double)md.sp_nu[e] * sl.ay[j];
          }
          bv[s] = (L)(-((sl.y[s] - c[q]) - tau * acc));
        }
      }
#pragma unroll
      for (int q = 0; q < kRPL; ++q) {
        const int j = lane + 32 * q;
        if (j < M) {
          const int nr = md.nreact[j];
          for (int k = 0; k < 3; ++k) {
            L dv = L(0);
            if (k < nr && bit(nc, j)) {
              if (analytic) {
                L v = L(1);
                for (int kk = 0; kk < nr; ++kk) {
                  const L ys = (L)sl.y[md.rsp[j][kk]];
                  const int m = md.rmul[j][kk];
                  v = v * (kk == k ? comb_factor_deriv<L>(ys, m) : comb_factor<L>(ys, m));
                }
                dv = (L)th[q] * v;
              } else {
                const int sq = md.rsp[j][k];
                const double yq = sl.y[sq];
                const double aq = fabs(yq);
                const double h = fd_h * (aq > 1.0 ? aq : 1.0);
                const double yp = yq + h;
                const double he = yp - yq;
                dv = (L)(((double)th[q] * g_real(md, j, sl.y, sq, yp) - sl.ay[j]) / he);
              }
            }
            Dm[j * 3 + k] = dv;
          }
        }
      }
      __syncwarp();
      // Jacobian rows: J[s][q] = [s == q] - tau sum_j nu_js D_jq (j increasing)
#pragma unroll
      for (int q = 0; q < kSPL; ++q) {
        const int s = lane + 32 * q;
        if (s < N) {
          L* row = Jm + (size_t)s * N;
          for (int cc = 0; cc < N; ++cc) row[cc] = L(0);
          for (int e = md.sp_ptr[s]; e < md.sp_ptr[s + 1]; ++e) {
            const int j = md.sp_j[e];
            if (!bit(nc, j)) continue;
            const L v = (L)md.sp_nu[e];
            const int nr = md.nreact[j];
            for (int k = 0; k < nr; ++k) {
              const int qq = md.rsp[j][k];
              row[qq] = row[qq] + v * Dm[j * 3 + k];
            }
          }
          for (int cc = 0; cc < N; ++cc) row[cc] = (s == cc ? L(1) : L(0)) - taur * row[cc];
        }
      }
      __syncwarp();
      // Gaussian elimination with partial pivoting (largest |pivot|, lowest row on ties)
      for (int k = 0; k < N; ++k) {
        L best = L(-1);
        int piv = N;
        for (int i = k + lane; i < N; i += 32) {
          const L v = fabs(Jm[(size_t)i * N + k]);
          if (v > best) {
            best = v;
            piv = i;
          }
        }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
          const L ob = __shfl_xor_sync(0xffffffffu, best, d);
          const int op = __shfl_xor_sync(0xffffffffu, piv, d);
          if (ob > best || (ob == best && op < piv)) {
            best = ob;
            piv = op;
          }
        }
        if (!(best > L(0)) || piv >= N) return 2;  // zero or non-finite column: singular
        if (piv != k) {
          for (int cc = lane; cc < N; cc += 32) {
            const L t = Jm[(size_t)k * N + cc];
            Jm[(size_t)k * N + cc] = Jm[(size_t)piv * N + cc];
            Jm[(size_t)piv * N + cc] = t;
          }
          if (lane == 0) {
            const L t = bv[k];
            bv[k] = bv[piv];
            bv[piv] = t;
          }
        }
        __syncwarp();
        const L pk = Jm[(size_t)k * N + k];
        const L bk = bv[k];
        for (int i = k + 1 + lane; i < N; i += 32) {
          const L l = Jm[(size_t)i * N + k] / pk;
          for (int cc = k + 1; cc < N; ++cc)
            Jm[(size_t)i * N + cc] = Jm[(size_t)i * N + cc] - l * Jm[(size_t)k * N + cc];
          bv[i] = bv[i] - l * bk;
        }
        __syncwarp();
      }
      // column-oriented back substitution
      for (int i = N - 1; i >= 0; --i) {
        const L di = bv[i] / Jm[(size_t)i * N + i];
        __syncwarp();
        for (int rr = lane; rr < i; rr += 32) bv[rr] = bv[rr] - Jm[(size_t)rr * N + i] * di;
        if (lane == 0) bv[i] = di;
        __syncwarp();
      }
      double dmax = 0.0, ymax = 0.0;
#pragma unroll
      for (int q = 0; q < kSPL; ++q) {
        const int s = lane + 32 * q;
        if (s < N) {
          const double d = (double)bv[s];
          const double yn = sl.y[s] + d;
          sl.y[s] = yn;
          dmax = fabs(d) > dmax ? fabs(d) : dmax;
          ymax = fabs(yn) > ymax ? fabs(yn) : ymax;
        }
      }
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) {
        const double o1 = __shfl_xor_sync(0xffffffffu, dmax, d);
        const double o2 = __shfl_xor_sync(0xffffffffu, ymax, d);
        dmax = o1 > dmax ? o1 : dmax;
        ymax = o2 > ymax ? o2 : ymax;
      }
      __syncwarp();
      if (dmax <= tol * (ymax > 1.0 ? ymax : 1.0)) return 0;
    }
    return 1;
  }

  // kGrid: time-grid output compiled in (absent from the build that serves plain calls).
  template <bool kGrid>
  __device__ static void run(const WarpModel& md, const WarpSlab& sl, const SimArgs& A,
                             long long i, int lane) {
    const int N = md.N, M = md.M;
    const uint32_t k0 = (uint32_t)A.seed, k1 = (uint32_t)(A.seed >> 32);
    const uint32_t id = (uint32_t)(A.id_base + (unsigned long long)i);
    const uint32_t Mr = (uint32_t)M;
    R* a_s = static_cast<R*>(sl.a);
    R* ac_s = static_cast<R*>(sl.ac);
    uint32_t status = 0;

    R th[kRPL];
    bool bad = false;
#pragma unroll
    for (int q = 0; q < kRPL; ++q) {
      const int j = lane + 32 * q;
      double v = 0.0;
      if (j < M) v = A.theta ? A.theta[i * M + j] : md.rates[j];
      if (!(v >= 0.0)) bad = true;
      th[q] = (R)v;
    }
    const int64_t* x0 = A.x0_per ? A.x0 + i * N : A.x0;
#pragma unroll
    for (int q = 0; q < kSPL; ++q) {
      const int s = lane + 32 * q;
      if (s < N) {
        sl.x[s] = x0[s];
        if (x0[s] < 0) bad = true;
      }
    }
    // a malformed observation grid (not finite, negative or decreasing) is bad input
    if (kGrid && A.K_obs > 0 && lane == 0) {
      double prev = 0.0;
      for (int k = 0; k < A.K_obs; ++k) {
        const double tk = A.t_obs[k];
        if (!(tk >= prev) || !(tk <= 1.0e300)) bad = true;
        prev = tk;
      }
    }
    bad = __any_sync(0xffffffffu, bad);
    __syncwarp();
    const double T = A.T_per ? A.T[i] : A.T[0];
    long long r[kRPL];
    double G[kRPL];
    R g[kRPL], a[kRPL];
#pragma unroll
    for (int q = 0; q < kRPL; ++q) {
      r[q] = 0;
      G[q] = 0.0;
    }
    long long cnt[4] = {0, 0, 0, 0};
    double t = 0.0;
    uint32_t step = 0;
    int reject_run = 0;
    if (bad) {
      status |= ML_ST_BAD_INPUT;
      t = T;
    }
    if (T != T) t = 0.0;

    // Time-grid output: X(t_k) of the right-continuous path; each lane writes its own
    // species, the grid index is warp-uniform.
    int kobs = 0;
    auto record = [&](double tcut, bool inclusive) {
      while (kobs < A.K_obs) {
        const double tk = A.t_obs[kobs];
        if (inclusive ? !(tk <= tcut) : !(tk < tcut)) break;
        int64_t* o = A.X_obs + ((long long)i * A.K_obs + kobs) * N;
#pragma unroll
        for (int q = 0; q < kSPL; ++q) {
          const int s = lane + 32 * q;
          if (s < N) o[s] = sl.x[s];
        }
        ++kobs;
      }
    };
    auto stop_time = [&]() -> double {
      if (kobs < A.K_obs) {
        const double tk = A.t_obs[kobs];
        if (tk < T) return tk;
      }
      return T;
    };
    if (kGrid && A.K_obs > 0) record(t, true);

    auto eval_props = [&]() {
#pragma unroll
      for (int q = 0; q < kRPL; ++q) {
        const int j = lane + 32 * q;
        g[q] = R(0);
        a[q] = R(0);
        if (j < M) {
          g[q] = g_int(md, j, sl.x);
          a[q] = th[q] * g[q];
          a_s[j] = a[q];
        }
      }
      __syncwarp();
    };
    // After a firing of reaction k inside a burst: recompute only the propensities of the
    // reactions with a reactant that k changed (the others' reactant counts, hence their
    // values, are unchanged, so the result equals eval_props bit for bit).
    auto update_props = [&](int k) {
      const uint64_t changed = k >= 0 ? md.cmask[k] : ~0ULL;  // unknown: recompute all
#pragma unroll
      for (int q = 0; q < kRPL; ++q) {
        const int j = lane + 32 * q;
        if (j < M && (md.rmask[j] & changed) != 0ULL) {
          g[q] = g_int(md, j, sl.x);
          a[q] = th[q] * g[q];
          a_s[j] = a[q];
        }
      }
      __syncwarp();
    };

    // Fast precision: inside a burst each lane accumulates its G_j and the elapsed time in
    // compensated FP32 and folds them into the FP64 totals once at the end of the burst.
    // The propensities come from an FP32 copy of the state (kept in the leap's xn storage,
    // unused during a burst, and updated with each firing), one FP32 warp scan gives a0
    // and the pick, and the next firing's random block is generated one firing ahead.
    auto ssa_burst_fast = [&](int n_max, R a0_unused) {
      (void)a0_unused;
      const double rem = T - t;
      const float remf = (float)rem;
      float el = 0.f, elc = 0.f;
      float Gs[kRPL], Gc[kRPL];
#pragma unroll
      for (int q = 0; q < kRPL; ++q) Gs[q] = Gc[q] = 0.f;
      bool to_horizon = false;
      int fired = -1;
      float* xf = reinterpret_cast<float*>(sl.xn);
#pragma unroll
      for (int q = 0; q < kSPL; ++q) {
        const int s = lane + 32 * q;
        if (s < N) xf[s] = (float)sl.x[s];
      }
      __syncwarp();
      Words4 w = philox_block(k0, k1, id, step, Mr + 2u, 0u);
      for (int b = 0; b < n_max; ++b) {
        if (b > 0) {  // reactions with a reactant the last firing changed
          const uint64_t changed = fired >= 0 ? md.cmask[fired] : ~0ULL;
#pragma unroll
          for (int q = 0; q < kRPL; ++q) {
            const int j = lane + 32 * q;
            if (j < M && (md.rmask[j] & changed) != 0ULL) {
              g[q] = (R)WarpTraj<P>::g_flt(md, j, xf);
              a[q] = th[q] * g[q];
            }
          }
        }
        float S, E;
        const float a0 = WarpTraj<P>::scan_total(a, M, lane, S, E);
        if (a0 == 0.f) {
          to_horizon = true;
          break;
        }
        const Words4 w_next = philox_block(k0, k1, id, step, Mr + 2u, (uint32_t)b + 1u);
        const float dt = __fdividef(-P::log(P::u(w, 0)), a0);  // about 2 ulp
        if ((el - elc) + dt > remf) {
          to_horizon = true;
          break;
        }
#pragma unroll
        for (int q = 0; q < kRPL; ++q) kahan_add(Gs[q], Gc[q], (float)g[q] * dt);
        kahan_add(el, elc, dt);
        if (kGrid && A.K_obs > 0) {
          record(t + ((double)el - (double)elc), false);  // before the firing: old state
          __syncwarp();
        }
        const int pk = WarpTraj<P>::pick_scanned(a_s, a, w, M, lane, S, E, a0);
        fired = pk;
        if (pk >= 0) {
          const int e0 = md.rx_ptr[pk], e1 = md.rx_ptr[pk + 1];
          for (int e = e0 + lane; e < e1; e += 32) {
            const int sp = md.rx_s[e], v = md.rx_nu[e];
            sl.x[sp] += v;
            xf[sp] += (float)v;
          }
#pragma unroll
          for (int q = 0; q < kRPL; ++q)
            if (lane + 32 * q == pk) r[q] += 1;
          cnt[2] += 1;
        }
        __syncwarp();
        if (kGrid && A.K_obs > 0) record(t + ((double)el - (double)elc), true);
        w = w_next;
      }
      // the propensities in shared memory (read by the next evaluation's step sizes) are
      // recomputed there; g and a stay current for the horizon term below
      const double elapsed = (double)el - (double)elc;
#pragma unroll
      for (int q = 0; q < kRPL; ++q) G[q] = G[q] + ((double)Gs[q] - (double)Gc[q]);
      if (to_horizon) {
        const double left = rem - elapsed > 0.0 ? rem - elapsed : 0.0;
#pragma unroll
        for (int q = 0; q < kRPL; ++q) G[q] = G[q] + (double)g[q] * left;
        t = T;
      } else {
        t = t + elapsed;
      }
    };

    auto ssa_burst = [&](int n_max, R a0) {
      if (!P::kRef) {
        ssa_burst_fast(n_max, a0);
        return;
      }
      int fired = -1;
      for (int b = 0; b < n_max; ++b) {
        if (b > 0) {
          update_props(fired);
          a0 = tree_sum(a, lane, M);
        }
        if (a0 == R(0)) {
          const double rem = T - t;
#pragma unroll
          for (int q = 0; q < kRPL; ++q) G[q] = G[q] + (double)g[q] * rem;
          t = T;
          return;
        }
        const Words4 w = philox_block(k0, k1, id, step, Mr + 2u, (uint32_t)b);
        const R u1 = P::u(w, 0);
        const R dt = -P::log(u1) / a0;
        const double tn = t + (double)dt;
        if (tn > T) {
          const double rem = T - t;
#pragma unroll
          for (int q = 0; q < kRPL; ++q) G[q] = G[q] + (double)g[q] * rem;
          t = T;
          return;
        }
#pragma unroll
        for (int q = 0; q < kRPL; ++q) {
          if (P::kRef) G[q] = G[q] + (double)g[q] * (double)dt;
          else G[q] = G[q] + (double)(g[q] * dt);  // FP32 increment, FP64 accumulation
        }
        if (kGrid && A.K_obs > 0) {
          record(tn, false);  // points before the firing see the old state
          __syncwarp();
        }
        t = tn;
        const int pk = pick(a_s, a, w, M, lane);
        fired = pk;
        if (pk >= 0) {
          const int e0 = md.rx_ptr[pk], e1 = md.rx_ptr[pk + 1];
          for (int e = e0 + lane; e < e1; e += 32) sl.x[md.rx_s[e]] += md.rx_nu[e];
#pragma unroll
          for (int q = 0; q < kRPL; ++q)
            if (lane + 32 * q == pk) r[q] += 1;
          cnt[2] += 1;
        }
        __syncwarp();
        if (kGrid && A.K_obs > 0) record(t, true);  // a point at the firing time: new state
      }
    };

    const R eps = (R)A.eps;
    for (;;) {
      if (!(t < T)) break;
      if ((long long)step >= A.max_steps) {
        status |= ML_ST_STEP_LIMIT;
        break;
      }
      {
        bool big = false;
#pragma unroll
        for (int q = 0; q < kSPL; ++q) {
          const int s = lane + 32 * q;
          big = big || (s < N && sl.x[s] > kCountLimit);
        }
#pragma unroll
        for (int q = 0; q < kRPL; ++q) big = big || r[q] > kCountLimit;
        if (__any_sync(0xffffffffu, big)) {
          status |= ML_ST_OVERFLOW;
          break;
        }
      }
      eval_props();
      const R a0 = tree_sum(a, lane, M);
      if (a0 == R(0)) {
        const double rem = T - t;
#pragma unroll
        for (int q = 0; q < kRPL; ++q) G[q] = G[q] + (double)g[q] * rem;
        t = T;
        break;
      }
      int burst = 0;
      if (A.mode == ML_MODE_SSA_ONLY) burst = A.n_ssa_ex;
      else {
        // critical reactions
        uint32_t nc[kRPL];
        R ac[kRPL];
#pragma unroll
        for (int q = 0; q < kRPL; ++q) {
          const int j = lane + 32 * q;
          bool crit = false;
          if (j < M && a[q] > R(0)) {
            // min over consumed species of floor(x_s/|nu_js|) below n_c, i.e. some
            // consumed species has x_s < n_c |nu_js|
            for (int e = md.rx_ptr[j]; e < md.rx_ptr[j + 1]; ++e) {
              const int v = md.rx_nu[e];
              if (v < 0 && sl.x[md.rx_s[e]] < (long long)A.n_c * (long long)(-v)) crit = true;
            }
          }
          ac[q] = crit ? a[q] : R(0);
          if (j < M) ac_s[j] = ac[q];
          nc[q] = __ballot_sync(0xffffffffu, !crit);
        }
        __syncwarp();
        const R a0c = tree_sum(ac, lane, M);
        const R tau_ex = tau_select(md, a_s, sl.x, nc, eps, lane);
        bool implicit = false;
        R tau1 = tau_ex;
        if (A.mode == ML_MODE_ADAPTIVE && md.n_pairs > 0) {
          uint32_t pe[kRPL];
          bool any = false;
#pragma unroll
          for (int q = 0; q < kRPL; ++q) {
            const int j = lane + 32 * q;
            bool on = false;
            if (j < M) {
              int k = md.partner[j];
              int lo_j = j, hi_j = k;
              if (k < 0) {
                // j may be the higher reaction of a pair: find it
                for (int jj = 0; jj < j; ++jj)
                  if (md.partner[jj] == j) {
                    lo_j = jj;
                    hi_j = j;
                    k = jj;
                    break;
                  }
              }
              if (k >= 0 && bit(nc, lo_j) && bit(nc, hi_j)) {
                const R aj = a_s[lo_j], ak = a_s[hi_j];
                const R lo = aj < ak ? aj : ak;
                on = fabs(aj - ak) <= (R)A.pe_delta * lo;
              }
            }
            pe[q] = __ballot_sync(0xffffffffu, on);
            any = any || pe[q] != 0;
          }
          if (any) {
            uint32_t use[kRPL];
#pragma unroll
            for (int q = 0; q < kRPL; ++q) use[q] = nc[q] & ~pe[q];
            const R tau_im = tau_select(md, a_s, sl.x, use, eps, lane);
            if (tau_im > (R)A.stiff_ratio * tau_ex) {
              implicit = true;
              tau1 = tau_im;
            }
          }
        }
        bool overflow = false;
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
          const double stop = kGrid ? stop_time() : T;
          const double rem = stop - t;
          R tau = tau1;
          if (tau2 < tau) tau = tau2;
          bool at_horizon = false;
          if ((R)rem <= tau) {
            tau = (R)rem;
            at_horizon = true;
          }
          const bool crit_fire = (tau2 <= tau1) && (tau2 <= (R)rem);
          {
            bool over = false;
#pragma unroll
            for (int q = 0; q < kRPL; ++q) {
              const int j = lane + 32 * q;
              over = over || (j < M && bit(nc, j) && a[q] * tau > (R)kLeapLimit);
            }
            overflow = __any_sync(0xffffffffu, over);
            if (overflow) break;
          }
          int cpk = -1;
          if (crit_fire) {
            const Words4 w = philox_block(k0, k1, id, step, Mr + 1u, 0u);
            cpk = pick(ac_s, ac, Words4{0u, 0u, w.w0, w.w1}, M, lane);
          }
          const bool implicit_step = implicit && tau > tau_ex;
          long long K[kRPL];
#pragma unroll
          for (int q = 0; q < kRPL; ++q) {
            const int j = lane + 32 * q;
            K[q] = 0;
            if (j < M) {
              if (bit(nc, j))
                K[q] = poisson_draw<P>(a[q] * tau, k0, k1, id, step, (uint32_t)j, status);
              sl.K[j] = K[q];
            }
          }
          __syncwarp();
          if (implicit_step) {
            const double taud = (double)tau;
            const bool an = A.jacobian == ML_JAC_ANALYTIC;
            const int rc = (!P::kRef && A.newton_fp32)
                               ? implicit_solve<float>(md, sl, th, nc, a_s, taud, A.newton_tol,
                                                       A.newton_maxit, A.fd_h, an, lane)
                               : implicit_solve<double>(md, sl, th, nc, a_s, taud,
                                                        A.newton_tol, A.newton_maxit, A.fd_h,
                                                        an, lane);
            if (rc != 0) {
              status |= ML_ST_NEWTON_FAIL;
              implicit = false;
              tau1 = tau_ex;
              step++;
              __syncwarp();
              continue;
            }
#pragma unroll
            for (int q = 0; q < kRPL; ++q) {
              const int j = lane + 32 * q;
              if (j < M && bit(nc, j)) {
                const double ayj = (double)th[q] * g_real(md, j, sl.y, -1, 0.0);
                const double v = (ayj * taud + (double)K[q]) - (double)a[q] * taud;
                const double rv = round(v);
                K[q] = !(rv < 0x1p62) ? kCountLimit : (rv > 0.0 ? (long long)rv : 0);
              }
            }
            bool over = false;
#pragma unroll
            for (int q = 0; q < kRPL; ++q) {
              const int j = lane + 32 * q;
              over = over || (j < M && bit(nc, j) && K[q] > kLeapLimitInt);
            }
            overflow = __any_sync(0xffffffffu, over);
            if (overflow) break;
          }
#pragma unroll
          for (int q = 0; q < kRPL; ++q) {
            const int j = lane + 32 * q;
            if (j == cpk) K[q] = 1;
            else if (j < M && !bit(nc, j)) K[q] = 0;
            if (j < M) sl.K[j] = K[q];
          }
          __syncwarp();
          bool negative = false;
#pragma unroll
          for (int q = 0; q < kSPL; ++q) {
            const int s = lane + 32 * q;
            if (s < N) {
              long long v = sl.x[s];
              for (int e = md.sp_ptr[s]; e < md.sp_ptr[s + 1]; ++e)
                v += (long long)md.sp_nu[e] * sl.K[md.sp_j[e]];
              sl.xn[s] = v;
              if (v < 0) negative = true;
            }
          }
          negative = __any_sync(0xffffffffu, negative);
          __syncwarp();
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
          for (int q = 0; q < kRPL; ++q) {
            const int j = lane + 32 * q;
            if (j < M) {
              const R gn = g_int(md, j, sl.xn);
              r[q] += K[q];
              if (P::kRef) G[q] = G[q] + half * ((double)g[q] + (double)gn);
              else G[q] = G[q] + (double)(half_r * (g[q] + gn));  // FP32 increment
            }
          }
          __syncwarp();
#pragma unroll
          for (int q = 0; q < kSPL; ++q) {
            const int s = lane + 32 * q;
            if (s < N) sl.x[s] = sl.xn[s];
          }
          __syncwarp();
          t = at_horizon ? stop : t + (double)tau;
          if (kGrid && A.K_obs > 0) record(t, true);
          cnt[implicit_step ? 1 : 0] += 1;
          step++;
          reject_run = 0;
          break;
        }
        if (overflow) {
          status |= ML_ST_OVERFLOW;
          break;
        }
      }
      if (burst > 0) {
        ssa_burst(burst, a0);
        step++;
        reject_run = 0;
      }
    }
    status = __reduce_or_sync(0xffffffffu, status);
    // grid points past the end (beyond T, after a step-limit stop, or all of a rejected
    // grid): the final state
    if (kGrid) {
      for (; kobs < A.K_obs; ++kobs) {
        int64_t* o = A.X_obs + ((long long)i * A.K_obs + kobs) * N;
#pragma unroll
        for (int q = 0; q < kSPL; ++q) {
          const int s = lane + 32 * q;
          if (s < N) o[s] = sl.x[s];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kSPL; ++q) {
      const int s = lane + 32 * q;
      if (s < N) A.X[i * N + s] = sl.x[s];
    }
#pragma unroll
    for (int q = 0; q < kRPL; ++q) {
      const int j = lane + 32 * q;
      if (j < M) {
        A.r[i * M + j] = r[q];
        A.G[i * M + j] = G[q];
      }
    }
    if (lane == 0) {
      A.status[i] = status;
      if (A.counters)
        for (int c = 0; c < 4; ++c) A.counters[i * 4 + c] = cnt[c];
    }
    __syncwarp();
  }
};

// Kernel: model tables staged once per CTA into the front of dynamic shared memory, one
// slab per warp after them.  Plain form: warp w of CTA b runs trajectory b*warps + w.
// Persistent form: lane 0 claims the next trajectory from the device queue.
// Bounds (256, ML_WARP_MIN_BLOCKS): without a minimum-CTA hint ptxas held the kernel to 80
// registers and spilled about 1.4 KB per thread.
#ifndef ML_WARP_MIN_BLOCKS
#define ML_WARP_MIN_BLOCKS 1
#endif
template <class P, bool kGrid = false>
__global__ void __launch_bounds__(256, ML_WARP_MIN_BLOCKS) k_warp(const WarpModel* __restrict__ gmd,
                                              const SimArgs args) {
  extern __shared__ __align__(16) char smem[];
  __shared__ uint64_t mbar;
  WarpModel& md = *reinterpret_cast<WarpModel*>(smem);
  const bool staged = stage_model_bulk(&md, gmd, (uint32_t)((sizeof(WarpModel) + 15) / 16 * 16), &mbar,
                                       args.stage_polls);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const size_t mbytes = (sizeof(WarpModel) + 15) / 16 * 16;
  const int rbytes = (int)sizeof(typename P::R);
  const int lbytes = (!P::kRef && args.newton_fp32) ? 4 : 8;
  char* slab_base = smem + mbytes + (size_t)warp * warp_slab_bytes(md.N, md.M, rbytes, lbytes);
  const WarpSlab sl = carve_slab(slab_base, md.N, md.M, rbytes, lbytes);
  long long i;
  if (args.queue) {
    long long c = 0;
    if (lane == 0) c = queue_claim(args.queue, args.order, args.n_traj);
    i = __shfl_sync(0xffffffffu, c, 0);
  } else {
    i = (long long)blockIdx.x * warps + warp;
  }
  while (i < args.n_traj) {
    WarpTraj<P>::template run<kGrid>(md, sl, args, i, lane);
    if (!staged && lane == 0) args.status[i] |= ML_ST_STAGE_TIMEOUT;
    if (!args.queue) break;
    long long c = 0;
    if (lane == 0) c = queue_claim(args.queue, args.order, args.n_traj);
    i = __shfl_sync(0xffffffffu, c, 0);
  }
}

}  // namespace mlk
