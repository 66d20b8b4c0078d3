/*
 * ml_oracle.h -- plain single-threaded CPU oracle for adaptive explicit-implicit
 * tau-leaping (matLeap, Feigelman, Ganscha & Claassen 2016, arXiv:1608.07058).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path: only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant generator with the CUDA library; both are
 * written independently from the same algorithm statement (the "Implementation"
 * section of the paper plus the published methods it builds on: Gillespie 1977 SSA,
 * Gillespie 2001 tau-leaping, Cao-Gillespie-Petzold 2006 step-size selection,
 * Cao-Gillespie-Petzold 2007 adaptive explicit-implicit leaping, Rathinam-Petzold-Cao
 * 2003 implicit leaping).
 *
 * Everything is FP64 and compiled with -ffp-contract=off so that every +,-,*,/ is one
 * IEEE-754 round-to-nearest operation in the order written.
 *
 * Parity status of each function is stated in the file header of ml_oracle.c.
 */
#ifndef ML_ORACLE_H
#define ML_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Simulation modes (Section "Results": matLeap can run fully explicit or as SSA). */
#define MLO_MODE_ADAPTIVE 0      /* explicit / implicit / SSA switching (Section 2)  */
#define MLO_MODE_EXPLICIT_ONLY 1 /* never take the implicit branch                    */
#define MLO_MODE_SSA_ONLY 2      /* exact Gillespie direct method throughout          */

/* Per-trajectory status bits. */
#define MLO_ST_STEP_LIMIT 1u   /* max_steps reached before T (output is state at stop) */
#define MLO_ST_NEWTON_FAIL 2u  /* an implicit solve failed; explicit leap used instead */
#define MLO_ST_REJECT_LIMIT 4u /* max_reject consecutive negativity rejections -> SSA  */
#define MLO_ST_PTRS_CAP 8u     /* a Poisson draw hit the trial cap                     */
#define MLO_ST_OVERFLOW 64u    /* counts left the exact int64 range: stopped early;
                                  see mlo_count_limit / mlo_leap_limit                */

/* Count limits: a trajectory stops (status MLO_ST_OVERFLOW, state and statistics as at
 * the stop) when, at the start of an outer step, a count x_s or firing total r_j exceeds
 * MLO_COUNT_LIMIT, or when a leap would draw a Poisson mean a_j tau, or an implicit leap
 * would fire a reaction, more than MLO_LEAP_LIMIT times.  With at most 128 reactions and
 * |nu| <= 127 every int64 sum then stays below 2^63. */
#define MLO_COUNT_LIMIT 4611686018427387904LL /* 2^62 */
#define MLO_LEAP_LIMIT 281474976710656.0      /* 2^48 */

typedef struct {
  double eps;             /* Cao 2006 relative-change bound epsilon                  */
  int32_t n_c;            /* critical threshold: fewer than n_c firings to exhaustion */
  double ssa_factor;      /* switch to SSA when min(tau1,tau2) < ssa_factor / a0      */
  int32_t n_ssa_explicit; /* SSA burst length after an explicit choice               */
  int32_t n_ssa_implicit; /* SSA burst length after an implicit choice               */
  double pe_delta;        /* partial-equilibrium tolerance                            */
  double stiff_ratio;     /* implicit iff tau_im > stiff_ratio * tau_ex               */
  double newton_tol;      /* Newton stop: |dy|_inf <= tol * max(1,|y|_inf)          */
  int32_t newton_maxit;   /* Newton iteration cap                                     */
  double fd_h;            /* finite-difference step factor                            */
  int64_t max_steps;      /* safety cap on outer steps per trajectory                 */
  int32_t max_reject;     /* consecutive rejections before forcing an SSA burst       */
  int32_t mode;           /* MLO_MODE_*                                               */
  int32_t jacobian;       /* MLO_JAC_FD or MLO_JAC_ANALYTIC                           */
} mlo_params;

/* Jacobian of the propensities in the implicit solve: forward differences (the paper's
 * "estimated numerically") or the exact derivative of the mass-action polynomials (the
 * paper's symbolic Jacobian, Section 3). */
#define MLO_JAC_FD 0
#define MLO_JAC_ANALYTIC 1

void mlo_default_params(mlo_params* p);

/* Simulate n_traj trajectories.  Model: N species, M reactions, orders[j*N+s] = m_js
 * (reactant multiplicity), stoich[j*N+s] = nu_js (net change), rates[j] = base theta.
 * theta: [n_traj][M] per-trajectory rate constants or NULL (use rates).
 * x0: [N] (x0_per_traj=0) or [n_traj][N].  T: [1] or [n_traj].
 * Trajectory i draws its random numbers with id traj_id_base + i.
 * Outputs (host): X_out [n_traj][N], r_out [n_traj][M], G_out [n_traj][M],
 * status_out [n_traj], counters_out [n_traj][4] (explicit leaps, implicit leaps,
 * SSA firings, rejections) or NULL.
 * Returns 0, or -1 on a malformed model/argument. */
int mlo_simulate(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                 const double* rates, int64_t n_traj, const double* theta,
                 const int64_t* x0, int32_t x0_per_traj, const double* T,
                 int32_t T_per_traj, const mlo_params* p, uint64_t seed,
                 uint64_t traj_id_base, int64_t* X_out, int64_t* r_out, double* G_out,
                 uint32_t* status_out, int64_t* counters_out);

/* mlo_simulate with time-grid output: t_obs[K] finite, >= 0 and nondecreasing; X_obs
 * [n_traj][K][N] receives X(t_k), the state after every change at a time <= t_k (the path
 * is right-continuous).  Leaps end exactly at each grid point as they do at T; SSA
 * firings are not moved.  Points beyond a trajectory's end (t_k > T, or after a step-limit
 * stop) get its final state.  K = 0 is mlo_simulate. */
int mlo_simulate_grid(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                      const double* rates, int64_t n_traj, const double* theta,
                      const int64_t* x0, int32_t x0_per_traj, const double* T,
                      int32_t T_per_traj, const mlo_params* p, uint64_t seed,
                      uint64_t traj_id_base, const double* t_obs, int32_t K, int64_t* X_obs,
                      int64_t* X_out, int64_t* r_out, double* G_out, uint32_t* status_out,
                      int64_t* counters_out);

/* ---- Accuracy metric (Section 3, Table 1) ------------------------------------------
 * KL(p || q) of two integer samples (n_ref values a[i*sa], n_test values b[i*sb]):
 * histograms on the pooled range [lo, hi] with integer bin width
 * w = ceil((hi - lo + 1) / max_bins), 1/2 added to every bin of both, p from the
 * reference sample; sum over bins in lane-tree order. */
double mlo_kl_sample(int64_t n_ref, const int64_t* a, int64_t sa, int64_t n_test,
                     const int64_t* b, int64_t sb, int32_t max_bins);
/* kl_out[k][s] = mlo_kl_sample over time point k and species s of X_ref [n_ref][K][N] and
 * X_test [n_test][K][N]; *kl_mean (optional) = lane-tree sum of kl_out / (K N). */
int mlo_kl_grid(int64_t n_ref, const int64_t* X_ref, int64_t n_test, const int64_t* X_test,
                int32_t K, int32_t N, int32_t max_bins, double* kl_out, double* kl_mean);

/* Building blocks, exported so that tests can pin each one on its own. */
void mlo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double mlo_u01_from_words(uint32_t w0, uint32_t w1);
double mlo_exp(double x);
double mlo_log(double x);
double mlo_log_factorial(int64_t k);
int64_t mlo_poisson(double mu, uint64_t seed, uint32_t traj_id, uint32_t step,
                    uint32_t stream, uint32_t* status);
void mlo_poisson_batch(double mu, uint64_t seed, int64_t n, int64_t* out);
/* Cao 2006 step size for one state (all reactions non-critical unless crit_mask set). */
double mlo_tau_select(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                      const double* a, const int64_t* x, const uint8_t* use, double eps);
/* Critical reactions: crit_out[j] = 1 iff a_j > 0 and L_j = min over species consumed by
 * j (nu_js < 0) of floor(x_s / |nu_js|) is below n_c; ac_out[j] = a_j for critical j,
 * else 0.  Returns a0c (lane-tree sum of ac_out), NaN for a malformed model. */
double mlo_critical_set(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                        const double* a, const int64_t* x, int32_t n_c, uint8_t* crit_out,
                        double* ac_out);
/* Inverse-CDF pick: first j whose sequential prefix sum of w exceeds target, else the
 * last j with w_j > 0, else -1. */
int32_t mlo_pick(int32_t M, const double* w, double target);
/* The SSA switch: 1 iff min(tau1, tau2) < ssa_factor / a0. */
int mlo_ssa_switch(double tau1, double tau2, double a0, double ssa_factor);
/* Implicit firing count max(0, round((a_y tau + P) - a_x tau)), half away from zero,
 * saturated at 2^62 (which exceeds MLO_LEAP_LIMIT, so the caller stops the trajectory). */
int64_t mlo_implicit_count(double a_y, double tau, double P, double a_x);
/* Implicit solve followed by mlo_implicit_count for every j with nc[j] (K_out of the
 * others untouched).  Returns the solve's code (0 converged, 1 not, 2 singular). */
int mlo_implicit_leap(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                      const double* theta, const int64_t* x, const uint8_t* nc,
                      const double* P, const double* a_x, double tau, const mlo_params* p,
                      int64_t* K_out, int32_t* iters_out);
/* Canonical lane-tree sum (used for a0 and a0c). */
double mlo_lane_tree_sum(const double* v, int32_t n);
/* One implicit solve (Rathinam 2003): returns 0 on convergence and writes y, iterations. */
int mlo_implicit_solve(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                       const double* theta, const int64_t* x, const uint8_t* nc,
                       const double* P, const double* a_x, double tau, const mlo_params* p,
                       double* y_out, int32_t* iters_out);

/* ---- Bayesian step (Section 1: Gamma(alpha + r, beta + G) posterior) ------------- */
/* Gamma(shape, rate) draw by Marsaglia & Tsang (2000) with normals from the Marsaglia
 * polar method; shape < 1 by Gamma(shape + 1) U^(1/shape).  Random numbers: counter
 * (traj_id, 0x80000000 + stream, 0, block), block 2t the polar pair of trial t, block 2t+1
 * the acceptance uniform (words 0, 1) and the boost uniform (words 2, 3).  Returns NaN
 * for shape <= 0 or rate <= 0; sets *status bit 1 if the trial cap was hit. */
double mlo_gamma(double shape, double rate, uint64_t seed, uint32_t traj_id, uint32_t stream,
                 uint32_t* status);
/* theta[i][j] ~ Gamma(alpha_j + r[i][j], beta_j + G[i][j]) for n trajectories (alpha,
 * beta: [M] or [n][M] with *_per_traj), trajectory i with id traj_id_base + i, stream j. */
int mlo_posterior_sample(int64_t n, int32_t M, const double* alpha, int32_t alpha_per_traj,
                         const double* beta, int32_t beta_per_traj, const int64_t* r,
                         const double* G, uint64_t seed, uint64_t traj_id_base,
                         double* theta_out, uint32_t* status_out);
/* Systematic resampling of n particles from log-weights: weights w_i = exp(logw_i - max)
 * are quantized to integers q_i = floor(w_i 2^40) (so every prefix sum is exact), Q = sum
 * q_i, u = uniform from counter (id_base, 0xC0000000, 0, 0) words 0,1, and ancestor k is
 * the first i with prefix_i > floor(((k + u) / n) Q) computed as
 * floor((k Q + floor(u Q)) / n) in 128-bit integer arithmetic.  A NaN log-weight counts
 * as weight 0.  Returns -1 (every ancestor -1) when no weight is positive or the maximum
 * log-weight is +inf. */
int mlo_resample_systematic(int64_t n, const double* logw, uint64_t seed,
                            uint64_t id_base, int64_t* ancestors);

#ifdef __cplusplus
}
#endif
#endif
