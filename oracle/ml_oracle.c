/*
 * ml_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the adaptive
 * explicit-implicit tau-leaping hot path of matLeap (arXiv:1608.07058).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the benchmark's
 * CPU-baseline leg.  The CUDA library never links, includes or calls this file, and
 * this file includes nothing of the CUDA library.  Compile with -ffp-contract=off.
 *
 * What it computes (paper, Section 1 "Background" and Section 2 "Implementation"):
 *   per trajectory, X(T), the firing counts r_j and the integrals G_j = int g_j(X_s) ds
 *   (trapezoid while leaping, exact under SSA), for a mass-action network with
 *   propensities a_j(x) = theta_j g_j(x), simulated by adaptive explicit/implicit
 *   tau-leaping with critical reactions and the paper's SSA switch.
 * The method is an approximation, so the oracle is the algorithm itself, step by step:
 *   1. propensities a_j, a0                                 (Section 1, a_i = theta_i g_i)
 *   2. critical set: a_j > 0 and fewer than n_c firings to exhaustion   (Section 2)
 *   3. tau_ex by the Cao 2006 epsilon bound on mean and variance of each reactant
 *   4. partial-equilibrium pairs and tau_im without them; implicit iff tau_im is much
 *      longer (Cao 2007, Section 2 of the paper)
 *   5. tau2 ~ Exp(a0c) to the next critical firing; SSA burst when min(tau1,tau2) is
 *      comparable to 1/a0 (the paper's modification, Section 2)
 *   6. explicit Poisson leap or implicit Newton leap (Rathinam 2003); one critical firing
 *   7. negativity check and halving of tau1; commit, r += K, G += trapezoid.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py against
 * something other than itself (an independent Philox, libm/mpmath error bounds, scipy
 * Poisson distributions, closed-form network laws, exact CME solutions, hand-computed
 * step sizes, Gamma conjugacy).  Nothing here is "parity unpinned".
 */
#include "ml_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC11).  Ten rounds of two 32x32->64 multiplies with Weyl key bumps.
 * ---------------------------------------------------------------------------------- */
#define PHILOX_MUL_A 0xD2511F53u
#define PHILOX_MUL_B 0xCD9E8D57u
#define PHILOX_WEYL_A 0x9E3779B9u /* golden ratio */
#define PHILOX_WEYL_B 0xBB67AE85u /* sqrt(3) - 1  */

void mlo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_WEYL_A;
      k1 += PHILOX_WEYL_B;
    }
    uint64_t pa = (uint64_t)PHILOX_MUL_A * (uint64_t)c0;
    uint64_t pb = (uint64_t)PHILOX_MUL_B * (uint64_t)c2;
    uint32_t hi_a = (uint32_t)(pa >> 32), lo_a = (uint32_t)pa;
    uint32_t hi_b = (uint32_t)(pb >> 32), lo_b = (uint32_t)pb;
    uint32_t n0 = hi_b ^ c1 ^ k0;
    uint32_t n1 = lo_b;
    uint32_t n2 = hi_a ^ c3 ^ k1;
    uint32_t n3 = lo_a;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random-number layout: key = (seed lo, seed hi); counter = (trajectory id, step,
 * stream, block).  Streams: j in [0,M) Poisson draws of reaction j (block = trial),
 * M the time to the next critical firing, M+1 the critical pick, M+2 the SSA burst
 * (block = SSA step within the burst). */
static void block_words(uint64_t seed, uint32_t id, uint32_t step, uint32_t stream,
                        uint32_t block, uint32_t w[4]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {id, step, stream, block};
  mlo_philox4x32_10(ctr, key, w);
}

/* Uniform on (0,1): 52 random bits n = (w0>>6)*2^26 + (w1>>6); u = (n + 0.5) * 2^-52.
 * Every step is exact, so u in [2^-53, 1 - 2^-53]. */
double mlo_u01_from_words(uint32_t w0, uint32_t w1) {
  double n = (double)(w0 >> 6) * 67108864.0 + (double)(w1 >> 6);
  return (n + 0.5) * 0x1p-52;
}

/* ------------------------------------------------------------------------------------
 * Elementary functions, written from Cody & Waite, "Software Manual for the Elementary
 * Functions" (1980): additive range reduction by k*ln2 with ln2 split into a 32-bit
 * head and a tail, then a polynomial on the reduced argument.  Plain +,-,*,/ only.
 * ---------------------------------------------------------------------------------- */
static const double LN2_HEAD = 0x1.62e42fee00000p-1; /* ln 2 to 32 significant bits */
static const double LN2_TAIL = 0x1.a39ef35793c76p-33; /* ln 2 - LN2_HEAD              */
static const double INV_LN2 = 0x1.71547652b82fep+0;   /* 1 / ln 2                     */
static const double SQRT_2 = 0x1.6a09e667f3bcdp+0;
static const double HALF_LOG_2PI = 0x1.d67f1c864beb5p-1; /* log(2 pi) / 2 */

static double pow2_int(int k) { /* 2^k for -1022 <= k <= 1023, exact */
  uint64_t bits = (uint64_t)(k + 1023) << 52;
  double r;
  memcpy(&r, &bits, sizeof r);
  return r;
}

/* exp(x) for x in [-708, 709]: x = k ln2 + r, |r| <= ln2/2, exp(r) by its Taylor series
 * to degree 13 (truncation below 2^-57 relative), Horner from the highest term.
 * x < -708 returns 0; x > 709 returns +inf. */
double mlo_exp(double x) {
  if (x != x) return x;
  if (x < -708.0) return 0.0;
  if (x > 709.0) return INFINITY;
  double kd = floor(x * INV_LN2 + 0.5);
  double r = (x - kd * LN2_HEAD) - kd * LN2_TAIL;
  double p = 1.0 / 6227020800.0; /* 1/13! */
  p = p * r + 1.0 / 479001600.0;  /* 1/12! */
  p = p * r + 1.0 / 39916800.0;   /* 1/11! */
  p = p * r + 1.0 / 3628800.0;    /* 1/10! */
  p = p * r + 1.0 / 362880.0;     /* 1/9!  */
  p = p * r + 1.0 / 40320.0;      /* 1/8!  */
  p = p * r + 1.0 / 5040.0;       /* 1/7!  */
  p = p * r + 1.0 / 720.0;        /* 1/6!  */
  p = p * r + 1.0 / 120.0;        /* 1/5!  */
  p = p * r + 1.0 / 24.0;         /* 1/4!  */
  p = p * r + 1.0 / 6.0;          /* 1/3!  */
  p = p * r + 0.5;                /* 1/2!  */
  p = p * r + 1.0;
  p = p * r + 1.0;
  return p * pow2_int((int)kd);
}

/* log(x) for positive normal x: x = 2^e m with m in [sqrt(1/2), sqrt(2)),
 * f = m - 1 (exact), s = f / (2 + f), log m = 2 atanh(s) = 2 s (1 + z/3 + z^2/5 + ...),
 * z = s^2 <= 0.0295, series to z^11/23 (truncation below 2^-60). */
double mlo_log(double x) {
  if (x != x || x < 0.0) return NAN;
  if (x == 0.0) return -INFINITY;
  if (x == INFINITY) return x;
  uint64_t bits;
  memcpy(&bits, &x, sizeof bits);
  int e = (int)((bits >> 52) & 0x7ff) - 1023;
  uint64_t mbits = (bits & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
  double m;
  memcpy(&m, &mbits, sizeof m);
  if (m > SQRT_2) {
    m = m * 0.5;
    e = e + 1;
  }
  double f = m - 1.0;
  double s = f / (2.0 + f);
  double z = s * s;
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
  double two_s = s + s;
  double logm = two_s + (two_s * z) * q;
  double ed = (double)e;
  return ed * LN2_HEAD + (ed * LN2_TAIL + logm);
}

/* log k!: below 16 the log of the exact product k! (k! < 2^53 there); from 16 on the
 * Stirling series of log Gamma(z), z = k + 1:
 *   (z - 1/2) log z - z + log(2 pi)/2 + 1/(12z) - 1/(360z^3) + 1/(1260z^5)
 *   - 1/(1680z^7) + 1/(1188z^9),   truncation error below 1e-16 for z >= 17. */
double mlo_log_factorial(int64_t k) {
  if (k < 2) return 0.0;
  if (k < 16) {
    double f = 1.0;
    for (int64_t i = 2; i <= k; ++i) f = f * (double)i;
    return mlo_log(f);
  }
  double z = (double)k + 1.0;
  double w = 1.0 / z;
  double w2 = w * w;
  double ser = 1.0 / 1188.0;
  ser = ser * w2 - 1.0 / 1680.0;
  ser = ser * w2 + 1.0 / 1260.0;
  ser = ser * w2 - 1.0 / 360.0;
  ser = ser * w2 + 1.0 / 12.0;
  ser = ser * w;
  return (((z - 0.5) * mlo_log(z) - z) + HALF_LOG_2PI) + ser;
}

/* ------------------------------------------------------------------------------------
 * Poisson(mu).  mu == 0: 0 without drawing.  mu < 10: inversion by sequential search
 * from k = 0 (p = e^-mu, F = p; while u > F: k++, p *= mu/k, F += p; stop if p
 * underflows).  mu >= 10: PTRS, the transformed rejection method with squeeze of
 * Hoermann, "The transformed rejection method for generating Poisson random
 * variables", Insurance: Mathematics and Economics 12 (1993).  Trial b uses block b of
 * the reaction's stream: U from words 0,1 and V from words 2,3.
 * ---------------------------------------------------------------------------------- */
#define PTRS_MAX_TRIALS 256

int64_t mlo_poisson(double mu, uint64_t seed, uint32_t traj_id, uint32_t step,
                    uint32_t stream, uint32_t* status) {
  if (!(mu > 0.0)) return 0;
  uint32_t w[4];
  if (mu < 10.0) {
    block_words(seed, traj_id, step, stream, 0, w);
    double u = mlo_u01_from_words(w[0], w[1]);
    double p = mlo_exp(-mu);
    double F = p;
    int64_t k = 0;
    while (u > F) {
      k = k + 1;
      p = p * (mu / (double)k);
      if (p == 0.0) break;
      F = F + p;
    }
    return k;
  }
  double slam = sqrt(mu);
  double loglam = mlo_log(mu);
  double b = 0.931 + 2.53 * slam;
  double a = -0.059 + 0.02483 * b;
  double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
  double v_r = 0.9277 - 3.6224 / (b - 2.0);
  for (uint32_t trial = 0; trial < PTRS_MAX_TRIALS; ++trial) {
    block_words(seed, traj_id, step, stream, trial, w);
    double U = mlo_u01_from_words(w[0], w[1]) - 0.5;
    double V = mlo_u01_from_words(w[2], w[3]);
    double us = 0.5 - fabs(U);
    double kd = floor((((2.0 * a) / us + b) * U + mu) + 0.43);
    if (us >= 0.07 && V <= v_r) return (int64_t)kd;
    if (kd < 0.0 || (us < 0.013 && V > us)) continue;
    double lhs = (mlo_log(V) + mlo_log(inv_alpha)) - mlo_log(a / (us * us) + b);
    double rhs = (-mu + kd * loglam) - mlo_log_factorial((int64_t)kd);
    if (lhs <= rhs) return (int64_t)kd;
  }
  if (status) *status |= MLO_ST_PTRS_CAP;
  return (int64_t)floor(mu + 0.5);
}

/* n draws of Poisson(mu), draw i keyed by trajectory id i, step 0, stream 0. */
void mlo_poisson_batch(double mu, uint64_t seed, int64_t n, int64_t* out) {
  uint32_t st = 0;
  for (int64_t i = 0; i < n; ++i) out[i] = mlo_poisson(mu, seed, (uint32_t)i, 0u, 0u, &st);
}

/* ------------------------------------------------------------------------------------
 * Canonical order of a sum over reactions (a0 and a0c): element j belongs to lane
 * j mod 32; each lane adds its elements in increasing j (an empty lane holds 0.0);
 * then lanes are combined pairwise, lane l with lane l xor d, for d = 16, 8, 4, 2, 1,
 * and lane 0's value is the sum.  Written out lane by lane.
 * ---------------------------------------------------------------------------------- */
double mlo_lane_tree_sum(const double* v, int32_t n) {
  double lane[32], next[32];
  for (int l = 0; l < 32; ++l) lane[l] = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    int l = j % 32;
    if (j < 32) lane[l] = v[j];
    else lane[l] = lane[l] + v[j];
  }
  for (int d = 16; d >= 1; d /= 2) {
    for (int l = 0; l < 32; ++l) next[l] = lane[l] + lane[l ^ d];
    for (int l = 0; l < 32; ++l) lane[l] = next[l];
  }
  return lane[0];
}

/* ------------------------------------------------------------------------------------
 * Model tables (mass action, Section 1: a_j = theta_j g_j(X), g_j a function of the
 * reactant counts; here g_j = prod_s C(x_s, m_js), the number of distinct reactant
 * combinations).
 * ---------------------------------------------------------------------------------- */
typedef struct {
  int32_t N, M;
  const int32_t* ord; /* [M][N] */
  const int32_t* nu;  /* [M][N] */
  int32_t* order_tot; /* [M] total reactant order of reaction j */
  uint8_t* is_reactant; /* [N] species is a reactant of some reaction */
  int32_t* pair_of;   /* [M] partner reaction of a reversible pair, -1 if none */
  int32_t n_pairs;
  int32_t* pair_a;    /* [n_pairs] lower index of the pair */
  int32_t* pair_b;    /* [n_pairs] higher index */
} model_t;

static int model_init(model_t* md, int32_t N, int32_t M, const int32_t* ord,
                      const int32_t* nu) {
  memset(md, 0, sizeof *md);
  if (N < 1 || M < 1) return -1;
  md->N = N; md->M = M; md->ord = ord; md->nu = nu;
  md->order_tot = (int32_t*)calloc((size_t)M, sizeof(int32_t));
  md->is_reactant = (uint8_t*)calloc((size_t)N, 1);
  md->pair_of = (int32_t*)malloc((size_t)M * sizeof(int32_t));
  md->pair_a = (int32_t*)malloc((size_t)M * sizeof(int32_t));
  md->pair_b = (int32_t*)malloc((size_t)M * sizeof(int32_t));
  if (!md->order_tot || !md->is_reactant || !md->pair_of || !md->pair_a || !md->pair_b)
    return -1;
  for (int32_t j = 0; j < M; ++j) {
    int32_t tot = 0;
    for (int32_t s = 0; s < N; ++s) {
      int32_t m = ord[j * N + s];
      if (m < 0 || nu[j * N + s] < -m) return -1;
      tot += m;
      if (m > 0) md->is_reactant[s] = 1;
    }
    if (tot > 3) return -1;
    md->order_tot[j] = tot;
  }
  /* Reversible pairs: reaction k is the chemical reverse of reaction j (the reactants
   * of k are the products m_j + nu_j of j and the products of k are the reactants of
   * j, so nu_k = -nu_j), nu_j is not zero, and both reactions have at least one reactant
   * (a zero-order source has no chemical reverse).  Scanned in index order, each
   * reaction in at most one pair, the partner the lowest unpaired index. */
  for (int32_t j = 0; j < M; ++j) md->pair_of[j] = -1;
  for (int32_t j = 0; j < M; ++j) {
    if (md->pair_of[j] >= 0 || md->order_tot[j] == 0) continue;
    int nonzero = 0;
    for (int32_t s = 0; s < N; ++s) nonzero |= nu[j * N + s] != 0;
    if (!nonzero) continue;
    for (int32_t k = j + 1; k < M; ++k) {
      if (md->pair_of[k] >= 0 || md->order_tot[k] == 0) continue;
      int opposite = 1;
      for (int32_t s = 0; s < N; ++s) {
        opposite &= ord[k * N + s] == ord[j * N + s] + nu[j * N + s];
        opposite &= ord[j * N + s] == ord[k * N + s] + nu[k * N + s];
      }
      if (opposite) {
        md->pair_of[j] = k;
        md->pair_of[k] = j;
        md->pair_a[md->n_pairs] = j;
        md->pair_b[md->n_pairs] = k;
        md->n_pairs++;
        break;
      }
    }
  }
  return 0;
}

static void model_free(model_t* md) {
  free(md->order_tot); free(md->is_reactant); free(md->pair_of);
  free(md->pair_a); free(md->pair_b);
}

/* Binomial coefficient factor C(v, m) for m = 1, 2, 3 evaluated on a real argument,
 * in this operation order. */
static double comb_factor(double v, int32_t m) {
  if (m == 1) return v;
  if (m == 2) return (v * (v - 1.0)) * 0.5;
  return ((v * (v - 1.0)) * (v - 2.0)) / 6.0;
}

/* g_j at an integer state: 0 when some x_s < m_js, else the product over reactant
 * species in increasing s of C(x_s, m_js). */
static double g_int(const model_t* md, int32_t j, const int64_t* x) {
  double v = 1.0;
  for (int32_t s = 0; s < md->N; ++s) {
    int32_t m = md->ord[j * md->N + s];
    if (m == 0) continue;
    if (x[s] < m) return 0.0;
    v = v * comb_factor((double)x[s], m);
  }
  return v;
}

/* d/dv C(v, m) for m = 1, 2, 3: 1, v - 1/2, (3 v^2 - 6 v + 2) / 6, in this order. */
static double comb_factor_deriv(double v, int32_t m) {
  if (m == 1) return 1.0;
  if (m == 2) return v - 0.5;
  return ((3.0 * (v * v) - 6.0 * v) + 2.0) / 6.0;
}

/* g_j at a real state (implicit solve): the same polynomial without the clamp. */
static double g_real(const model_t* md, int32_t j, const double* y) {
  double v = 1.0;
  for (int32_t s = 0; s < md->N; ++s) {
    int32_t m = md->ord[j * md->N + s];
    if (m == 0) continue;
    v = v * comb_factor(y[s], m);
  }
  return v;
}

/* Exact partial derivative of g_j with respect to y_q: the product in increasing s with
 * the factor of species q replaced by its derivative (0 if q is not a reactant). */
static double g_real_deriv(const model_t* md, int32_t j, const double* y, int32_t q) {
  if (md->ord[j * md->N + q] == 0) return 0.0;
  double v = 1.0;
  for (int32_t s = 0; s < md->N; ++s) {
    int32_t m = md->ord[j * md->N + s];
    if (m == 0) continue;
    v = v * (s == q ? comb_factor_deriv(y[s], m) : comb_factor(y[s], m));
  }
  return v;
}

/* Highest-order-reaction factor of Cao 2006 for species s at count x: the maximum over
 * reactions j consuming s of 1 (order 1); 2 or 2 + 1/(x-1) (order 2, one or two
 * molecules of s); 3, 1.5 (2 + 1/(x-1)) or 3 + 1/(x-1) + 2/(x-2) (order 3, one, two or
 * three molecules of s).  Fractional terms are dropped while x < m. */
static double hor_factor(const model_t* md, int32_t s, int64_t x) {
  double h = 0.0, xd = (double)x;
  for (int32_t j = 0; j < md->M; ++j) {
    int32_t m = md->ord[j * md->N + s];
    if (m == 0) continue;
    int32_t o = md->order_tot[j];
    double v;
    if (o == 1) v = 1.0;
    else if (o == 2) v = (m == 1) ? 2.0 : (x >= 2 ? 2.0 + 1.0 / (xd - 1.0) : 2.0);
    else if (m == 1) v = 3.0;
    else if (m == 2) v = x >= 2 ? 1.5 * (2.0 + 1.0 / (xd - 1.0)) : 3.0;
    else v = x >= 3 ? (3.0 + 1.0 / (xd - 1.0)) + 2.0 / (xd - 2.0) : 3.0;
    if (v > h) h = v;
  }
  return h;
}

/* Cao 2006 step size over the reactions with use[j] != 0:
 *   mu_s = sum_j nu_js a_j, sigma2_s = sum_j nu_js^2 a_j   (sequential, increasing j,
 *   nonzero nu_js only), for every species that is a reactant of some reaction;
 *   bound_s = max(eps x_s / h_s, 1);
 *   tau = min_s min(bound_s / |mu_s|, bound_s^2 / sigma2_s)   (+inf if none bounds). */
static double tau_select_md(const model_t* md, const double* a, const int64_t* x,
                            const uint8_t* use, double eps) {
  double tau = INFINITY;
  for (int32_t s = 0; s < md->N; ++s) {
    if (!md->is_reactant[s]) continue;
    double mu = 0.0, var = 0.0;
    for (int32_t j = 0; j < md->M; ++j) {
      int32_t v = md->nu[j * md->N + s];
      if (!use[j] || v == 0) continue;
      mu = mu + (double)v * a[j];
      var = var + (double)(v * v) * a[j];
    }
    double h = hor_factor(md, s, x[s]);
    double bound = (eps * (double)x[s]) / h;
    if (bound < 1.0) bound = 1.0;
    double t1 = bound / fabs(mu);
    double t2 = (bound * bound) / var;
    double ts = t1 < t2 ? t1 : t2;
    if (ts < tau) tau = ts;
  }
  return tau;
}

double mlo_tau_select(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                      const double* a, const int64_t* x, const uint8_t* use, double eps) {
  model_t md;
  if (model_init(&md, N, M, orders, stoich) != 0) {
    model_free(&md);
    return NAN;
  }
  double t = tau_select_md(&md, a, x, use, eps);
  model_free(&md);
  return t;
}

/* ------------------------------------------------------------------------------------
 * Implicit leap (Rathinam, Petzold & Cao 2003; Cao 2007): given Poisson draws P_j with
 * means a_j(x) tau for the non-critical reactions, solve for the real state y
 *   y = c + tau sum_j nu_j a_j(y),   c = x + sum_j nu_j (P_j - a_j(x) tau)
 * by Newton's method with a forward-difference Jacobian of the propensities (the
 * paper's "estimated numerically", Section 1) or, on request, the exact derivative of
 * the mass-action polynomials (the paper's symbolic Jacobian, Section 3):
 *   F(y) = (y - c) - tau sum_j nu_j a_j(y),
 *   J[s][q] = [s == q] - tau sum_j nu_js D_jq,  D_jq = (a_j(y + h e_q) - a_j(y)) / h,
 *   h = ((y_q + fd_h max(1,|y_q|)) - y_q);
 * solve J d = -F by Gaussian elimination with partial pivoting (largest |pivot|, the
 * lowest row on ties) and column-oriented back substitution; y += d; stop when
 * |d|_inf <= tol max(1, |y|_inf).  Sums over j are sequential in increasing j over
 * nonzero nu_js.  Returns 0 on convergence, 1 when not converged, 2 when singular.
 * ---------------------------------------------------------------------------------- */
static int implicit_solve_md(const model_t* md, const double* th, const int64_t* x,
                             const uint8_t* nc, const double* P, const double* a_x,
                             double tau, const mlo_params* p, double* y, int32_t* iters) {
  const int32_t N = md->N, M = md->M;
  double* c = (double*)malloc(sizeof(double) * (size_t)N);
  double* F = (double*)malloc(sizeof(double) * (size_t)N);
  double* ay = (double*)malloc(sizeof(double) * (size_t)M);
  double* D = (double*)malloc(sizeof(double) * (size_t)M * (size_t)N);
  double* A = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
  double* b = (double*)malloc(sizeof(double) * (size_t)N);
  double* yq = (double*)malloc(sizeof(double) * (size_t)N);
  int rc = 1;
  *iters = 0;
  for (int32_t s = 0; s < N; ++s) {
    double acc = (double)x[s];
    for (int32_t j = 0; j < M; ++j) {
      int32_t v = md->nu[j * N + s];
      if (!nc[j] || v == 0) continue;
      acc = acc + (double)v * (P[j] - a_x[j] * tau);
    }
    c[s] = acc;
    y[s] = (double)x[s];
  }
  for (int32_t it = 0; it < p->newton_maxit; ++it) {
    *iters = it + 1;
    for (int32_t j = 0; j < M; ++j) ay[j] = th[j] * g_real(md, j, y);
    for (int32_t s = 0; s < N; ++s) {
      double acc = 0.0;
      for (int32_t j = 0; j < M; ++j) {
        int32_t v = md->nu[j * N + s];
        if (!nc[j] || v == 0) continue;
        acc = acc + (double)v * ay[j];
      }
      F[s] = (y[s] - c[s]) - tau * acc;
    }
    /* D_jq = d a_j / d y_q: exact, or forward differences one species at a time */
    if (p->jacobian == MLO_JAC_ANALYTIC) {
      for (int32_t q = 0; q < N; ++q)
        for (int32_t j = 0; j < M; ++j)
          D[j * N + q] = (nc[j] && md->ord[j * N + q] != 0)
                             ? th[j] * g_real_deriv(md, j, y, q)
                             : 0.0;
    }
    for (int32_t q = 0; q < N && p->jacobian != MLO_JAC_ANALYTIC; ++q) {
      double aq = fabs(y[q]);
      double h = p->fd_h * (aq > 1.0 ? aq : 1.0);
      for (int32_t s = 0; s < N; ++s) yq[s] = y[s];
      yq[q] = y[q] + h;
      double he = yq[q] - y[q];
      for (int32_t j = 0; j < M; ++j) {
        if (!nc[j] || md->ord[j * N + q] == 0) {
          D[j * N + q] = 0.0;
          continue;
        }
        D[j * N + q] = (th[j] * g_real(md, j, yq) - ay[j]) / he;
      }
    }
    for (int32_t s = 0; s < N; ++s) {
      for (int32_t q = 0; q < N; ++q) {
        double acc = 0.0;
        for (int32_t j = 0; j < M; ++j) {
          int32_t v = md->nu[j * N + s];
          if (!nc[j] || v == 0 || md->ord[j * N + q] == 0) continue;
          acc = acc + (double)v * D[j * N + q];
        }
        A[s * N + q] = (s == q ? 1.0 : 0.0) - tau * acc;
      }
      b[s] = -F[s];
    }
    /* Gaussian elimination with partial pivoting */
    int singular = 0;
    for (int32_t k = 0; k < N; ++k) {
      int32_t piv = k;
      double best = fabs(A[k * N + k]);
      for (int32_t i = k + 1; i < N; ++i) {
        if (fabs(A[i * N + k]) > best) {
          best = fabs(A[i * N + k]);
          piv = i;
        }
      }
      if (best == 0.0) {
        singular = 1;
        break;
      }
      if (piv != k) {
        for (int32_t cc = 0; cc < N; ++cc) {
          double tmp = A[k * N + cc];
          A[k * N + cc] = A[piv * N + cc];
          A[piv * N + cc] = tmp;
        }
        double tb = b[k]; b[k] = b[piv]; b[piv] = tb;
      }
      for (int32_t i = k + 1; i < N; ++i) {
        double l = A[i * N + k] / A[k * N + k];
        for (int32_t cc = k + 1; cc < N; ++cc) A[i * N + cc] = A[i * N + cc] - l * A[k * N + cc];
        b[i] = b[i] - l * b[k];
      }
    }
    if (singular) {
      rc = 2;
      break;
    }
    /* column-oriented back substitution: d_i = b_i / A_ii, then b_r -= A_ri d_i, r < i */
    double dmax = 0.0, ymax = 0.0;
    for (int32_t i = N - 1; i >= 0; --i) {
      double d = b[i] / A[i * N + i];
      F[i] = d; /* reuse F as the update vector */
      for (int32_t r = 0; r < i; ++r) b[r] = b[r] - A[r * N + i] * d;
    }
    for (int32_t s = 0; s < N; ++s) {
      y[s] = y[s] + F[s];
      if (fabs(F[s]) > dmax) dmax = fabs(F[s]);
      if (fabs(y[s]) > ymax) ymax = fabs(y[s]);
    }
    if (dmax <= p->newton_tol * (ymax > 1.0 ? ymax : 1.0)) {
      rc = 0;
      break;
    }
  }
  free(c); free(F); free(ay); free(D); free(A); free(b); free(yq);
  return rc;
}

int mlo_implicit_solve(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                       const double* theta, const int64_t* x, const uint8_t* nc,
                       const double* P, const double* a_x, double tau, const mlo_params* p,
                       double* y_out, int32_t* iters_out) {
  model_t md;
  if (model_init(&md, N, M, orders, stoich) != 0) {
    model_free(&md);
    return -1;
  }
  int rc = implicit_solve_md(&md, theta, x, nc, P, a_x, tau, p, y_out, iters_out);
  model_free(&md);
  return rc;
}

/* ------------------------------------------------------------------------------------
 * The decisions of one outer step (Section 2), one function each.  The trajectory loop
 * below calls exactly these, and they are exported so that tests pin each one on
 * hand-computed states.
 * ---------------------------------------------------------------------------------- */

/* Critical reactions (Section 2: a reaction fewer than n_c firings away from exhausting
 * one of its reactants fires at most once per leap).  L_j = min over the species that
 * reaction j consumes (nu_js < 0; a catalyst, with nu_js = 0, is not consumed) of
 * floor(x_s / |nu_js|); j is critical iff a_j > 0 and L_j < n_c (a reaction that
 * consumes nothing is never critical).  crit[j] = 1 for a critical reaction, else 0;
 * ac[j] = a_j for a critical reaction, else 0.  Returns a0c, the lane-tree sum of ac. */
static double critical_set_md(const model_t* md, const double* a, const int64_t* x,
                              int32_t n_c, uint8_t* crit, double* ac) {
  const int32_t N = md->N, M = md->M;
  for (int32_t j = 0; j < M; ++j) {
    int c = 0;
    if (a[j] > 0.0) {
      int64_t L = -1;
      for (int32_t s = 0; s < N; ++s) {
        int32_t v = md->nu[j * N + s];
        if (v >= 0) continue;
        int64_t l = x[s] / (int64_t)(-v);
        if (L < 0 || l < L) L = l;
      }
      c = (L >= 0 && L < (int64_t)n_c);
    }
    crit[j] = (uint8_t)c;
    ac[j] = c ? a[j] : 0.0;
  }
  return mlo_lane_tree_sum(ac, M);
}

double mlo_critical_set(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                        const double* a, const int64_t* x, int32_t n_c, uint8_t* crit_out,
                        double* ac_out) {
  model_t md;
  if (model_init(&md, N, M, orders, stoich) != 0) {
    model_free(&md);
    return NAN;
  }
  double a0c = critical_set_md(&md, a, x, n_c, crit_out, ac_out);
  model_free(&md);
  return a0c;
}

/* Inverse-CDF choice of one reaction (Gillespie 1977 direct method; also the critical
 * pick): the first j, in index order, whose sequential prefix sum w_0 + ... + w_j exceeds
 * target; when rounding leaves none, the last j with w_j > 0; -1 when no weight is
 * positive. */
int32_t mlo_pick(int32_t M, const double* w, double target) {
  double acc = 0.0;
  int32_t last = -1;
  for (int32_t j = 0; j < M; ++j) {
    if (w[j] > 0.0) last = j;
    acc = acc + w[j];
    if (target < acc) return j;
  }
  return last;
}

/* The paper's switch to exact SSA (Section 2), folded with Cao's rule that a leap of
 * fewer than ssa_factor mean inter-reaction waits is not worth taking: 1 iff
 * min(tau1, tau2) < ssa_factor / a0, where tau2 is the drawn wait to the next critical
 * firing (+inf without critical reactions). */
int mlo_ssa_switch(double tau1, double tau2, double a0, double ssa_factor) {
  double tmin = tau1 < tau2 ? tau1 : tau2;
  return tmin < ssa_factor / a0;
}

/* Firings of one non-critical reaction in an implicit leap (Rathinam 2003): the real
 * solution y gives a_j(y) tau + P_j - a_j(x) tau, rounded half away from zero and clamped
 * at 0 (this project's reading: the clamp keeps r >= 0 and X = x0 + nu^T r exact). */
int64_t mlo_implicit_count(double a_y, double tau, double P, double a_x) {
  double v = (a_y * tau + P) - a_x * tau;
  double rv = round(v);
  if (!(rv < 0x1p62)) return MLO_COUNT_LIMIT; /* beyond any leap limit (also NaN) */
  return rv > 0.0 ? (int64_t)rv : 0;
}

/* The count limits above: 1 when a count or a firing total exceeds MLO_COUNT_LIMIT. */
static int counts_beyond_limit(const int64_t* x, int32_t N, const int64_t* r, int32_t M) {
  for (int32_t s = 0; s < N; ++s)
    if (x[s] > MLO_COUNT_LIMIT) return 1;
  for (int32_t j = 0; j < M; ++j)
    if (r[j] > MLO_COUNT_LIMIT) return 1;
  return 0;
}

/* One implicit leap: solve for y (implicit_solve_md), then K[j] = mlo_implicit_count for
 * every non-critical j (K of critical reactions untouched).  Returns the solve's code. */
static int implicit_leap_md(const model_t* md, const double* th, const int64_t* x,
                            const uint8_t* nc, const double* P, const double* a_x, double tau,
                            const mlo_params* p, double* y, int64_t* K, int32_t* iters) {
  int rc = implicit_solve_md(md, th, x, nc, P, a_x, tau, p, y, iters);
  if (rc != 0) return rc;
  for (int32_t j = 0; j < md->M; ++j)
    if (nc[j]) K[j] = mlo_implicit_count(th[j] * g_real(md, j, y), tau, P[j], a_x[j]);
  return 0;
}

int mlo_implicit_leap(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                      const double* theta, const int64_t* x, const uint8_t* nc,
                      const double* P, const double* a_x, double tau, const mlo_params* p,
                      int64_t* K_out, int32_t* iters_out) {
  model_t md;
  if (model_init(&md, N, M, orders, stoich) != 0) {
    model_free(&md);
    return -1;
  }
  double* y = (double*)malloc(sizeof(double) * (size_t)N);
  int rc = implicit_leap_md(&md, theta, x, nc, P, a_x, tau, p, y, K_out, iters_out);
  free(y);
  model_free(&md);
  return rc;
}

/* ------------------------------------------------------------------------------------
 * Parameters
 * ---------------------------------------------------------------------------------- */
void mlo_default_params(mlo_params* p) {
  p->eps = 0.03;
  p->n_c = 10;
  p->ssa_factor = 10.0;
  p->n_ssa_explicit = 100;
  p->n_ssa_implicit = 10;
  p->pe_delta = 0.05;
  p->stiff_ratio = 100.0;
  p->newton_tol = 1e-10;
  p->newton_maxit = 20;
  p->fd_h = 1e-7;
  p->max_steps = 100000000;
  p->max_reject = 64;
  p->mode = MLO_MODE_ADAPTIVE;
  p->jacobian = MLO_JAC_FD;
}

/* ------------------------------------------------------------------------------------
 * One trajectory.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  const model_t* md;
  const double* th;
  const mlo_params* p;
  uint64_t seed;
  uint32_t id;
  double T;
  int64_t* x;
  int64_t* r;
  double* G;
  double* g;
  double* a;
  double t;
  uint32_t status;
  int64_t cnt[4];
  /* observation grid: K nondecreasing times, the next unrecorded index kn, and this
   * trajectory's rows X_obs[k][s] */
  const double* tobs;
  int32_t K, kn;
  int64_t* xobs;
} traj_t;

/* Time-grid output.  The path X(t) is right-continuous and piecewise constant: it changes
 * only at SSA firing times and at the ends of leaps, so X(t_k) is the state after every
 * change at a time <= t_k.  record_obs writes the current state to every pending grid
 * point with t_k < tcut (strict) or t_k <= tcut (inclusive). */
static void record_obs(traj_t* tr, double tcut, int inclusive) {
  const int32_t N = tr->md->N;
  while (tr->kn < tr->K) {
    const double tk = tr->tobs[tr->kn];
    if (inclusive ? !(tk <= tcut) : !(tk < tcut)) break;
    for (int32_t s = 0; s < N; ++s) tr->xobs[(int64_t)tr->kn * N + s] = tr->x[s];
    tr->kn += 1;
  }
}

/* A leap may not pass the next grid point: it ends there exactly, as it does at T. */
static double next_stop(const traj_t* tr) {
  if (tr->kn < tr->K && tr->tobs[tr->kn] < tr->T) return tr->tobs[tr->kn];
  return tr->T;
}

static void eval_props(traj_t* tr) {
  for (int32_t j = 0; j < tr->md->M; ++j) {
    tr->g[j] = g_int(tr->md, j, tr->x);
    tr->a[j] = tr->th[j] * tr->g[j];
  }
}

/* SSA burst (Gillespie 1977 direct method) of at most n_max firings at outer step
 * `step`.  The state's g, a and a0 are current on entry.  Each firing: u1, u2 from block
 * b of stream M+2; dt = -log(u1)/a0; a step that would pass T integrates g to T and
 * stops; otherwise G += g dt (exact for a piecewise-constant state, Section 1), t += dt,
 * and reaction j fires, the first j whose sequential prefix sum of a exceeds u2 a0
 * (the last j with a_j > 0 if rounding leaves none). */
static void ssa_burst(traj_t* tr, uint32_t step, int32_t n_max, double a0) {
  const model_t* md = tr->md;
  const int32_t N = md->N, M = md->M;
  for (int32_t b = 0; b < n_max; ++b) {
    if (b > 0) {
      eval_props(tr);
      a0 = mlo_lane_tree_sum(tr->a, M);
    }
    if (a0 == 0.0) {
      double rem = tr->T - tr->t;
      for (int32_t j = 0; j < M; ++j) tr->G[j] = tr->G[j] + tr->g[j] * rem;
      tr->t = tr->T;
      return;
    }
    uint32_t w[4];
    block_words(tr->seed, tr->id, step, (uint32_t)M + 2u, (uint32_t)b, w);
    double u1 = mlo_u01_from_words(w[0], w[1]);
    double u2 = mlo_u01_from_words(w[2], w[3]);
    double dt = -mlo_log(u1) / a0;
    double tn = tr->t + dt;
    if (tn > tr->T) {
      double rem = tr->T - tr->t;
      for (int32_t j = 0; j < M; ++j) tr->G[j] = tr->G[j] + tr->g[j] * rem;
      tr->t = tr->T;
      return;
    }
    for (int32_t j = 0; j < M; ++j) tr->G[j] = tr->G[j] + tr->g[j] * dt;
    record_obs(tr, tn, 0); /* grid points before the firing see the old state */
    tr->t = tn;
    int32_t pick = mlo_pick(M, tr->a, u2 * a0);
    for (int32_t s = 0; s < N; ++s) tr->x[s] += md->nu[pick * N + s];
    tr->r[pick] += 1;
    tr->cnt[2] += 1;
    record_obs(tr, tr->t, 1); /* a grid point at the firing time sees the new state */
  }
}

static void simulate_one(traj_t* tr) {
  const model_t* md = tr->md;
  const mlo_params* p = tr->p;
  const int32_t N = md->N, M = md->M;
  double* ac = (double*)malloc(sizeof(double) * (size_t)M);
  double* gn = (double*)malloc(sizeof(double) * (size_t)M);
  double* Pd = (double*)malloc(sizeof(double) * (size_t)M);
  double* y = (double*)malloc(sizeof(double) * (size_t)N);
  uint8_t* nc = (uint8_t*)malloc((size_t)M);
  uint8_t* crit = (uint8_t*)malloc((size_t)M);
  uint8_t* use_im = (uint8_t*)malloc((size_t)M);
  uint8_t* pe_on = (uint8_t*)malloc((size_t)M);
  int64_t* K = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
  int64_t* xn = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  uint32_t step = 0;
  int32_t reject_run = 0;
  record_obs(tr, tr->t, 1); /* grid points at t = 0 see x0 */

  for (;;) {
    if (!(tr->t < tr->T)) break;
    if ((int64_t)step >= p->max_steps) {
      tr->status |= MLO_ST_STEP_LIMIT;
      break;
    }
    if (counts_beyond_limit(tr->x, N, tr->r, M)) {
      tr->status |= MLO_ST_OVERFLOW;
      break;
    }
    /* 1. propensities */
    eval_props(tr);
    double a0 = mlo_lane_tree_sum(tr->a, M);
    if (a0 == 0.0) {
      double rem = tr->T - tr->t;
      for (int32_t j = 0; j < M; ++j) tr->G[j] = tr->G[j] + tr->g[j] * rem;
      tr->t = tr->T;
      break;
    }
    if (p->mode == MLO_MODE_SSA_ONLY) {
      ssa_burst(tr, step, p->n_ssa_explicit, a0);
      step++;
      continue;
    }
    /* 2. critical reactions and a0c */
    double a0c = critical_set_md(md, tr->a, tr->x, p->n_c, crit, ac);
    for (int32_t j = 0; j < M; ++j) nc[j] = (uint8_t)!crit[j];
    /* 3. explicit step size */
    double tau_ex = tau_select_md(md, tr->a, tr->x, nc, p->eps);
    /* 4. partial equilibrium and the implicit step size */
    int implicit = 0;
    double tau1 = tau_ex;
    if (p->mode == MLO_MODE_ADAPTIVE && md->n_pairs > 0) {
      int any = 0;
      for (int32_t j = 0; j < M; ++j) pe_on[j] = 0;
      for (int32_t q = 0; q < md->n_pairs; ++q) {
        int32_t j = md->pair_a[q], k = md->pair_b[q];
        if (!nc[j] || !nc[k]) continue;
        double lo = tr->a[j] < tr->a[k] ? tr->a[j] : tr->a[k];
        if (fabs(tr->a[j] - tr->a[k]) <= p->pe_delta * lo) {
          pe_on[j] = pe_on[k] = 1;
          any = 1;
        }
      }
      if (any) {
        for (int32_t j = 0; j < M; ++j) use_im[j] = (uint8_t)(nc[j] && !pe_on[j]);
        double tau_im = tau_select_md(md, tr->a, tr->x, use_im, p->eps);
        if (tau_im > p->stiff_ratio * tau_ex) {
          implicit = 1;
          tau1 = tau_im;
        }
      }
    }
    /* 5.-7. attempt loop: draw tau2, SSA switch, leap, negativity check */
    int overflow = 0;
    for (;;) {
      if (reject_run >= p->max_reject) {
        tr->status |= MLO_ST_REJECT_LIMIT;
        ssa_burst(tr, step, p->n_ssa_explicit, a0);
        step++;
        reject_run = 0;
        break;
      }
      double tau2 = INFINITY;
      if (a0c > 0.0) {
        uint32_t w[4];
        block_words(tr->seed, tr->id, step, (uint32_t)M, 0u, w);
        tau2 = -mlo_log(mlo_u01_from_words(w[0], w[1])) / a0c;
      }
      if (mlo_ssa_switch(tau1, tau2, a0, p->ssa_factor)) {
        ssa_burst(tr, step, implicit ? p->n_ssa_implicit : p->n_ssa_explicit, a0);
        step++;
        reject_run = 0;
        break;
      }
      const double stop = next_stop(tr);
      double rem = stop - tr->t;
      double tau = tau1;
      if (tau2 < tau) tau = tau2;
      int at_horizon = 0;
      if (rem <= tau) {
        tau = rem;
        at_horizon = 1;
      }
      int crit_fire = (tau2 <= tau1) && (tau2 <= rem);
      for (int32_t j = 0; j < M; ++j)
        if (nc[j] && tr->a[j] * tau > MLO_LEAP_LIMIT) overflow = 1;
      if (overflow) break;
      for (int32_t j = 0; j < M; ++j) K[j] = 0;
      if (crit_fire) {
        uint32_t w[4];
        block_words(tr->seed, tr->id, step, (uint32_t)M + 1u, 0u, w);
        K[mlo_pick(M, ac, mlo_u01_from_words(w[0], w[1]) * a0c)] = 1;
      }
      int implicit_step = implicit && tau > tau_ex;
      if (implicit_step) {
        for (int32_t j = 0; j < M; ++j)
          Pd[j] = nc[j] ? (double)mlo_poisson(tr->a[j] * tau, tr->seed, tr->id, step,
                                              (uint32_t)j, &tr->status)
                        : 0.0;
        int32_t its;
        if (implicit_leap_md(md, tr->th, tr->x, nc, Pd, tr->a, tau, p, y, K, &its) != 0) {
          tr->status |= MLO_ST_NEWTON_FAIL;
          implicit = 0;
          tau1 = tau_ex;
          step++;
          continue;
        }
        for (int32_t j = 0; j < M; ++j)
          if (nc[j] && (double)K[j] > MLO_LEAP_LIMIT) overflow = 1;
        if (overflow) break;
      } else {
        for (int32_t j = 0; j < M; ++j)
          if (nc[j])
            K[j] = mlo_poisson(tr->a[j] * tau, tr->seed, tr->id, step, (uint32_t)j,
                               &tr->status);
      }
      int negative = 0;
      for (int32_t s = 0; s < N; ++s) {
        int64_t v = tr->x[s];
        for (int32_t j = 0; j < M; ++j) v += (int64_t)md->nu[j * N + s] * K[j];
        xn[s] = v;
        if (v < 0) negative = 1;
      }
      if (negative) {
        tau1 = tau1 * 0.5;
        step++;
        reject_run++;
        tr->cnt[3] += 1;
        continue;
      }
      for (int32_t j = 0; j < M; ++j) gn[j] = g_int(md, j, xn);
      double half = tau * 0.5;
      for (int32_t j = 0; j < M; ++j) {
        tr->r[j] += K[j];
        tr->G[j] = tr->G[j] + half * (tr->g[j] + gn[j]);
      }
      for (int32_t s = 0; s < N; ++s) tr->x[s] = xn[s];
      tr->t = at_horizon ? stop : tr->t + tau;
      record_obs(tr, tr->t, 1);
      tr->cnt[implicit_step ? 1 : 0] += 1;
      step++;
      reject_run = 0;
      break;
    }
    if (overflow) {
      tr->status |= MLO_ST_OVERFLOW;
      break;
    }
  }
  /* grid points after the end (beyond T, or after a step-limit stop) see the final state */
  record_obs(tr, INFINITY, 1);
  free(ac); free(gn); free(Pd); free(y); free(nc); free(crit); free(use_im); free(pe_on);
  free(K); free(xn);
}

int mlo_simulate_grid(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                      const double* rates, int64_t n_traj, const double* theta,
                      const int64_t* x0, int32_t x0_per_traj, const double* T,
                      int32_t T_per_traj, const mlo_params* p, uint64_t seed,
                      uint64_t traj_id_base, const double* t_obs, int32_t K, int64_t* X_obs,
                      int64_t* X_out, int64_t* r_out, double* G_out, uint32_t* status_out,
                      int64_t* counters_out) {
  model_t md;
  if (n_traj < 0 || !p || !x0 || !T || (!theta && !rates)) return -1;
  if (K < 0 || (K > 0 && (!t_obs || !X_obs))) return -1;
  for (int32_t k = 0; k < K; ++k) /* finite, >= 0, nondecreasing */
    if (!(t_obs[k] >= 0.0) || !(t_obs[k] <= 1.0e300) || (k > 0 && t_obs[k] < t_obs[k - 1]))
      return -1;
  if (traj_id_base + (uint64_t)n_traj > 0x100000000ULL) return -1;
  if (model_init(&md, N, M, orders, stoich) != 0) {
    model_free(&md);
    return -1;
  }
  double* g = (double*)malloc(sizeof(double) * (size_t)M);
  double* a = (double*)malloc(sizeof(double) * (size_t)M);
  for (int64_t i = 0; i < n_traj; ++i) {
    traj_t tr;
    memset(&tr, 0, sizeof tr);
    tr.md = &md;
    tr.th = theta ? theta + i * M : rates;
    tr.p = p;
    tr.seed = seed;
    tr.id = (uint32_t)(traj_id_base + (uint64_t)i);
    tr.T = T_per_traj ? T[i] : T[0];
    tr.x = X_out + i * N;
    tr.r = r_out + i * M;
    tr.G = G_out + i * M;
    tr.g = g;
    tr.a = a;
    const int64_t* xi = x0_per_traj ? x0 + i * N : x0;
    for (int32_t s = 0; s < N; ++s) tr.x[s] = xi[s];
    for (int32_t j = 0; j < M; ++j) {
      tr.r[j] = 0;
      tr.G[j] = 0.0;
    }
    tr.t = 0.0;
    tr.tobs = t_obs;
    tr.K = K;
    tr.kn = 0;
    tr.xobs = K > 0 ? X_obs + i * (int64_t)K * N : NULL;
    simulate_one(&tr);
    status_out[i] = tr.status;
    if (counters_out)
      for (int c = 0; c < 4; ++c) counters_out[i * 4 + c] = tr.cnt[c];
  }
  free(g);
  free(a);
  model_free(&md);
  return 0;
}

int mlo_simulate(int32_t N, int32_t M, const int32_t* orders, const int32_t* stoich,
                 const double* rates, int64_t n_traj, const double* theta,
                 const int64_t* x0, int32_t x0_per_traj, const double* T,
                 int32_t T_per_traj, const mlo_params* p, uint64_t seed,
                 uint64_t traj_id_base, int64_t* X_out, int64_t* r_out, double* G_out,
                 uint32_t* status_out, int64_t* counters_out) {
  return mlo_simulate_grid(N, M, orders, stoich, rates, n_traj, theta, x0, x0_per_traj, T,
                           T_per_traj, p, seed, traj_id_base, NULL, 0, NULL, X_out, r_out,
                           G_out, status_out, counters_out);
}

/* ------------------------------------------------------------------------------------
 * Accuracy metric (Section 3): the Kullback-Leibler divergence of a method's marginal
 * distributions from those of exact SSA, averaged over all time points and species.
 * The paper does not say how the empirical distributions are formed; this reading bins
 * the integer counts of both samples on their pooled range [lo, hi] with integer width
 * w = ceil((hi - lo + 1) / max_bins) (one count per bin while the range fits), adds 1/2
 * to every bin of both histograms so that the divergence is finite, and computes
 *   KL(p || q) = sum_b p_b (log p_b - log q_b),
 *   p_b = (c_ref,b + 1/2) / (n_ref + nbins/2),  q_b = (c_test,b + 1/2) / (n_test + nbins/2),
 * with p the exact-SSA (reference) sample.  The sum over bins and the mean over the K x N
 * (time point, species) pairs take the canonical lane-tree order.
 * ---------------------------------------------------------------------------------- */
double mlo_kl_sample(int64_t n_ref, const int64_t* a, int64_t sa, int64_t n_test,
                     const int64_t* b, int64_t sb, int32_t max_bins) {
  int64_t lo = a[0], hi = a[0];
  for (int64_t i = 0; i < n_ref; ++i) {
    if (a[i * sa] < lo) lo = a[i * sa];
    if (a[i * sa] > hi) hi = a[i * sa];
  }
  for (int64_t i = 0; i < n_test; ++i) {
    if (b[i * sb] < lo) lo = b[i * sb];
    if (b[i * sb] > hi) hi = b[i * sb];
  }
  const int64_t span = hi - lo + 1;
  const int64_t w = (span + max_bins - 1) / max_bins;
  const int64_t nbins = (hi - lo) / w + 1;
  int64_t* ca = (int64_t*)calloc((size_t)nbins, sizeof(int64_t));
  int64_t* cb = (int64_t*)calloc((size_t)nbins, sizeof(int64_t));
  double* term = (double*)malloc(sizeof(double) * (size_t)nbins);
  for (int64_t i = 0; i < n_ref; ++i) ca[(a[i * sa] - lo) / w] += 1;
  for (int64_t i = 0; i < n_test; ++i) cb[(b[i * sb] - lo) / w] += 1;
  const double da = (double)n_ref + 0.5 * (double)nbins;
  const double db = (double)n_test + 0.5 * (double)nbins;
  for (int64_t k = 0; k < nbins; ++k) {
    const double pk = ((double)ca[k] + 0.5) / da;
    const double qk = ((double)cb[k] + 0.5) / db;
    term[k] = pk * (mlo_log(pk) - mlo_log(qk));
  }
  const double kl = mlo_lane_tree_sum(term, (int32_t)nbins);
  free(ca);
  free(cb);
  free(term);
  return kl;
}

int mlo_kl_grid(int64_t n_ref, const int64_t* X_ref, int64_t n_test, const int64_t* X_test,
                int32_t K, int32_t N, int32_t max_bins, double* kl_out, double* kl_mean) {
  if (n_ref < 1 || n_test < 1 || K < 1 || N < 1 || max_bins < 1 || !X_ref || !X_test ||
      !kl_out)
    return -1;
  const int64_t stride = (int64_t)K * N; /* layout [n][K][N] */
  for (int32_t k = 0; k < K; ++k)
    for (int32_t s = 0; s < N; ++s)
      kl_out[k * N + s] = mlo_kl_sample(n_ref, X_ref + k * N + s, stride, n_test,
                                        X_test + k * N + s, stride, max_bins);
  if (kl_mean) *kl_mean = mlo_lane_tree_sum(kl_out, K * N) / (double)(K * N);
  return 0;
}


/* ------------------------------------------------------------------------------------
 * Bayesian step.  The conjugate posterior of each rate constant given one path's
 * statistics is Gamma(alpha_j + r_j, beta_j + G_j) (Section 1).
 * ---------------------------------------------------------------------------------- */
#define GAMMA_MAX_TRIALS 64

double mlo_gamma(double shape, double rate, uint64_t seed, uint32_t traj_id, uint32_t stream,
                 uint32_t* status) {
  if (!(shape > 0.0) || !(rate > 0.0)) return NAN;
  const int boost = shape < 1.0;
  const double a = boost ? shape + 1.0 : shape;
  const double d = a - 1.0 / 3.0;
  const double c = 1.0 / sqrt(9.0 * d);
  const uint32_t ctr_step = 0x80000000u + stream;
  for (uint32_t t = 0; t < GAMMA_MAX_TRIALS; ++t) {
    uint32_t w[4], w2[4];
    block_words(seed, traj_id, ctr_step, 0u, 2u * t, w);
    /* Marsaglia polar method: (v1, v2) uniform in the square, accepted inside the disk */
    const double v1 = 2.0 * mlo_u01_from_words(w[0], w[1]) - 1.0;
    const double v2 = 2.0 * mlo_u01_from_words(w[2], w[3]) - 1.0;
    const double s = v1 * v1 + v2 * v2;
    if (!(s < 1.0) || s == 0.0) continue;
    const double z = v1 * sqrt((-2.0 * mlo_log(s)) / s);
    const double base = 1.0 + c * z;
    if (!(base > 0.0)) continue;
    const double v = (base * base) * base;
    block_words(seed, traj_id, ctr_step, 0u, 2u * t + 1u, w2);
    const double u = mlo_u01_from_words(w2[0], w2[1]);
    /* accept iff log u < z^2/2 + d - d v + d log v */
    if (mlo_log(u) < ((0.5 * (z * z) + d) - d * v) + d * mlo_log(v)) {
      double x = d * v;
      if (boost) {
        const double ub = mlo_u01_from_words(w2[2], w2[3]);
        x = x * mlo_exp(mlo_log(ub) / shape);
      }
      return x / rate;
    }
  }
  if (status) *status |= 1u;
  return shape / rate; /* the mean, after GAMMA_MAX_TRIALS rejections (never observed) */
}

int mlo_posterior_sample(int64_t n, int32_t M, const double* alpha, int32_t alpha_per_traj,
                         const double* beta, int32_t beta_per_traj, const int64_t* r,
                         const double* G, uint64_t seed, uint64_t traj_id_base,
                         double* theta_out, uint32_t* status_out) {
  if (n < 0 || M < 1 || !alpha || !beta || !r || !G || !theta_out) return -1;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t st = 0;
    const uint32_t id = (uint32_t)(traj_id_base + (uint64_t)i);
    for (int32_t j = 0; j < M; ++j) {
      const double al = alpha_per_traj ? alpha[i * M + j] : alpha[j];
      const double be = beta_per_traj ? beta[i * M + j] : beta[j];
      theta_out[i * M + j] = mlo_gamma(al + (double)r[i * M + j], be + G[i * M + j], seed, id,
                                       (uint32_t)j, &st);
    }
    if (status_out) status_out[i] = st;
  }
  return 0;
}

int mlo_resample_systematic(int64_t n, const double* logw, uint64_t seed, uint64_t id_base,
                            int64_t* ancestors) {
  if (n < 1 || !logw || !ancestors) return -1;
  double mx = -INFINITY;
  for (int64_t i = 0; i < n; ++i)
    if (logw[i] > mx) mx = logw[i]; /* NaN never compares greater: weight 0 */
  if (mx == -INFINITY || mx == INFINITY) {
    for (int64_t k = 0; k < n; ++k) ancestors[k] = -1;
    return -1;
  }
  uint64_t* q = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  unsigned __int128 total = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double wgt = logw[i] == logw[i] ? mlo_exp(logw[i] - mx) : 0.0; /* in [0, 1] */
    q[i] = (uint64_t)floor(wgt * 1099511627776.0); /* 2^40 */
    total += q[i];
  }
  if (total == 0) {
    for (int64_t k = 0; k < n; ++k) ancestors[k] = -1;
    free(q);
    return -1;
  }
  uint32_t w[4];
  block_words(seed, (uint32_t)id_base, 0xC0000000u, 0u, 0u, w);
  const double u = mlo_u01_from_words(w[0], w[1]);
  const unsigned __int128 uQ = (unsigned __int128)floor(u * (double)(uint64_t)total);
  /* ancestor k: first i whose inclusive prefix exceeds target_k = (k Q + uQ) / n */
  unsigned __int128 prefix = 0;
  int64_t i = 0;
  for (int64_t k = 0; k < n; ++k) {
    const unsigned __int128 target = ((unsigned __int128)k * total + uQ) / (unsigned __int128)n;
    while (i < n && prefix + q[i] <= target) {
      prefix += q[i];
      ++i;
    }
    ancestors[k] = i < n ? i : n - 1;
  }
  free(q);
  return 0;
}
