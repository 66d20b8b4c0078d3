/*
 * matleap.h -- C ABI of the GB300 (sm_103a) ensemble simulator for adaptive
 * explicit-implicit tau-leaping of mass-action chemical reaction networks
 * (matLeap, Feigelman, Ganscha & Claassen, arXiv:1608.07058).
 *
 * What one trajectory computes (paper, Section 1 "Background" and Section 2
 * "Implementation"): starting from x0 at t = 0 it advances the network to the horizon T
 * by the adaptive method -- Cao-Gillespie-Petzold (2006) epsilon-bounded leaps,
 * critical reactions (fewer than n_c firings from exhaustion fire at most once per
 * leap), implicit leaps (Rathinam-Petzold-Cao 2003) when leaving out reaction pairs in
 * partial equilibrium gives a much longer leap (Cao-Gillespie-Petzold 2007), and the
 * paper's switch to exact SSA bursts when the wait to the next critical firing, or the
 * leap itself, is comparable to the wait to the next reaction -- and returns
 *   X(T)  the final state,
 *   r_j   the number of firings of reaction j,
 *   G_j   the integral over [0, T] of g_j(X_s), where a_j(x) = theta_j g_j(x) and
 *         g_j(x) = prod_s C(x_s, m_js) (trapezoid on leaps, exact under SSA),
 * which are the sufficient statistics of the Gamma(alpha_j + r_j, beta_j + G_j)
 * posterior of each rate constant (Section 1).
 *
 * Conventions for every entry point:
 *  - Return value: ML_OK (0) or a negative ML_ERR_* code.  Nothing aborts or throws.
 *    ml_last_error() returns a thread-local message for the last failure.
 *  - Argument errors are detected synchronously on the host, before any launch.
 *  - Device pointers must be device (or managed) memory of the current device; a host
 *    pointer where a device pointer is expected is rejected with ML_ERR_ARG.
 *  - The caller owns every buffer it passes; the library owns ml_model / ml_server
 *    objects and their internal device tables.
 *  - Per-trajectory anomalies are reported in status_out (ML_ST_* bits), never through
 *    the return code.
 *  - Random numbers: Philox4x32-10 keyed by (seed) with counter (trajectory id, step,
 *    stream, block), trajectory id = traj_id_base + i, so results do not depend on
 *    batch composition, launch shape or sharding.
 */
#ifndef MATLEAP_H
#define MATLEAP_H

#ifndef __CUDACC_RTC__  /* the library's runtime-compiled kernels bring their own types */
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------------------ */
#define ML_OK 0
#define ML_ERR_ARG (-1)     /* malformed model or argument                           */
#define ML_ERR_OOM (-2)     /* device or host allocation failed                      */
#define ML_ERR_CUDA (-3)    /* a CUDA runtime call failed (message in ml_last_error) */
#define ML_ERR_TIMEOUT (-4) /* a bounded wait ran out                                */
#define ML_ERR_BUSY (-5)    /* the server cannot admit the request now               */
#define ML_ERR_UNSUPPORTED (-6) /* no kernel variant for this model size/precision   */

/* ---- per-trajectory status bits (status_out) --------------------------------------- */
#define ML_ST_STEP_LIMIT 1u    /* max_steps reached before T; X is the state at the stop */
#define ML_ST_NEWTON_FAIL 2u   /* an implicit solve failed; an explicit leap was taken   */
#define ML_ST_REJECT_LIMIT 4u  /* max_reject rejections in a row forced an SSA burst     */
#define ML_ST_PTRS_CAP 8u      /* a Poisson draw hit its trial cap                       */
#define ML_ST_BAD_INPUT 16u    /* negative x0 or theta, or a NaN: trajectory not run     */
#define ML_ST_STAGE_TIMEOUT 32u /* model staging wait ran out; plain loads were used     */
#define ML_ST_OVERFLOW 64u     /* counts would leave the exact int64 range: the trajectory
                                  stopped early (state and statistics as at the stop)
                                  because, at the start of a step, a count or firing total
                                  exceeded 2^62, or a leap's Poisson mean or an implicit
                                  firing count exceeded 2^48                             */

/* ---- modes (Section 3: matLeap can also run fully explicit or as SSA) -------------- */
#define ML_MODE_ADAPTIVE 0      /* explicit / implicit / SSA switching                  */
#define ML_MODE_EXPLICIT_ONLY 1 /* never take the implicit branch                       */
#define ML_MODE_SSA_ONLY 2      /* exact Gillespie direct method throughout             */

/* ---- arithmetic ------------------------------------------------------------------- */
#define ML_PREC_REF_FP64 0  /* FP64 everywhere, fixed operation order, no FMA: per
                               trajectory bit-identical to the CPU reference            */
#define ML_PREC_FAST_FP32 1 /* FP32 propensities, step sizes, Poisson means and G
                               increments; FP64 time and G totals; the implicit Newton
                               solve in FP64 (default) or FP32 (newton_precision)      */

/* ---- launch forms ----------------------------------------------------------------- */
#define ML_FORM_PLAIN 0      /* one launch, one thread (or warp) per trajectory         */
#define ML_FORM_PERSISTENT 1 /* resident CTAs refill finished slots from a device work
                                queue; optionally replayed from a CUDA graph           */

/* ---- kernel shapes ---------------------------------------------------------------- */
#define ML_SHAPE_AUTO 0   /* thread per trajectory when the model fits, else warp     */
#define ML_SHAPE_THREAD 1 /* one trajectory per thread (N <= 8, M <= 16), round-based  */
#define ML_SHAPE_WARP 2   /* one trajectory per warp (N <= 64, M <= 128)               */
#define ML_SHAPE_THREAD_OCC 3 /* fast precision only: one trajectory per thread, built
                                 for more resident warps (about 168 registers, some
                                 spilling, at most 128 threads per CTA)              */
#define ML_SHAPE_THREAD_SEQ 4 /* one trajectory per thread, each run to its end before
                                 the next (whole SSA bursts at once); the default
                                 thread shape interleaves leap evaluations and slices
                                 of SSA bursts round by round                         */
#define ML_SHAPE_THREAD_SEQ_OCC 5 /* fast precision only: the sequential per-lane driver
                                     in the occupancy build                           */
#define ML_SHAPE_THREAD_POOL 6 /* persistent form only: one trajectory per thread at a
                                  time, each warp keeping 64 trajectories in shared
                                  memory and running one phase (SSA slices or leap
                                  evaluations) for 32 of them per round, so that its
                                  lanes do not diverge between the phases             */
#define ML_SHAPE_THREAD_POOL_OCC 7 /* fast precision, persistent form: the pool driver
                                      in the occupancy build                          */

/* ---- Jacobian of the implicit solve (Section 1: estimated numerically, or the
 *      symbolic Jacobian of Section 3).  Every FP64 solve follows the choice; the FP32
 *      increment solve of the fast thread kernel (ML_NEWTON_FP32) always uses the exact
 *      derivative (there the Jacobian only sets the convergence rate). --------------- */
#define ML_JAC_FD 0       /* forward differences                                          */
#define ML_JAC_ANALYTIC 1 /* exact derivative of the mass-action polynomials              */

/* ---- arithmetic of the implicit Newton solve in fast precision (reference precision
 *      always solves in FP64) ------------------------------------------------------ */
#define ML_NEWTON_FP64 0 /* FP64 propensities at x and y, residual, Jacobian, elimination
                            and rounding (the default)                                 */
#define ML_NEWTON_FP32 1 /* FP32: the thread kernel solves for the increment z = y - x
                            (no cancellation of propensities of size a tau), the warp
                            kernel factorizes the Jacobian in FP32 under an FP64 residual */

typedef struct ml_model ml_model;

/* Control parameters.  Defaults from ml_default_params():
 * eps 0.03, n_c 10, ssa_factor 10, n_ssa_explicit 100, n_ssa_implicit 10,
 * pe_delta 0.05, stiff_ratio 100, newton_tol 1e-10, newton_maxit 20, fd_h 1e-7,
 * max_steps 1e8, max_reject 64, mode ADAPTIVE, precision REF_FP64, form PLAIN,
 * shape AUTO, block_size 0 (tuned or default), ctas_per_sm 0, use_graph 0,
 * jacobian FD, newton_precision FP64, stage_poll_limit 4194304, queue_order NULL,
 * specialize 0. */
typedef struct {
  double eps;             /* Cao 2006 bound on the relative change of each reactant    */
  int32_t n_c;            /* critical threshold (Section 2)                            */
  double ssa_factor;      /* SSA burst when min(tau1, tau2) < ssa_factor / a0          */
  int32_t n_ssa_explicit; /* burst length after an explicit choice                     */
  int32_t n_ssa_implicit; /* burst length after an implicit choice                     */
  double pe_delta;        /* pair in partial equilibrium: |a_j - a_k| <= pe_delta min  */
  double stiff_ratio;     /* implicit iff tau_im > stiff_ratio * tau_ex                */
  double newton_tol;      /* Newton stop: |dy|_inf <= newton_tol * max(1, |y|_inf)     */
  int32_t newton_maxit;   /* Newton iteration cap                                      */
  double fd_h;            /* forward-difference step factor for the Jacobian           */
  int64_t max_steps;      /* outer-step cap per trajectory                             */
  int32_t max_reject;     /* rejections in a row before an SSA burst is forced         */
  int32_t mode;           /* ML_MODE_*                                                 */
  int32_t precision;      /* ML_PREC_*                                                 */
  int32_t form;           /* ML_FORM_*                                                 */
  int32_t shape;          /* ML_SHAPE_*                                                */
  int32_t block_size;     /* threads per CTA; 0 = autotuned value or default           */
  int32_t ctas_per_sm;    /* persistent form: resident CTAs per SM; 0 = tuned/default  */
  int32_t use_graph;      /* persistent form: launch through a cached CUDA graph       */
  int32_t jacobian;       /* ML_JAC_*: Jacobian of the propensities in implicit leaps  */
  int32_t newton_precision; /* ML_NEWTON_*: fast precision's implicit solve            */
  int32_t stage_poll_limit; /* polls of each thread's wait for the bulk copy of the
                               model tables before the CTA falls back to plain loads
                               and sets ML_ST_STAGE_TIMEOUT (>= 0; 0 forces the
                               fallback, which tests use to exercise it)               */
  const int64_t* queue_order; /* persistent form: NULL, or [n_traj] int64, a permutation of
                               0..n_traj-1: the work queue hands trajectories out in this
                               order.  Giving the longest first removes the tail of lanes
                               that pick up a long trajectory last (e.g. sorted by a
                               previous call's per-trajectory event counts).  Results do
                               not depend on it.  Device memory for ml_simulate and
                               ml_simulate_noalloc and ml_autotune, host memory for
                               ml_simulate_host; ignored by the plain form, the server
                               and an autotuner sample shorter than the batch.
                               Entries outside [0, n_traj) are passed over; trajectories
                               the order leaves out are not run (their outputs are not
                               written)                                               */
  int32_t specialize;     /* thread-per-trajectory shapes: 1 = run kernels compiled for
                               this model, its tables built in as constants (the first
                               call per model, precision and driver compiles one, about
                               a second, and loads it on the device), 0 = the
                               precompiled kernels that read the tables at run time.
                               Results are identical (reference precision: bitwise).
                               Ignored by the warp shape, time-grid calls and
                               ml_simulate_noalloc; the server passes it on.          */
} ml_sim_params;

/* Fills *p with the defaults above.  Returns ML_ERR_ARG if p is NULL. */
int ml_default_params(ml_sim_params* p);

/* Thread-local message describing the last failed call on this thread ("" if none). */
const char* ml_last_error(void);

/* Creates a model (paper Section 1: mass-action network, a_j = theta_j g_j(X)).
 *   n_species N >= 1, n_reactions M >= 1 (N <= 64, M <= 128).
 *   reactant_orders [M][N] row-major host array: m_js >= 0, sum_s m_js <= 3.
 *   net_stoich      [M][N] row-major host array: nu_js >= -m_js, |nu_js| <= 127.
 *   rates           [M] host array: default rate constants, finite and >= 0.
 * The arrays are copied; device tables are uploaded lazily on first use per device.
 * Reversible pairs (reaction k the chemical reverse of reaction j, both with a
 * reactant) are found here.  Errors: ML_ERR_ARG, ML_ERR_OOM. */
int ml_model_create(int32_t n_species, int32_t n_reactions, const int32_t* reactant_orders,
                    const int32_t* net_stoich, const double* rates, ml_model** out);

/* Frees the model and its device tables and cached graphs.  NULL is a no-op.  The
 * caller must make sure no launch that uses the model is still running. */
int ml_model_destroy(ml_model* model);

/* Number of reversible pairs found in the model (>= 0), or ML_ERR_ARG. */
int ml_model_num_pairs(const ml_model* model);

/* Simulates n_traj independent trajectories on the current device, asynchronously on
 * cuda_stream (a cudaStream_t; NULL = legacy default stream).
 *   theta  [n_traj][M] device FP64 per-trajectory rate constants, or NULL for the
 *          model's rates.
 *   x0     device int64: [N] (x0_per_traj = 0, shared) or [n_traj][N].
 *   T      device FP64: [1] (T_per_traj = 0) or [n_traj] horizons.
 *   p      control parameters (NULL = defaults).
 *   seed, traj_id_base: trajectory i uses id traj_id_base + i; ids must stay below 2^32.
 *   X_out  [n_traj][N] int64, r_out [n_traj][M] int64, G_out [n_traj][M] FP64,
 *   status_out [n_traj] uint32, counters_out [n_traj][4] int64 or NULL (accepted
 *          explicit leaps, implicit leaps, SSA firings, rejected leaps) -- all device.
 * n_traj == 0 returns ML_OK without launching.  Errors: ML_ERR_ARG (bad sizes, host
 * pointers, parameters out of range), ML_ERR_UNSUPPORTED (no variant for this size),
 * ML_ERR_CUDA (launch failure), ML_ERR_OOM (internal scratch). */
int ml_simulate(const ml_model* model, int64_t n_traj, const double* theta,
                const int64_t* x0, int32_t x0_per_traj, const double* T,
                int32_t T_per_traj, const ml_sim_params* p, uint64_t seed,
                uint64_t traj_id_base, int64_t* X_out, int64_t* r_out, double* G_out,
                uint32_t* status_out, int64_t* counters_out, void* cuda_stream);

/* Same as ml_simulate with HOST buffers (same shapes): copies inputs to device
 * workspace owned by the model, runs, copies results back and synchronizes the stream
 * before returning.  Pinned host memory makes the copies asynchronous DMA.
 * Not reentrant for one model: concurrent calls on the same model must be serialized
 * by the caller (ML_ERR_BUSY is returned if a call is already running). */
int ml_simulate_host(ml_model* model, int64_t n_traj, const double* theta,
                     const int64_t* x0, int32_t x0_per_traj, const double* T,
                     int32_t T_per_traj, const ml_sim_params* p, uint64_t seed,
                     uint64_t traj_id_base, int64_t* X_out, int64_t* r_out, double* G_out,
                     uint32_t* status_out, int64_t* counters_out, void* cuda_stream);

/* Project autotuner: times candidate kernel shapes (trajectory per thread -- round-based,
 * sequential or pool driver, each also in the occupancy build where that exists -- or per
 * warp, threads per CTA 64/128/256, resident CTAs per SM 0 (as many as fit), 1, 2 or 4
 * up to what fits at once; a model that fits one thread tries the warp kernel in one
 * launch shape only) on the first min(n_traj, n_sample) trajectories of the given
 * inputs, with p's mode/precision/form (one warm-up run, then the median of three timed
 * runs per candidate; a candidate whose warm-up takes more than twice the best median so
 * far is dropped; candidates in a fixed order, a later one replacing the best so far only
 * when more than 3 % faster), and stores the choice in the model (used when a later call
 * passes block_size = 0) and in *best.  Synchronizes cuda_stream.  Uses internal scratch
 * outputs. */
int ml_autotune(ml_model* model, int64_t n_traj, const double* theta, const int64_t* x0,
                int32_t x0_per_traj, const double* T, int32_t T_per_traj,
                const ml_sim_params* p, uint64_t seed, int64_t n_sample,
                ml_sim_params* best, void* cuda_stream);

/* Allocation-free variant of ml_simulate, for callers that cannot let a library allocate
 * device memory: code running under a device-memory pool owned by a host framework (a
 * deep-learning runtime, an MPS client with a capped budget), latency-bound loops that
 * cannot afford cudaMalloc's implicit synchronization, and code that must not take the
 * CUDA allocator's lock.  The paper has no counterpart; this is a deployment interface.
 *   Same arguments and results as ml_simulate (all buffers caller-owned device memory).
 *   Always runs the persistent refill kernel, one trajectory per thread, in p's precision
 *   (p->form and p->use_graph are ignored).
 *   Its only scratch (the work-queue counter and a copy of the model tables) is a fixed
 *   4 KiB device array inside the library, reserved on every GPU that loads it until the
 *   process exits.  Each call launches two kernels on cuda_stream: one that zeroes the
 *   counter and writes the model tables (passed by value as its parameter, so no host
 *   memory is read by a copy) and the simulation.  Models with more than 8 species or 16
 *   reactions (which need one warp per trajectory) are rejected with ML_ERR_ARG and a
 *   message naming the size; p->shape = ML_SHAPE_WARP gives ML_ERR_UNSUPPORTED.
 *   Every call looks up the array's device address for the current device; the first
 *   call on a device also loads the library's module there, so make that first call
 *   before any stream capture.
 *   Every call reuses the same array and overwrites what the previous call left there:
 *   calls whose kernels overlap on the GPU (other streams, other threads) race and must
 *   be serialized by the caller.
 *   Makes no cudaMalloc, cudaFree or other allocating call.
 * Errors: as ml_simulate. */
int ml_simulate_noalloc(const ml_model* model, int64_t n_traj, const double* theta,
                        const int64_t* x0, int32_t x0_per_traj, const double* T,
                        int32_t T_per_traj, const ml_sim_params* p, uint64_t seed,
                        uint64_t traj_id_base, int64_t* X_out, int64_t* r_out, double* G_out,
                        uint32_t* status_out, int64_t* counters_out, void* cuda_stream);

/* Number of species N / reactions M of the model (>= 1), or ML_ERR_ARG. */
int ml_model_num_species(const ml_model* model);
int ml_model_num_reactions(const ml_model* model);

/* ---- continuous-batching server --------------------------------------------------- *
 * Serves simulate requests of different models and sizes as they arrive (paper Section
 * 2: the simulator is called repeatedly with new parameter matrices, e.g. inside a
 * particle filter).  A scheduler thread admits requests in arrival order whenever one of
 * max_inflight slots and enough of the device-memory budget are free, keeps each
 * admitted request's inputs and outputs in a device arena of hbm_budget_bytes, runs it on
 * the slot's own stream (admitted requests execute concurrently on the GPU) and copies the
 * results to pinned host memory.  Results depend only on the request (random numbers are
 * keyed by trajectory id), never on what else is in flight. */
typedef struct ml_server ml_server;
typedef struct ml_request ml_request;

/* Creates a server on the current device.  hbm_budget_bytes >= 1 MiB is reserved at once;
 * 1 <= max_inflight <= 64; p = simulation parameters for every request (NULL = defaults;
 * use_graph is ignored).  Errors: ML_ERR_ARG, ML_ERR_OOM, ML_ERR_CUDA (no device). */
int ml_server_create(size_t hbm_budget_bytes, int32_t max_inflight, const ml_sim_params* p,
                     ml_server** out);

/* Queues a request without blocking: host inputs in the layouts of ml_simulate (theta
 * [n][M] or NULL, x0 [N] or [n][N], T [1] or [n]) are copied at once, so the caller may
 * reuse its buffers on return.  *out is owned by the caller (ml_request_free).
 * Errors: ML_ERR_ARG; ML_ERR_BUSY if the request alone exceeds the budget or the server
 * is shutting down; ML_ERR_OOM. */
int ml_server_submit(ml_server* server, const ml_model* model, int64_t n_traj,
                     const double* theta, const int64_t* x0, int32_t x0_per_traj,
                     const double* T, int32_t T_per_traj, uint64_t seed,
                     uint64_t traj_id_base, ml_request** out);

/* Waits up to timeout_ms (< 0: no limit) for the request.  ML_OK when its results are
 * ready, ML_ERR_TIMEOUT if it is still queued or running, else the request's error. */
int ml_request_wait(ml_server* server, ml_request* req, int32_t timeout_ms);

/* Copies a finished request's results to host buffers (any may be NULL): X [n][N],
 * r [n][M], G [n][M], status [n], counters [n][4]; latency_s = completion - submission,
 * queue_s = admission - submission.  ML_ERR_BUSY if not finished. */
int ml_request_result(const ml_request* req, int64_t* X_out, int64_t* r_out, double* G_out,
                      uint32_t* status_out, int64_t* counters_out, double* latency_s,
                      double* queue_s);

/* Frees a finished request (ML_ERR_BUSY while it is queued or running).  Free requests
 * before destroying their server (or pass server = NULL afterwards). */
int ml_request_free(ml_server* server, ml_request* req);

/* Counters since creation: requests admitted and completed, trajectories admitted, peak
 * arena bytes in use, peak number of requests in flight (any pointer may be NULL). */
int ml_server_stats(ml_server* server, int64_t* admitted, int64_t* completed,
                    int64_t* trajectories, size_t* peak_bytes, int32_t* peak_inflight);

/* Stops admitting, fails requests that were never admitted (ML_ERR_BUSY), waits for the
 * running ones and frees the server.  NULL is a no-op. */
int ml_server_destroy(ml_server* server);

/* ml_simulate with time-grid output (paper, Section 3: the accuracy study compares
 * marginal distributions at a series of time points).  t_obs: K observation times, device
 * memory, shared by all trajectories; they must be finite, >= 0 and nondecreasing, which
 * the kernel checks (status ML_ST_BAD_INPUT on every trajectory otherwise, so the call
 * stays asynchronous).  X_obs: [n_traj][K][N] int64, device memory, receives X(t_k): the
 * path is right-continuous and piecewise constant, so X(t_k) is the state after every
 * change at a time <= t_k.  A leap is shortened to end exactly at the next grid point (as
 * it is at T), so a grid changes the trajectory itself; SSA firings are not moved.  Grid
 * points beyond the trajectory's end (t_k > T, or after a step-limit stop) receive its
 * final state.  K = 0 (t_obs, X_obs may be NULL) is ml_simulate.  Other arguments,
 * errors and asynchrony as ml_simulate. */
int ml_simulate_grid(const ml_model* model, int64_t n_traj, const double* theta,
                     const int64_t* x0, int32_t x0_per_traj, const double* T,
                     int32_t T_per_traj, const ml_sim_params* params, uint64_t seed,
                     uint64_t traj_id_base, const double* t_obs, int32_t K, int64_t* X_obs,
                     int64_t* X_out, int64_t* r_out, double* G_out, uint32_t* status_out,
                     int64_t* counters_out, void* stream);

/* Accuracy metric (paper, Section 3 and Table 1): the Kullback-Leibler divergence of a
 * method's marginal distributions from those of exact SSA, per time point and species,
 * and its average over all of them.  The paper does not define the empirical
 * distributions; this library bins the integer counts of both samples on their pooled
 * range [lo, hi] with integer width w = ceil((hi - lo + 1) / max_bins), adds 1/2 to every
 * bin of both histograms, and computes KL(p || q) = sum_b p_b (log p_b - log q_b) with
 * p_b = (c_ref,b + 1/2) / (n_ref + nbins/2) from the reference (SSA) sample and q from the
 * test sample.  Sums over bins and the mean over the K x N pairs use a fixed order
 * (32 lanes in index order, then a butterfly), so results are bit-reproducible.
 *   X_ref [n_ref][K][N], X_test [n_test][K][N]: int64 device memory (ml_simulate_grid's
 *   X_obs layout).  kl_out [K][N] double, device memory.  kl_mean_out: optional device
 *   double.  1 <= max_bins <= 4096; n_ref, n_test >= 1 and below 2^31.
 * Asynchronous on stream; argument errors as ML_ERR_ARG before any launch. */
int ml_kl_divergence(int64_t n_ref, const int64_t* X_ref, int64_t n_test,
                     const int64_t* X_test, int32_t K, int32_t N, int32_t max_bins,
                     double* kl_out, double* kl_mean_out, void* stream);

/* Measurement utility for the roofline (the paper has no counterpart): sustained
 * throughput of the pipes the simulation kernels use, from project microbenchmarks of
 * independent dependency chains on every SM of the current device, each run about 20 ms:
 *   out3[0] FP64 FMA flop/s (an FMA counts 2), out3[1] FP32 FMA flop/s, out3[2]
 *   special-function (base-2 logarithm) operations/s.
 * out3: host array of 3 doubles.  Synchronizes stream.  Allocates no device memory. */
int ml_measure_pipe_peaks(double* out3, void* stream);

/* Number of kernel launches the last ml_simulate/ml_simulate_host call on this model
 * issued (a graph replay counts its kernel nodes), or ML_ERR_ARG. */
int64_t ml_model_last_launch_count(const ml_model* model);

/* ---- The Bayesian step (paper, Section 1) ---------------------------------------------
 * With a Gamma(alpha_j, beta_j) prior on each rate constant theta_j, the likelihood of a
 * path is conjugate and the posterior given a simulated path is Gamma(alpha_j + r_j,
 * beta_j + G_j) (shape, rate).  These two calls turn ml_simulate's r and G into posterior
 * draws and resample particles by their weights, so that a particle-filter or ABC step
 * runs on the device between simulations.  Both are FP64 and bit-reproducible. */

/* One draw theta_ij ~ Gamma(alpha_ij + r_ij, beta_ij + G_ij) per trajectory i and
 * reaction j (Marsaglia & Tsang 2000, with the U^(1/shape) boost for shape < 1).
 *   alpha, beta  prior shape and rate: [n * M] row-major when *_per_traj is non-zero,
 *                else one row [M] shared by every trajectory.  Device memory.
 *   r, G         [n * M] row-major, as written by ml_simulate.  Device memory.
 *   theta_out    [n * M] row-major.  Device memory.  A non-positive or NaN posterior
 *                shape or rate gives NaN.
 *   status_out   optional [n] device array: bit 1 set when 64 proposals of one draw were
 *                all rejected (the draw is then the posterior mean; never observed).
 * Random numbers: Philox4x32-10 keyed by seed, counter (traj_id_base + i, 0x80000000 + j,
 * 0, block); traj_id_base + n must not exceed 2^32 (ML_ERR_ARG).  Asynchronous on stream
 * (a cudaStream_t, NULL for the legacy default stream).  n = 0 is a no-op. */
int ml_posterior_sample(int64_t n, int32_t M, const double* alpha, int32_t alpha_per_traj,
                        const double* beta, int32_t beta_per_traj, const int64_t* r,
                        const double* G, uint64_t seed, uint64_t traj_id_base, double* theta_out,
                        uint32_t* status_out, void* stream);

/* Workspace bytes ml_resample_systematic needs for n particles (0 for n < 1). */
size_t ml_resample_workspace_bytes(int64_t n);

/* Systematic resampling of n particles from log-weights logw[n] (device memory) into
 * ancestors[n] (device memory, int64).  Weights are quantized to integers
 * q_i = floor(exp(logw_i - max logw) 2^40) -- a NaN log-weight counts as weight 0 -- so
 * that the cumulative sums are exact; ancestor k is the first i whose inclusive prefix
 * sum exceeds floor((k Q + floor(u Q)) / n), Q = sum q_i, u one uniform from counter
 * (id_base, 0xC0000000, 0, 0).  When no weight is positive (all -inf or NaN) or the
 * maximum is +inf, every ancestor is -1: the call itself still returns ML_OK because the
 * check runs on the device.  workspace: device memory, 16-byte aligned, at least
 * ml_resample_workspace_bytes(n), owned by the caller and not shared by concurrent calls.
 * Requires 1 <= n < 2^24 (ML_ERR_ARG otherwise).  Asynchronous on stream. */
int ml_resample_systematic(int64_t n, const double* logw, uint64_t seed, uint64_t id_base,
                           int64_t* ancestors, void* workspace, size_t workspace_bytes,
                           void* stream);

#ifdef __cplusplus
}
#endif
#endif
