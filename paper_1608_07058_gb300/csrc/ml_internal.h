// Internal declarations shared by the CUDA library's translation units (host API and
// kernels).  Nothing here is visible through include/matleap.h.
#pragma once
#ifndef __CUDACC_RTC__  // runtime compilation (model-specialized kernels) brings its own types
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>
#endif

namespace mlk {

// Thread-per-trajectory variants, (species, reactions) capacities.  A model is run on
// the smallest variant that holds it; padded species start at 0 and are touched by no
// reaction, padded reactions have no reactants, no effect and rate 0.
constexpr int kThreadVariants = 4;
constexpr int kThreadN[kThreadVariants] = {1, 3, 3, 8};
constexpr int kThreadM[kThreadVariants] = {2, 4, 6, 16};

// Count limits (status ML_ST_OVERFLOW): a count or firing total above kCountLimit at the
// start of a step, or a leap's Poisson mean or implicit firing count above kLeapLimit,
// stops the trajectory; with M <= 128 and |nu| <= 127 every int64 sum stays below 2^63.
constexpr long long kCountLimit = 1LL << 62;
constexpr long long kLeapLimitInt = 1LL << 48;
constexpr double kLeapLimit = 281474976710656.0;  // 2^48

// Trajectories each warp of the pool driver keeps in shared memory, and the 32-bit words
// of one trajectory's record there (mode, id, status, step, reject run, burst index and
// length; trajectory index, t, T; theta; x, r, G and the four event counters).
constexpr int kPoolSlots = 64;
__host__ __device__ constexpr int lane_record_words(int NM, int MM, bool ref) {
  return 13 + (ref ? 2 : 1) * MM + 2 * NM + 4 * MM + 8;
}

// Warp-per-trajectory capacities.
constexpr int kWarpMaxN = 64;
constexpr int kWarpMaxM = 128;

// Highest-order-reaction flags per species (Cao 2006): which (reaction order, molecules
// of this species) combinations occur among the reactions that consume it.
enum : uint8_t {
  kHorO1 = 1,     // first order
  kHorO2M1 = 2,   // S + S'
  kHorO2M2 = 4,   // 2S
  kHorO3M1 = 8,   // S + S' + S''
  kHorO3M2 = 16,  // 2S + S'
  kHorO3M3 = 32,  // 3S
};

// Model tables for the thread-per-trajectory kernels, one fixed layout per variant.
// Staged into shared memory at kernel start by one bulk copy.
template <int NM, int MM>
struct alignas(16) ThreadModel {
  static constexpr bool kCompiled = false;  // tables read at run time (see JitModel)
  double rates[MM];
  float nuf[MM][NM];    // nu_js as FP32 (updates of the fast SSA slice's FP32 state copy)
  int8_t ord[MM][NM];   // m_js
  int8_t nu[MM][NM];    // nu_js
  int8_t partner[MM];   // for the lower reaction of a reversible pair: the other; else -1
  uint8_t isreact[NM];  // species consumed by some reaction
  uint8_t hor[NM];      // kHor* flags
  int32_t n_pairs;
  int32_t N, M;         // real sizes
};

template <int NM, int MM>
__host__ __device__ constexpr size_t thread_model_bytes() {
  return (sizeof(ThreadModel<NM, MM>) + 15) / 16 * 16;
}

// Model tables for the warp-per-trajectory kernels (compact sparse lists).
struct alignas(16) WarpModel {
  double rates[kWarpMaxM];
  // species bit masks (N <= 64): the reactants of reaction j, and the species reaction j
  // changes.  After a firing of k, exactly the reactions j with rmask[j] & cmask[k] != 0
  // have new propensities.
  uint64_t rmask[kWarpMaxM];
  uint64_t cmask[kWarpMaxM];
  int32_t N, M, n_pairs, nnz;
  // reactants of reaction j: up to 3 (species, multiplicity), increasing species
  int8_t rsp[kWarpMaxM][3];
  int8_t rmul[kWarpMaxM][3];
  int8_t nreact[kWarpMaxM];
  int8_t partner[kWarpMaxM];      // as in ThreadModel
  uint8_t isreact[kWarpMaxN];
  uint8_t hor[kWarpMaxN];
  // nonzero net changes of reaction j: rx_ptr[j] .. rx_ptr[j+1]
  int16_t rx_ptr[kWarpMaxM + 1];
  // reactions changing species s, increasing j: sp_ptr[s] .. sp_ptr[s+1]
  int16_t sp_ptr[kWarpMaxN + 1];
  int16_t pad0;
  // entries (filled up to nnz): per-reaction lists then per-species lists
  int8_t rx_s[kWarpMaxM * 8];
  int8_t rx_nu[kWarpMaxM * 8];
  int16_t sp_j[kWarpMaxM * 8];
  int8_t sp_nu[kWarpMaxM * 8];
};

// Everything a simulation kernel needs besides the model tables.
struct SimArgs {
  int64_t n_traj;
  const double* theta;  // [n_traj][M] or null
  const int64_t* x0;    // [N] or [n_traj][N]
  const double* T;      // [1] or [n_traj]
  int32_t x0_per, T_per;
  int32_t N, M;         // real sizes (I/O strides, random-stream numbering)
  uint64_t seed;
  uint64_t id_base;
  int64_t* X;
  int64_t* r;
  double* G;
  uint32_t* status;
  int64_t* counters;    // or null
  // control parameters
  double eps;
  double ssa_factor;
  double pe_delta;
  double stiff_ratio;
  double newton_tol;
  double fd_h;
  int64_t max_steps;
  int32_t n_c;
  int32_t n_ssa_ex;
  int32_t n_ssa_im;
  int32_t newton_maxit;
  int32_t max_reject;
  int32_t mode;
  int32_t jacobian;  // ML_JAC_*
  int32_t newton_fp32;  // fast precision: FP32 implicit solve (ML_NEWTON_FP32)
  int32_t stage_polls;  // bounded wait for the model-table bulk copy
  // persistent form: next unclaimed trajectory (zeroed before each launch), and the
  // optional order in which the queue hands trajectories out ([n_traj] or null)
  unsigned long long* queue;
  const int64_t* order;
  // time-grid output: K_obs observation times (nondecreasing, >= 0, finite; checked on the
  // device, BAD_INPUT otherwise) and X_obs [n_traj][K_obs][N]; K_obs = 0 records nothing
  const double* t_obs;
  int64_t* X_obs;
  int32_t K_obs;
};

#ifndef __CUDACC_RTC__
// One compiled kernel variant: its launcher and its function pointer (for occupancy
// queries and CUDA-graph kernel nodes).  Every kernel takes (model tables, SimArgs).
using LaunchFn = cudaError_t (*)(const void* dmodel, const SimArgs& a, int grid, int block,
                                 size_t smem, cudaStream_t s);
struct KernelEntry {
  LaunchFn launch;
  const void* kernel;
  int pool_words = 0;  // pool driver: 32-bit words of one trajectory's state record
};

// Thread-per-trajectory variants (kern_thread.cu, one object per precision x variant).
KernelEntry thread_entry_ref_0();
KernelEntry thread_entry_ref_1();
KernelEntry thread_entry_ref_2();
KernelEntry thread_entry_ref_3();
KernelEntry thread_entry_fast_0();
KernelEntry thread_entry_fast_1();
KernelEntry thread_entry_fast_2();
KernelEntry thread_entry_fast_3();
KernelEntry thread_entry_fastocc_0();
KernelEntry thread_entry_fastocc_1();
KernelEntry thread_entry_fastocc_2();
KernelEntry thread_entry_fastocc_3();
// Sequential-driver builds (one per precision x variant).
KernelEntry thread_seq_entry_ref_0();
KernelEntry thread_seq_entry_ref_1();
KernelEntry thread_seq_entry_ref_2();
KernelEntry thread_seq_entry_ref_3();
KernelEntry thread_seq_entry_fast_0();
KernelEntry thread_seq_entry_fast_1();
KernelEntry thread_seq_entry_fast_2();
KernelEntry thread_seq_entry_fast_3();
KernelEntry thread_seq_entry_fastocc_0();
KernelEntry thread_seq_entry_fastocc_1();
KernelEntry thread_seq_entry_fastocc_2();
KernelEntry thread_seq_entry_fastocc_3();
// Pool-driver builds (one per precision x variant; persistent form only).
KernelEntry thread_pool_entry_ref_0();
KernelEntry thread_pool_entry_ref_1();
KernelEntry thread_pool_entry_ref_2();
KernelEntry thread_pool_entry_ref_3();
KernelEntry thread_pool_entry_fast_0();
KernelEntry thread_pool_entry_fast_1();
KernelEntry thread_pool_entry_fast_2();
KernelEntry thread_pool_entry_fast_3();
KernelEntry thread_pool_entry_fastocc_0();
KernelEntry thread_pool_entry_fastocc_1();
KernelEntry thread_pool_entry_fastocc_2();
KernelEntry thread_pool_entry_fastocc_3();
// Sequential driver with time-grid output (reference and fast builds).
KernelEntry thread_seq_grid_entry_ref_0();
KernelEntry thread_seq_grid_entry_ref_1();
KernelEntry thread_seq_grid_entry_ref_2();
KernelEntry thread_seq_grid_entry_ref_3();
KernelEntry thread_seq_grid_entry_fast_0();
KernelEntry thread_seq_grid_entry_fast_1();
KernelEntry thread_seq_grid_entry_fast_2();
KernelEntry thread_seq_grid_entry_fast_3();
// Warp-per-trajectory kernels (kern_warp.cu, one object per precision), without and with
// time-grid output.
KernelEntry warp_entry_ref();
KernelEntry warp_entry_fast();
KernelEntry warp_grid_entry_ref();
KernelEntry warp_grid_entry_fast();
// Dynamic shared memory of the warp kernel for a CTA of `warps` warps (newton_fp32: fast
// precision with an FP32 Newton system).
size_t warp_smem_bytes(int warps, int N, int M, int precision, bool newton_fp32);

// Launch description for the allocation-free entry point: everything is validated and
// chosen by the host API without touching device memory; the caller copies host_tables
// into its own scratch and fills args.queue.
struct NoAllocLaunch {
  KernelEntry entry;
  const void* host_tables;  // built at model creation, lives as long as the model
  size_t table_bytes;
  int grid, block;
  SimArgs args;
};
#endif  // __CUDACC_RTC__
}  // namespace mlk

#ifndef __CUDACC_RTC__
struct ml_model;
namespace mlk {
// Returns ML_OK and fills *out, or an ML_ERR_* code (message set).  `scratch_table_max`
// is the room for model tables in the caller's scratch.
int noalloc_prepare(const ml_model* m, int64_t n_traj, const double* theta, const int64_t* x0,
                    int32_t x0_per_traj, const double* T, int32_t T_per_traj,
                    const void* params, uint64_t seed, uint64_t id_base, int64_t* X,
                    int64_t* r, double* G, uint32_t* status, int64_t* counters,
                    size_t scratch_table_max, NoAllocLaunch* out);
int set_error(int code, const char* msg);
// True for device or managed memory (a failed query clears the CUDA error and is false).
bool is_device_pointer(const void* p);

}  // namespace mlk
#endif  // __CUDACC_RTC__
