// Host side of the C ABI declared in include/matleap.h: argument checking, model tables
// (built here, independently of any other implementation), kernel selection, the
// persistent work queue and its CUDA graph, the host-buffer path and the autotuner.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "jit.h"
#include "matleap.h"
#include "ml_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? ML_ERR_OOM : ML_ERR_CUDA, "%s: %s", where,
              cudaGetErrorString(e));
}

#define ML_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t e_ = (expr);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);   \
  } while (0)

constexpr int kQueueSlots = 256;  // in-flight persistent launches per model and device

struct GraphCache {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t memset_node = nullptr;
  cudaGraphNode_t kernel_node = nullptr;
  const void* kernel = nullptr;
};

struct Tuned {
  int shape = 0, block = 0, ctas_per_sm = 0;
};

// A model-specialized kernel, loaded as a CUDA library (valid in every context).
struct JitKernel {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
  int pool_words = 0;
};

struct DeviceState {
  void* thread_tables[mlk::kThreadVariants] = {};
  void* warp_tables = nullptr;
  unsigned long long* queues = nullptr;  // kQueueSlots counters
  unsigned next_slot = 0;
  int sm_count = 0;
  std::map<std::pair<int, int>, GraphCache> graphs;  // (precision, shape/variant)
  std::map<std::pair<int, int>, Tuned> tuned;        // (precision, form)
  // host-path workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool host_busy = false;
};

}  // namespace

struct ml_model {
  int32_t N = 0, M = 0;
  std::vector<int32_t> ord, nu;  // [M][N]
  std::vector<double> rates;
  std::vector<int32_t> otot;     // reactant order of each reaction
  std::vector<int32_t> partner;  // reversible partner (both directions), -1 if none
  int32_t n_pairs = 0;
  std::vector<uint8_t> hor, isreact;
  std::mutex mu;
  std::map<int, DeviceState> dev;
  int64_t last_launches = 0;
  int thread_variant = -1;                // smallest thread variant holding the model
  std::vector<uint8_t> host_thread_tables;  // its tables (for the allocation-free path)
  size_t warp_table_bytes = 0;
  std::map<int, JitKernel> jit;  // specialized kernels by (precision, driver, occupancy build)
};

namespace {

// ---- model tables -----------------------------------------------------------------

template <int NM, int MM>
std::vector<uint8_t> build_thread_tables(const ml_model& m) {
  mlk::ThreadModel<NM, MM> t;
  std::memset(&t, 0, sizeof t);
  for (int j = 0; j < MM; ++j) {
    t.rates[j] = j < m.M ? m.rates[j] : 0.0;
    t.partner[j] = -1;
    for (int s = 0; s < NM; ++s) {
      const bool in = j < m.M && s < m.N;
      t.ord[j][s] = in ? (int8_t)m.ord[j * m.N + s] : 0;
      t.nu[j][s] = in ? (int8_t)m.nu[j * m.N + s] : 0;
      t.nuf[j][s] = (float)t.nu[j][s];
    }
  }
  for (int j = 0; j < m.M && j < MM; ++j)  // the variant always holds the model (M <= MM)
    if (m.partner[j] > j) t.partner[j] = (int8_t)m.partner[j];
  for (int s = 0; s < NM; ++s) {
    t.isreact[s] = s < m.N ? m.isreact[s] : 0;
    t.hor[s] = s < m.N ? m.hor[s] : 0;
  }
  t.n_pairs = m.n_pairs;
  t.N = m.N;
  t.M = m.M;
  std::vector<uint8_t> out(mlk::thread_model_bytes<NM, MM>(), 0);
  std::memcpy(out.data(), &t, sizeof t);
  return out;
}

std::vector<uint8_t> thread_tables(int variant, const ml_model& m) {
  switch (variant) {
    case 0: return build_thread_tables<mlk::kThreadN[0], mlk::kThreadM[0]>(m);
    case 1: return build_thread_tables<mlk::kThreadN[1], mlk::kThreadM[1]>(m);
    case 2: return build_thread_tables<mlk::kThreadN[2], mlk::kThreadM[2]>(m);
    case 3: return build_thread_tables<mlk::kThreadN[3], mlk::kThreadM[3]>(m);
    default: return {};
  }
}

std::vector<uint8_t> warp_tables(const ml_model& m) {
  std::vector<uint8_t> out((sizeof(mlk::WarpModel) + 15) / 16 * 16, 0);
  mlk::WarpModel& w = *reinterpret_cast<mlk::WarpModel*>(out.data());
  w.N = m.N;
  w.M = m.M;
  w.n_pairs = m.n_pairs;
  for (int j = 0; j < mlk::kWarpMaxM; ++j) {
    w.rates[j] = j < m.M ? m.rates[j] : 0.0;
    w.partner[j] = -1;
    for (int q = 0; q < 3; ++q) w.rsp[j][q] = -1;
  }
  for (int j = 0; j < m.M; ++j) {
    int q = 0;
    for (int s = 0; s < m.N; ++s) {
      const int o = m.ord[j * m.N + s];
      if (o > 0) {
        w.rsp[j][q] = (int8_t)s;
        w.rmul[j][q] = (int8_t)o;
        ++q;
      }
    }
    w.nreact[j] = (int8_t)q;
    if (m.partner[j] > j) w.partner[j] = (int8_t)m.partner[j];
    uint64_t rm = 0, cm = 0;
    for (int s = 0; s < m.N; ++s) {
      if (m.ord[j * m.N + s] > 0) rm |= 1ULL << s;
      if (m.nu[j * m.N + s] != 0) cm |= 1ULL << s;
    }
    w.rmask[j] = rm;
    w.cmask[j] = cm;
  }
  int k = 0;
  for (int j = 0; j < m.M; ++j) {
    w.rx_ptr[j] = (int16_t)k;
    for (int s = 0; s < m.N; ++s) {
      const int v = m.nu[j * m.N + s];
      if (v != 0) {
        w.rx_s[k] = (int8_t)s;
        w.rx_nu[k] = (int8_t)v;
        ++k;
      }
    }
  }
  w.rx_ptr[m.M] = (int16_t)k;
  w.nnz = k;
  k = 0;
  for (int s = 0; s < m.N; ++s) {
    w.sp_ptr[s] = (int16_t)k;
    for (int j = 0; j < m.M; ++j) {
      const int v = m.nu[j * m.N + s];
      if (v != 0) {
        w.sp_j[k] = (int16_t)j;
        w.sp_nu[k] = (int8_t)v;
        ++k;
      }
    }
  }
  w.sp_ptr[m.N] = (int16_t)k;
  for (int s = 0; s < m.N; ++s) {
    w.isreact[s] = m.isreact[s];
    w.hor[s] = m.hor[s];
  }
  return out;
}

int thread_variant_for(const ml_model& m) {
  for (int v = 0; v < mlk::kThreadVariants; ++v)
    if (m.N <= mlk::kThreadN[v] && m.M <= mlk::kThreadM[v]) return v;
  return -1;
}

bool warp_fits(const ml_model& m) {
  size_t nnz = 0;
  for (int32_t v : m.nu) nnz += v != 0;
  return m.N <= mlk::kWarpMaxN && m.M <= mlk::kWarpMaxM && nnz <= (size_t)mlk::kWarpMaxM * 8;
}

mlk::KernelEntry thread_seq_entry(int precision, int variant, bool occ = false) {
  if (precision == ML_PREC_FAST_FP32 && occ) {
    switch (variant) {
      case 0: return mlk::thread_seq_entry_fastocc_0();
      case 1: return mlk::thread_seq_entry_fastocc_1();
      case 2: return mlk::thread_seq_entry_fastocc_2();
      default: return mlk::thread_seq_entry_fastocc_3();
    }
  }
  if (precision == ML_PREC_FAST_FP32) {
    switch (variant) {
      case 0: return mlk::thread_seq_entry_fast_0();
      case 1: return mlk::thread_seq_entry_fast_1();
      case 2: return mlk::thread_seq_entry_fast_2();
      default: return mlk::thread_seq_entry_fast_3();
    }
  }
  switch (variant) {
    case 0: return mlk::thread_seq_entry_ref_0();
    case 1: return mlk::thread_seq_entry_ref_1();
    case 2: return mlk::thread_seq_entry_ref_2();
    default: return mlk::thread_seq_entry_ref_3();
  }
}

mlk::KernelEntry thread_pool_entry(int precision, int variant, bool occ = false) {
  if (precision == ML_PREC_FAST_FP32 && occ) {
    switch (variant) {
      case 0: return mlk::thread_pool_entry_fastocc_0();
      case 1: return mlk::thread_pool_entry_fastocc_1();
      case 2: return mlk::thread_pool_entry_fastocc_2();
      default: return mlk::thread_pool_entry_fastocc_3();
    }
  }
  if (precision == ML_PREC_FAST_FP32) {
    switch (variant) {
      case 0: return mlk::thread_pool_entry_fast_0();
      case 1: return mlk::thread_pool_entry_fast_1();
      case 2: return mlk::thread_pool_entry_fast_2();
      default: return mlk::thread_pool_entry_fast_3();
    }
  }
  switch (variant) {
    case 0: return mlk::thread_pool_entry_ref_0();
    case 1: return mlk::thread_pool_entry_ref_1();
    case 2: return mlk::thread_pool_entry_ref_2();
    default: return mlk::thread_pool_entry_ref_3();
  }
}

mlk::KernelEntry thread_entry(int precision, int variant, bool occ = false) {
  if (precision == ML_PREC_FAST_FP32 && occ) {
    switch (variant) {
      case 0: return mlk::thread_entry_fastocc_0();
      case 1: return mlk::thread_entry_fastocc_1();
      case 2: return mlk::thread_entry_fastocc_2();
      default: return mlk::thread_entry_fastocc_3();
    }
  }
  if (precision == ML_PREC_FAST_FP32) {
    switch (variant) {
      case 0: return mlk::thread_entry_fast_0();
      case 1: return mlk::thread_entry_fast_1();
      case 2: return mlk::thread_entry_fast_2();
      default: return mlk::thread_entry_fast_3();
    }
  }
  switch (variant) {
    case 0: return mlk::thread_entry_ref_0();
    case 1: return mlk::thread_entry_ref_1();
    case 2: return mlk::thread_entry_ref_2();
    default: return mlk::thread_entry_ref_3();
  }
}

mlk::KernelEntry warp_entry(int precision) {
  return precision == ML_PREC_FAST_FP32 ? mlk::warp_entry_fast() : mlk::warp_entry_ref();
}

// Time-grid output: the sequential driver's grid build (thread shapes) or the warp
// kernel's grid build.
mlk::KernelEntry thread_seq_grid_entry(int precision, int variant) {
  if (precision == ML_PREC_FAST_FP32) {
    switch (variant) {
      case 0: return mlk::thread_seq_grid_entry_fast_0();
      case 1: return mlk::thread_seq_grid_entry_fast_1();
      case 2: return mlk::thread_seq_grid_entry_fast_2();
      default: return mlk::thread_seq_grid_entry_fast_3();
    }
  }
  switch (variant) {
    case 0: return mlk::thread_seq_grid_entry_ref_0();
    case 1: return mlk::thread_seq_grid_entry_ref_1();
    case 2: return mlk::thread_seq_grid_entry_ref_2();
    default: return mlk::thread_seq_grid_entry_ref_3();
  }
}

mlk::KernelEntry warp_grid_entry(int precision) {
  return precision == ML_PREC_FAST_FP32 ? mlk::warp_grid_entry_fast() : mlk::warp_grid_entry_ref();
}

using mlk::is_device_pointer;

int check_params(const ml_sim_params& p) {
  if (!(p.eps > 0.0 && p.eps < 1.0)) return fail(ML_ERR_ARG, "eps must be in (0, 1)");
  if (p.n_c < 0) return fail(ML_ERR_ARG, "n_c must be >= 0");
  if (!(p.ssa_factor >= 0.0) || !std::isfinite(p.ssa_factor))
    return fail(ML_ERR_ARG, "ssa_factor must be finite and >= 0");
  if (p.n_ssa_explicit < 1 || p.n_ssa_implicit < 1)
    return fail(ML_ERR_ARG, "SSA burst lengths must be >= 1");
  if (!(p.pe_delta >= 0.0) || !(p.stiff_ratio > 0.0))
    return fail(ML_ERR_ARG, "pe_delta must be >= 0 and stiff_ratio > 0");
  if (!(p.newton_tol > 0.0) || p.newton_maxit < 1 || !(p.fd_h > 0.0))
    return fail(ML_ERR_ARG, "newton_tol, newton_maxit and fd_h must be positive");
  if (p.max_steps < 1 || p.max_reject < 1)
    return fail(ML_ERR_ARG, "max_steps and max_reject must be >= 1");
  if (p.mode < ML_MODE_ADAPTIVE || p.mode > ML_MODE_SSA_ONLY)
    return fail(ML_ERR_ARG, "unknown mode %d", p.mode);
  if (p.precision != ML_PREC_REF_FP64 && p.precision != ML_PREC_FAST_FP32)
    return fail(ML_ERR_ARG, "unknown precision %d", p.precision);
  if (p.form != ML_FORM_PLAIN && p.form != ML_FORM_PERSISTENT)
    return fail(ML_ERR_ARG, "unknown form %d", p.form);
  if (p.shape < ML_SHAPE_AUTO || p.shape > ML_SHAPE_THREAD_POOL_OCC)
    return fail(ML_ERR_ARG, "unknown shape %d", p.shape);
  if ((p.shape == ML_SHAPE_THREAD_OCC || p.shape == ML_SHAPE_THREAD_SEQ_OCC ||
       p.shape == ML_SHAPE_THREAD_POOL_OCC) &&
      p.precision != ML_PREC_FAST_FP32)
    return fail(ML_ERR_ARG, "the 128-register thread build exists in fast precision only");
  if ((p.shape == ML_SHAPE_THREAD_POOL || p.shape == ML_SHAPE_THREAD_POOL_OCC) &&
      p.form != ML_FORM_PERSISTENT)
    return fail(ML_ERR_ARG, "the pool driver runs in the persistent form only");
  if (p.block_size != 0 && (p.block_size < 32 || p.block_size > 256 || p.block_size % 32))
    return fail(ML_ERR_ARG, "block_size must be 0 or a multiple of 32 in [32, 256]");
  if (p.ctas_per_sm < 0 || p.ctas_per_sm > 32)
    return fail(ML_ERR_ARG, "ctas_per_sm must be in [0, 32]");
  if (p.jacobian != ML_JAC_FD && p.jacobian != ML_JAC_ANALYTIC)
    return fail(ML_ERR_ARG, "unknown jacobian %d", p.jacobian);
  if (p.newton_precision != ML_NEWTON_FP64 && p.newton_precision != ML_NEWTON_FP32)
    return fail(ML_ERR_ARG, "unknown newton_precision %d", p.newton_precision);
  if (p.stage_poll_limit < 0) return fail(ML_ERR_ARG, "stage_poll_limit must be >= 0");
  if (p.specialize != 0 && p.specialize != 1) return fail(ML_ERR_ARG, "specialize must be 0 or 1");
  return ML_OK;
}

int device_state(ml_model* m, DeviceState** out, int* device) {
  int d = 0;
  ML_CUDA_TRY(cudaGetDevice(&d));
  DeviceState& st = m->dev[d];
  if (st.sm_count == 0) {
    ML_CUDA_TRY(cudaDeviceGetAttribute(&st.sm_count, cudaDevAttrMultiProcessorCount, d));
  }
  *out = &st;
  *device = d;
  return ML_OK;
}

int ensure_tables(ml_model* m, DeviceState& st, int shape, int variant) {
  if (shape == ML_SHAPE_THREAD) {
    if (!st.thread_tables[variant]) {
      std::vector<uint8_t> b = thread_tables(variant, *m);
      void* d = nullptr;
      ML_CUDA_TRY(cudaMalloc(&d, b.size()));
      cudaError_t e = cudaMemcpy(d, b.data(), b.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "upload thread tables");
      }
      st.thread_tables[variant] = d;
    }
  } else if (!st.warp_tables) {
    std::vector<uint8_t> b = warp_tables(*m);
    void* d = nullptr;
    ML_CUDA_TRY(cudaMalloc(&d, b.size()));
    cudaError_t e = cudaMemcpy(d, b.data(), b.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "upload warp tables");
    }
    st.warp_tables = d;
  }
  if (!st.queues) {
    void* q = nullptr;
    ML_CUDA_TRY(cudaMalloc(&q, sizeof(unsigned long long) * kQueueSlots));
    ML_CUDA_TRY(cudaMemset(q, 0, sizeof(unsigned long long) * kQueueSlots));
    st.queues = static_cast<unsigned long long*>(q);
  }
  return ML_OK;
}

// The specialized kernel for (precision, driver, occupancy build), compiled and loaded at
// first use (model lock held).
int jit_entry(ml_model* m, int variant, int precision, int driver, bool occ,
              mlk::KernelEntry* out) {
  const int key = precision * 100 + driver * 10 + (occ ? 1 : 0);
  auto it = m->jit.find(key);
  if (it == m->jit.end()) {
    mlk::JitSpec k;
    k.NM = mlk::kThreadN[variant];
    k.MM = mlk::kThreadM[variant];
    k.N = m->N;
    k.M = m->M;
    k.ord = m->ord.data();
    k.nu = m->nu.data();
    k.rates = m->rates.data();
    k.partner = m->partner.data();
    k.isreact = m->isreact.data();
    k.hor = m->hor.data();
    k.n_pairs = m->n_pairs;
    k.precision_ref = precision == ML_PREC_REF_FP64;
    k.driver = driver;
    k.occ = occ;
    std::vector<char> cubin;
    std::string log;
    if (mlk::jit_compile(mlk::jit_source(k), k.precision_ref, &cubin, &log) != 0)
      return fail(ML_ERR_CUDA, "runtime compilation of the specialized kernel failed: %.400s",
                  log.c_str());
    JitKernel jk;
    ML_CUDA_TRY(cudaLibraryLoadData(&jk.lib, cubin.data(), nullptr, nullptr, 0, nullptr,
                                    nullptr, 0));
    cudaError_t e = cudaLibraryGetKernel(&jk.kernel, jk.lib, "ml_jit_kernel");
    if (e != cudaSuccess) {
      cudaLibraryUnload(jk.lib);
      return cuda_fail(e, "specialized kernel lookup");
    }
    jk.pool_words = mlk::lane_record_words(k.NM, k.MM, k.precision_ref);
    it = m->jit.emplace(key, jk).first;
  }
  out->launch = nullptr;  // launched through cudaLaunchKernel
  out->kernel = reinterpret_cast<const void*>(it->second.kernel);
  out->pool_words = driver == mlk::kJitPool ? it->second.pool_words : 0;
  return ML_OK;
}

struct Plan {
  bool jit = false;
  bool occ = false;
  bool seq = false;
  bool pool = false;
  bool grid_out = false;  // kernel build with time-grid output
  int shape = ML_SHAPE_THREAD;
  int variant = 0;
  mlk::KernelEntry entry{};
  const void* tables = nullptr;
  int block = 128;
  int grid = 1;
  size_t smem = 0;
};

// Chooses the kernel and launch shape for one call (model lock held).
int make_plan(ml_model* m, DeviceState& st, const ml_sim_params& p, int64_t n_traj,
              Plan* plan, bool grid_out = false) {
  int shape = p.shape;
  const int variant = thread_variant_for(*m);
  auto tk = st.tuned.find({p.precision, p.form});
  const Tuned* tuned = tk == st.tuned.end() ? nullptr : &tk->second;
  if (shape == ML_SHAPE_AUTO) {
    shape = tuned && tuned->shape ? tuned->shape
                                  : (variant >= 0 ? ML_SHAPE_THREAD : ML_SHAPE_WARP);
  }
  const int req_shape = shape;
  // a call with time-grid output runs the grid build of the sequential driver (the
  // drivers give identical results), without the occupancy bound
  const bool occ = !grid_out &&
                   (shape == ML_SHAPE_THREAD_OCC || shape == ML_SHAPE_THREAD_SEQ_OCC ||
                    shape == ML_SHAPE_THREAD_POOL_OCC) &&
                   p.precision == ML_PREC_FAST_FP32;
  const bool seq = grid_out || shape == ML_SHAPE_THREAD_SEQ || shape == ML_SHAPE_THREAD_SEQ_OCC;
  const bool pool = !grid_out && p.form == ML_FORM_PERSISTENT &&
                    (shape == ML_SHAPE_THREAD_POOL || shape == ML_SHAPE_THREAD_POOL_OCC);
  if (shape != ML_SHAPE_WARP) shape = ML_SHAPE_THREAD;
  if (shape == ML_SHAPE_THREAD && variant < 0)
    return fail(ML_ERR_UNSUPPORTED, "model %dx%d is too large for one thread per trajectory",
                m->N, m->M);
  if (shape == ML_SHAPE_WARP && !warp_fits(*m))
    return fail(ML_ERR_UNSUPPORTED, "model %dx%d is too large for the warp kernel", m->N, m->M);
  const bool jit = p.specialize && shape == ML_SHAPE_THREAD && !grid_out;
  mlk::KernelEntry entry =
      grid_out ? (shape == ML_SHAPE_THREAD ? thread_seq_grid_entry(p.precision, variant)
                                           : warp_grid_entry(p.precision))
      : shape == ML_SHAPE_THREAD
          ? (seq ? thread_seq_entry(p.precision, variant, occ)
                 : pool ? thread_pool_entry(p.precision, variant, occ)
                        : thread_entry(p.precision, variant, occ))
          : warp_entry(p.precision);
  if (jit) {
    const int rc = jit_entry(m, variant, p.precision,
                             seq ? mlk::kJitSequential : pool ? mlk::kJitPool : mlk::kJitRounds,
                             occ, &entry);
    if (rc != ML_OK) return rc;
  } else if (!entry.kernel || !entry.launch) {
    return fail(ML_ERR_UNSUPPORTED, "no kernel built for this shape and precision");
  }
  int rc = ensure_tables(m, st, shape, variant);
  if (rc != ML_OK) return rc;
  plan->shape = shape;
  plan->jit = jit;
  plan->occ = occ;
  plan->seq = seq;
  plan->pool = pool;
  plan->grid_out = grid_out;
  plan->variant = variant;
  plan->entry = entry;
  plan->tables = shape == ML_SHAPE_THREAD ? st.thread_tables[variant] : st.warp_tables;
  const bool tuned_here = tuned && tuned->shape == req_shape;
  int block = p.block_size ? p.block_size
                           : (tuned_here && tuned->block ? tuned->block
                                                         : (shape == ML_SHAPE_THREAD ? 128 : 128));
  if (plan->occ && block > 128) block = 128;  // the occupancy build is bounded to 128 threads
  if (pool) {  // the warps' trajectory records must fit in one CTA's shared memory
    const size_t per_warp = (size_t)entry.pool_words * mlk::kPoolSlots * 4;
    const int max_warps = (int)((227 * 1024 - 1024) / per_warp);
    if (max_warps < 1) return fail(ML_ERR_UNSUPPORTED, "pool records too large for shared memory");
    if (block / 32 > max_warps) block = 32 * max_warps;
  }
  const int per_cta = shape == ML_SHAPE_THREAD ? (pool ? block / 32 * mlk::kPoolSlots : block)
                                               : block / 32;  // trajectories
  plan->smem = shape == ML_SHAPE_WARP
                   ? mlk::warp_smem_bytes(block / 32, m->N, m->M, p.precision,
                                          p.newton_precision == ML_NEWTON_FP32)
               : pool ? (size_t)(block / 32) * entry.pool_words * mlk::kPoolSlots * 4
                      : 0;
  if (plan->smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(plan->entry.kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plan->smem);
    if (e != cudaSuccess) return cuda_fail(e, "set dynamic shared memory");
  }
  int64_t grid;
  if (p.form == ML_FORM_PERSISTENT) {
    int per_sm = p.ctas_per_sm ? p.ctas_per_sm
                               : (tuned_here && tuned->ctas_per_sm ? tuned->ctas_per_sm : 0);
    if (per_sm == 0) {
      int occ = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, plan->entry.kernel,
                                                                    block, plan->smem);
      if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
      per_sm = std::max(1, occ);
    }
    grid = (int64_t)st.sm_count * per_sm;
    const int64_t needed = (n_traj + per_cta - 1) / per_cta;
    grid = std::max<int64_t>(1, std::min(grid, needed));
  } else {
    grid = (n_traj + per_cta - 1) / per_cta;
    if (grid > 0x7fffffff) return fail(ML_ERR_ARG, "n_traj too large for one launch");
  }
  plan->block = block;
  plan->grid = (int)grid;
  return ML_OK;
}

void fill_args(const ml_model* m, const ml_sim_params& p, int64_t n_traj, const double* theta,
               const int64_t* x0, int32_t x0_per, const double* T, int32_t T_per,
               uint64_t seed, uint64_t id_base, int64_t* X, int64_t* r, double* G,
               uint32_t* status, int64_t* counters, mlk::SimArgs* a) {
  std::memset(a, 0, sizeof *a);
  a->n_traj = n_traj;
  a->theta = theta;
  a->x0 = x0;
  a->T = T;
  a->x0_per = x0_per ? 1 : 0;
  a->T_per = T_per ? 1 : 0;
  a->N = m->N;
  a->M = m->M;
  a->seed = seed;
  a->id_base = id_base;
  a->X = X;
  a->r = r;
  a->G = G;
  a->status = status;
  a->counters = counters;
  a->eps = p.eps;
  a->ssa_factor = p.ssa_factor;
  a->pe_delta = p.pe_delta;
  a->stiff_ratio = p.stiff_ratio;
  a->newton_tol = p.newton_tol;
  a->fd_h = p.fd_h;
  a->max_steps = p.max_steps;
  a->n_c = p.n_c;
  a->n_ssa_ex = p.n_ssa_explicit;
  a->n_ssa_im = p.n_ssa_implicit;
  a->newton_maxit = p.newton_maxit;
  a->max_reject = p.max_reject;
  a->mode = p.mode;
  a->jacobian = p.jacobian;
  a->newton_fp32 = p.precision == ML_PREC_FAST_FP32 && p.newton_precision == ML_NEWTON_FP32;
  a->stage_polls = p.stage_poll_limit;
  a->queue = nullptr;
  a->order = p.form == ML_FORM_PERSISTENT ? p.queue_order : nullptr;
}

// Launches through a cached CUDA graph {queue reset, kernel}; kernel parameters are
// updated in place when they change.
int launch_graph(DeviceState& st, const ml_sim_params& p, const Plan& plan,
                 mlk::SimArgs& a, cudaStream_t stream) {
  const int key2 = (plan.shape == ML_SHAPE_THREAD ? plan.variant + (plan.occ ? 50 : 0) +
                                                      (plan.seq ? 25 : 0) + (plan.pool ? 12 : 0)
                                                    : 100) +
                   (plan.grid_out ? 1000 : 0) + (plan.jit ? 500 : 0);
  GraphCache& gc = st.graphs[{p.precision, key2}];
  const void* tables = plan.tables;
  void* kargs[2] = {const_cast<void**>(&tables), &a};
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void*>(plan.entry.kernel);
  kp.gridDim = dim3((unsigned)plan.grid);
  kp.blockDim = dim3((unsigned)plan.block);
  kp.sharedMemBytes = (unsigned)plan.smem;
  kp.kernelParams = kargs;
  cudaMemsetParams mp;
  std::memset(&mp, 0, sizeof mp);
  mp.dst = a.queue;
  mp.elementSize = 4;
  mp.width = 2;
  mp.height = 1;
  mp.pitch = 8;
  mp.value = 0;
  if (!gc.exec) {
    ML_CUDA_TRY(cudaGraphCreate(&gc.graph, 0));
    ML_CUDA_TRY(cudaGraphAddMemsetNode(&gc.memset_node, gc.graph, nullptr, 0, &mp));
    ML_CUDA_TRY(cudaGraphAddKernelNode(&gc.kernel_node, gc.graph, &gc.memset_node, 1, &kp));
    ML_CUDA_TRY(cudaGraphInstantiate(&gc.exec, gc.graph, 0));
  } else {
    ML_CUDA_TRY(cudaGraphExecMemsetNodeSetParams(gc.exec, gc.memset_node, &mp));
    ML_CUDA_TRY(cudaGraphExecKernelNodeSetParams(gc.exec, gc.kernel_node, &kp));
  }
  ML_CUDA_TRY(cudaGraphLaunch(gc.exec, stream));
  return ML_OK;
}

int run_plan(ml_model* m, DeviceState& st, const ml_sim_params& p, const Plan& plan,
             mlk::SimArgs& a, cudaStream_t stream) {
  if (p.form == ML_FORM_PERSISTENT) {
    a.queue = st.queues + (st.next_slot++ % kQueueSlots);
    if (p.use_graph) {
      int rc = launch_graph(st, p, plan, a, stream);
      if (rc == ML_OK) m->last_launches = 1;
      return rc;
    }
    ML_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), stream));
  }
  cudaError_t e;
  if (plan.entry.launch) {
    e = plan.entry.launch(plan.tables, a, plan.grid, plan.block, plan.smem, stream);
  } else {  // a specialized kernel: same parameters (tables, SimArgs)
    const void* tables = plan.tables;
    void* kargs[2] = {const_cast<void**>(&tables), &a};
    e = cudaLaunchKernel(plan.entry.kernel, dim3((unsigned)plan.grid), dim3((unsigned)plan.block),
                         kargs, plan.smem, stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  m->last_launches = 1;
  return ML_OK;
}

int check_sizes(const ml_model* m, int64_t n_traj, uint64_t id_base) {
  if (!m) return fail(ML_ERR_ARG, "model is NULL");
  if (n_traj < 0) return fail(ML_ERR_ARG, "n_traj must be >= 0");
  if (id_base > 0xffffffffULL || (uint64_t)n_traj > 0x100000000ULL - id_base)
    return fail(ML_ERR_ARG, "trajectory ids traj_id_base + i must stay below 2^32");
  return ML_OK;
}

}  // namespace

namespace mlk {

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int noalloc_prepare(const ml_model* m, int64_t n_traj, const double* theta, const int64_t* x0,
                    int32_t x0_per_traj, const double* T, int32_t T_per_traj,
                    const void* params, uint64_t seed, uint64_t id_base, int64_t* X,
                    int64_t* r, double* G, uint32_t* status, int64_t* counters,
                    size_t scratch_table_max, NoAllocLaunch* out) {
  int rc = check_sizes(m, n_traj, id_base);
  if (rc != ML_OK) return rc;
  ml_sim_params p;
  if (params) p = *static_cast<const ml_sim_params*>(params);
  else ml_default_params(&p);
  p.form = ML_FORM_PERSISTENT;
  p.use_graph = 0;
  rc = check_params(p);
  if (rc != ML_OK) return rc;
  const size_t need = m->thread_variant >= 0 ? m->host_thread_tables.size() : m->warp_table_bytes;
  if (m->thread_variant < 0 || need > scratch_table_max)
    return fail(ML_ERR_ARG,
                "model %dx%d needs %zu bytes of model tables; the allocation-free entry point "
                "holds at most %zu (one trajectory per thread: at most 8 species and 16 "
                "reactions)",
                m->N, m->M, need, scratch_table_max);
  if (p.shape == ML_SHAPE_WARP)
    return fail(ML_ERR_UNSUPPORTED, "the allocation-free entry point runs one trajectory per thread only");
  const struct {
    const void* ptr;
    const char* name;
    bool required;
  } ptrs[] = {{theta, "theta", false}, {x0, "x0", true},      {T, "T", true},
              {X, "X_out", true},      {r, "r_out", true},    {G, "G_out", true},
              {status, "status_out", true}, {counters, "counters_out", false},
              {p.queue_order, "queue_order", false}};
  if (n_traj > 0) {
    for (const auto& q : ptrs) {
      if (!q.ptr) {
        if (q.required) return fail(ML_ERR_ARG, "%s is NULL", q.name);
        continue;
      }
      if (!is_device_pointer(q.ptr))
        return fail(ML_ERR_ARG, "%s is not device memory of the current device", q.name);
    }
  }
  int dev = 0, sms = 0;
  ML_CUDA_TRY(cudaGetDevice(&dev));
  ML_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  out->entry = thread_entry(p.precision, m->thread_variant);
  if (!out->entry.kernel) return fail(ML_ERR_UNSUPPORTED, "no kernel built for this precision");
  out->host_tables = m->host_thread_tables.data();
  out->table_bytes = m->host_thread_tables.size();
  const int block = p.block_size ? p.block_size : 128;
  int per_sm = p.ctas_per_sm;
  if (per_sm == 0) {
    int occ = 0;
    ML_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, out->entry.kernel, block, 0));
    per_sm = occ > 0 ? occ : 1;
  }
  int64_t grid = (int64_t)sms * per_sm;
  const int64_t needed = (n_traj + block - 1) / block;
  grid = std::max<int64_t>(1, std::min(grid, needed));
  out->grid = (int)grid;
  out->block = block;
  fill_args(m, p, n_traj, theta, x0, x0_per_traj, T, T_per_traj, seed, id_base, X, r, G,
            status, counters, &out->args);
  return ML_OK;
}

}  // namespace mlk

extern "C" {

int ml_default_params(ml_sim_params* p) {
  if (!p) return fail(ML_ERR_ARG, "params is NULL");
  std::memset(p, 0, sizeof *p);
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
  p->mode = ML_MODE_ADAPTIVE;
  p->precision = ML_PREC_REF_FP64;
  p->form = ML_FORM_PLAIN;
  p->shape = ML_SHAPE_AUTO;
  p->block_size = 0;
  p->ctas_per_sm = 0;
  p->use_graph = 0;
  p->jacobian = ML_JAC_FD;
  p->newton_precision = ML_NEWTON_FP64;
  p->stage_poll_limit = 1 << 22;
  return ML_OK;
}

const char* ml_last_error(void) { return g_last_error.c_str(); }

int ml_model_create(int32_t N, int32_t M, const int32_t* ord, const int32_t* nu,
                    const double* rates, ml_model** out) {
  if (!out) return fail(ML_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (N < 1 || M < 1 || N > mlk::kWarpMaxN || M > mlk::kWarpMaxM)
    return fail(ML_ERR_ARG, "need 1 <= N <= %d and 1 <= M <= %d", mlk::kWarpMaxN,
                mlk::kWarpMaxM);
  if (!ord || !nu || !rates) return fail(ML_ERR_ARG, "model arrays must not be NULL");
  std::unique_ptr<ml_model> m(new (std::nothrow) ml_model);
  if (!m) return fail(ML_ERR_OOM, "host allocation failed");
  m->N = N;
  m->M = M;
  m->ord.assign(ord, ord + (size_t)N * M);
  m->nu.assign(nu, nu + (size_t)N * M);
  m->rates.assign(rates, rates + M);
  m->otot.assign(M, 0);
  m->isreact.assign(N, 0);
  m->hor.assign(N, 0);
  for (int j = 0; j < M; ++j) {
    if (!(rates[j] >= 0.0) || !std::isfinite(rates[j]))
      return fail(ML_ERR_ARG, "rate %d must be finite and >= 0", j);
    int tot = 0;
    for (int s = 0; s < N; ++s) {
      const int o = ord[j * N + s], v = nu[j * N + s];
      if (o < 0) return fail(ML_ERR_ARG, "reaction %d: negative order", j);
      if (v < -o) return fail(ML_ERR_ARG, "reaction %d consumes more of species %d than it uses", j, s);
      if (v > 127 || v < -127) return fail(ML_ERR_ARG, "reaction %d: |nu| > 127", j);
      tot += o;
    }
    if (tot > 3) return fail(ML_ERR_ARG, "reaction %d has order %d > 3", j, tot);
    m->otot[j] = tot;
  }
  // highest-order-reaction flags (Cao 2006) of every consumed species
  for (int j = 0; j < M; ++j) {
    for (int s = 0; s < N; ++s) {
      const int o = ord[j * N + s];
      if (o == 0) continue;
      m->isreact[s] = 1;
      const int tot = m->otot[j];
      uint8_t f;
      if (tot == 1) f = mlk::kHorO1;
      else if (tot == 2) f = o == 1 ? mlk::kHorO2M1 : mlk::kHorO2M2;
      else f = o == 1 ? mlk::kHorO3M1 : (o == 2 ? mlk::kHorO3M2 : mlk::kHorO3M3);
      m->hor[s] |= f;
    }
  }
  // reversible pairs: k is the chemical reverse of j (reactants of k = products of j and
  // the other way round), both have a reactant; lowest unpaired partner, in index order
  m->partner.assign(M, -1);
  for (int j = 0; j < M; ++j) {
    if (m->partner[j] >= 0 || m->otot[j] == 0) continue;
    bool moves = false;
    for (int s = 0; s < N; ++s) moves = moves || nu[j * N + s] != 0;
    if (!moves) continue;
    for (int k = j + 1; k < M; ++k) {
      if (m->partner[k] >= 0 || m->otot[k] == 0) continue;
      bool rev = true;
      for (int s = 0; s < N && rev; ++s) {
        const int pj = ord[j * N + s] + nu[j * N + s];  // products of j
        const int pk = ord[k * N + s] + nu[k * N + s];  // products of k
        rev = ord[k * N + s] == pj && ord[j * N + s] == pk;
      }
      if (rev) {
        m->partner[j] = k;
        m->partner[k] = j;
        m->n_pairs++;
        break;
      }
    }
  }
  m->thread_variant = thread_variant_for(*m);
  if (m->thread_variant >= 0) m->host_thread_tables = thread_tables(m->thread_variant, *m);
  m->warp_table_bytes = (sizeof(mlk::WarpModel) + 15) / 16 * 16;
  *out = m.release();
  return ML_OK;
}

int ml_model_destroy(ml_model* m) {
  if (!m) return ML_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : m->dev) {
    cudaSetDevice(kv.first);
    DeviceState& st = kv.second;
    for (auto& g : st.graphs) {
      if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
      if (g.second.graph) cudaGraphDestroy(g.second.graph);
    }
    for (void* t : st.thread_tables)
      if (t) cudaFree(t);
    if (st.warp_tables) cudaFree(st.warp_tables);
    if (st.queues) cudaFree(st.queues);
    if (st.ws) cudaFree(st.ws);
  }
  cudaSetDevice(cur);
  for (auto& kv : m->jit)
    if (kv.second.lib) cudaLibraryUnload(kv.second.lib);
  delete m;
  return ML_OK;
}

int ml_model_num_species(const ml_model* m) {
  if (!m) return fail(ML_ERR_ARG, "model is NULL");
  return m->N;
}

int ml_model_num_reactions(const ml_model* m) {
  if (!m) return fail(ML_ERR_ARG, "model is NULL");
  return m->M;
}

int ml_model_num_pairs(const ml_model* m) {
  if (!m) return fail(ML_ERR_ARG, "model is NULL");
  return m->n_pairs;
}

int64_t ml_model_last_launch_count(const ml_model* m) {
  if (!m) return fail(ML_ERR_ARG, "model is NULL");
  return m->last_launches;
}

int ml_simulate(const ml_model* cm, int64_t n_traj, const double* theta, const int64_t* x0,
                int32_t x0_per_traj, const double* T, int32_t T_per_traj,
                const ml_sim_params* pp, uint64_t seed, uint64_t id_base, int64_t* X,
                int64_t* r, double* G, uint32_t* status, int64_t* counters, void* stream) {
  return ml_simulate_grid(cm, n_traj, theta, x0, x0_per_traj, T, T_per_traj, pp, seed, id_base,
                          nullptr, 0, nullptr, X, r, G, status, counters, stream);
}

int ml_simulate_grid(const ml_model* cm, int64_t n_traj, const double* theta,
                     const int64_t* x0, int32_t x0_per_traj, const double* T,
                     int32_t T_per_traj, const ml_sim_params* pp, uint64_t seed,
                     uint64_t id_base, const double* t_obs, int32_t K, int64_t* X_obs,
                     int64_t* X, int64_t* r, double* G, uint32_t* status, int64_t* counters,
                     void* stream) {
  int rc = check_sizes(cm, n_traj, id_base);
  if (rc != ML_OK) return rc;
  if (K < 0) return fail(ML_ERR_ARG, "K must be >= 0");
  if (K > 0 && n_traj > 0) {
    if (!t_obs || !X_obs) return fail(ML_ERR_ARG, "t_obs and X_obs must not be NULL when K > 0");
    if (!is_device_pointer(t_obs) || !is_device_pointer(X_obs))
      return fail(ML_ERR_ARG, "t_obs and X_obs must be device memory of the current device");
  }
  ml_model* m = const_cast<ml_model*>(cm);
  ml_sim_params p;
  if (pp) p = *pp;
  else ml_default_params(&p);
  rc = check_params(p);
  if (rc != ML_OK) return rc;
  std::lock_guard<std::mutex> lk(m->mu);
  m->last_launches = 0;
  if (n_traj == 0) return ML_OK;
  const struct {
    const void* ptr;
    const char* name;
    bool required;
  } ptrs[] = {{theta, "theta", false}, {x0, "x0", true},      {T, "T", true},
              {X, "X_out", true},      {r, "r_out", true},    {G, "G_out", true},
              {status, "status_out", true}, {counters, "counters_out", false},
              {p.form == ML_FORM_PERSISTENT ? p.queue_order : nullptr, "queue_order", false}};
  for (const auto& q : ptrs) {
    if (!q.ptr) {
      if (q.required) return fail(ML_ERR_ARG, "%s is NULL", q.name);
      continue;
    }
    if (!is_device_pointer(q.ptr))
      return fail(ML_ERR_ARG, "%s is not device memory of the current device", q.name);
  }
  DeviceState* st = nullptr;
  int dev = 0;
  rc = device_state(m, &st, &dev);
  if (rc != ML_OK) return rc;
  Plan plan;
  rc = make_plan(m, *st, p, n_traj, &plan, K > 0 && n_traj > 0);
  if (rc != ML_OK) return rc;
  mlk::SimArgs a;
  fill_args(m, p, n_traj, theta, x0, x0_per_traj, T, T_per_traj, seed, id_base, X, r, G,
            status, counters, &a);
  if (K > 0) {
    a.t_obs = t_obs;
    a.X_obs = X_obs;
    a.K_obs = K;
  }
  return run_plan(m, *st, p, plan, a, static_cast<cudaStream_t>(stream));
}

int ml_simulate_host(ml_model* m, int64_t n_traj, const double* theta, const int64_t* x0,
                     int32_t x0_per_traj, const double* T, int32_t T_per_traj,
                     const ml_sim_params* pp, uint64_t seed, uint64_t id_base, int64_t* X,
                     int64_t* r, double* G, uint32_t* status, int64_t* counters,
                     void* stream_v) {
  int rc = check_sizes(m, n_traj, id_base);
  if (rc != ML_OK) return rc;
  if (!x0 || !T || !X || !r || !G || !status)
    return fail(ML_ERR_ARG, "x0, T, X_out, r_out, G_out and status_out must not be NULL");
  if (n_traj == 0) return ML_OK;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  const size_t N = (size_t)m->N, M = (size_t)m->M, n = (size_t)n_traj;
  auto up16 = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_theta = theta ? up16(n * M * 8) : 0;
  const size_t b_x0 = up16((x0_per_traj ? n : 1) * N * 8);
  const size_t b_T = up16((T_per_traj ? n : 1) * 8);
  const size_t b_X = up16(n * N * 8), b_r = up16(n * M * 8), b_G = up16(n * M * 8);
  const size_t b_st = up16(n * 4), b_c = counters ? up16(n * 32) : 0;
  ml_sim_params pq;
  if (pp) pq = *pp;
  else ml_default_params(&pq);
  const bool ordered = pq.queue_order && pq.form == ML_FORM_PERSISTENT;
  const size_t b_ord = ordered ? up16(n * 8) : 0;
  const size_t total = b_theta + b_x0 + b_T + b_X + b_r + b_G + b_st + b_c + b_ord;
  DeviceState* st = nullptr;
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    int dev = 0;
    rc = device_state(m, &st, &dev);
    if (rc != ML_OK) return rc;
    if (st->host_busy) return fail(ML_ERR_BUSY, "ml_simulate_host already running on this model");
    if (st->ws_bytes < total) {
      if (st->ws) {
        cudaStreamSynchronize(stream);
        cudaFree(st->ws);
        st->ws = nullptr;
        st->ws_bytes = 0;
      }
      ML_CUDA_TRY(cudaMalloc(&st->ws, total));
      st->ws_bytes = total;
    }
    st->host_busy = true;
    base = static_cast<char*>(st->ws);
  }
  struct Release {
    ml_model* m;
    DeviceState* st;
    ~Release() {
      std::lock_guard<std::mutex> lk(m->mu);
      st->host_busy = false;
    }
  } release{m, st};
  char* p = base;
  double* d_theta = theta ? reinterpret_cast<double*>(p) : nullptr;
  p += b_theta;
  int64_t* d_x0 = reinterpret_cast<int64_t*>(p);
  p += b_x0;
  double* d_T = reinterpret_cast<double*>(p);
  p += b_T;
  int64_t* d_X = reinterpret_cast<int64_t*>(p);
  p += b_X;
  int64_t* d_r = reinterpret_cast<int64_t*>(p);
  p += b_r;
  double* d_G = reinterpret_cast<double*>(p);
  p += b_G;
  uint32_t* d_st = reinterpret_cast<uint32_t*>(p);
  p += b_st;
  int64_t* d_c = counters ? reinterpret_cast<int64_t*>(p) : nullptr;
  p += b_c;
  if (ordered) {
    int64_t* d_ord = reinterpret_cast<int64_t*>(p);
    ML_CUDA_TRY(cudaMemcpyAsync(d_ord, pq.queue_order, n * 8, cudaMemcpyHostToDevice, stream));
    pq.queue_order = d_ord;
  }
  if (theta) ML_CUDA_TRY(cudaMemcpyAsync(d_theta, theta, n * M * 8, cudaMemcpyHostToDevice, stream));
  ML_CUDA_TRY(cudaMemcpyAsync(d_x0, x0, (x0_per_traj ? n : 1) * N * 8, cudaMemcpyHostToDevice, stream));
  ML_CUDA_TRY(cudaMemcpyAsync(d_T, T, (T_per_traj ? n : 1) * 8, cudaMemcpyHostToDevice, stream));
  rc = ml_simulate(m, n_traj, d_theta, d_x0, x0_per_traj, d_T, T_per_traj, &pq, seed, id_base,
                   d_X, d_r, d_G, d_st, d_c, stream);
  if (rc != ML_OK) return rc;
  ML_CUDA_TRY(cudaMemcpyAsync(X, d_X, n * N * 8, cudaMemcpyDeviceToHost, stream));
  ML_CUDA_TRY(cudaMemcpyAsync(r, d_r, n * M * 8, cudaMemcpyDeviceToHost, stream));
  ML_CUDA_TRY(cudaMemcpyAsync(G, d_G, n * M * 8, cudaMemcpyDeviceToHost, stream));
  ML_CUDA_TRY(cudaMemcpyAsync(status, d_st, n * 4, cudaMemcpyDeviceToHost, stream));
  if (counters) ML_CUDA_TRY(cudaMemcpyAsync(counters, d_c, n * 32, cudaMemcpyDeviceToHost, stream));
  ML_CUDA_TRY(cudaStreamSynchronize(stream));
  return ML_OK;
}

int ml_autotune(ml_model* m, int64_t n_traj, const double* theta, const int64_t* x0,
                int32_t x0_per_traj, const double* T, int32_t T_per_traj,
                const ml_sim_params* pp, uint64_t seed, int64_t n_sample, ml_sim_params* best,
                void* stream_v) {
  int rc = check_sizes(m, n_traj, 0);
  if (rc != ML_OK) return rc;
  ml_sim_params p;
  if (pp) p = *pp;
  else ml_default_params(&p);
  rc = check_params(p);
  if (rc != ML_OK) return rc;
  const int64_t n = std::min(n_traj, std::max<int64_t>(n_sample, 1));
  if (n <= 0) return fail(ML_ERR_ARG, "nothing to tune on");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  const size_t N = (size_t)m->N, M = (size_t)m->M;
  void* out = nullptr;
  const size_t bytes = (size_t)n * (N * 8 + M * 16 + 4 + 32) + 1024;
  ML_CUDA_TRY(cudaMalloc(&out, bytes));
  char* q = static_cast<char*>(out);
  int64_t* X = reinterpret_cast<int64_t*>(q);
  int64_t* r = X + n * N;
  double* G = reinterpret_cast<double*>(r + n * M);
  int64_t* cnt = reinterpret_cast<int64_t*>(G + n * M);
  uint32_t* stt = reinterpret_cast<uint32_t*>(cnt + n * 4);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int thread_ok = thread_variant_for(*m) >= 0;
  const int warp_ok = warp_fits(*m);
  std::vector<ml_sim_params> cands;
  for (int shape = ML_SHAPE_THREAD; shape <= ML_SHAPE_THREAD_POOL_OCC; ++shape) {
    const bool thread_like = shape != ML_SHAPE_WARP;
    const bool occ_shape = shape == ML_SHAPE_THREAD_OCC || shape == ML_SHAPE_THREAD_SEQ_OCC ||
                           shape == ML_SHAPE_THREAD_POOL_OCC;
    const bool pool_shape = shape == ML_SHAPE_THREAD_POOL || shape == ML_SHAPE_THREAD_POOL_OCC;
    if ((thread_like && !thread_ok) || (shape == ML_SHAPE_WARP && !warp_ok)) continue;
    if (occ_shape && p.precision != ML_PREC_FAST_FP32) continue;
    if (pool_shape && p.form != ML_FORM_PERSISTENT) continue;
    if (p.shape != ML_SHAPE_AUTO && p.shape != shape) continue;
    const int blocks[] = {64, 128, 256};
    for (int b : blocks) {
      if (occ_shape && b > 128) continue;
      // a model that fits one thread tries the warp kernel in one launch shape only
      if (shape == ML_SHAPE_WARP && thread_ok && b != 128) continue;
      // CTAs per SM beyond what can be resident at once only queue behind the others
      int resident = 0;
      {
        ml_sim_params q = p;
        q.shape = shape;
        q.block_size = b;
        q.ctas_per_sm = 0;
        std::lock_guard<std::mutex> lk(m->mu);
        DeviceState* st = nullptr;
        int dev = 0;
        Plan plan;
        if (device_state(m, &st, &dev) == ML_OK && make_plan(m, *st, q, n, &plan) == ML_OK)
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, plan.entry.kernel, b,
                                                        plan.smem);
      }
      const int per_sm_opts[] = {0, 1, 2, 4};
      for (int per_sm : per_sm_opts) {
        if (p.form != ML_FORM_PERSISTENT && per_sm != 0) continue;
        if (shape == ML_SHAPE_WARP && thread_ok && per_sm != 0) continue;
        if (per_sm > 0 && resident > 0 && per_sm >= resident) continue;  // 0 covers it
        ml_sim_params c = p;
        c.shape = shape;
        c.block_size = b;
        c.ctas_per_sm = per_sm;
        c.use_graph = 0;
        // an order is a permutation of the whole batch: used only when tuning on all of it
        c.queue_order = n == n_traj ? p.queue_order : nullptr;
        cands.push_back(c);
      }
    }
  }
  // Candidates run in a fixed order; each is timed kTimed times after one warm-up and
  // scored by the median.  A later candidate replaces the incumbent only if it is more
  // than 3 % faster, so run-to-run noise does not flip the choice between near-equal
  // shapes.  A candidate whose warm-up run takes more than twice the incumbent's median
  // is not timed further.
  constexpr int kTimed = 3;
  float best_ms = 1e30f;
  ml_sim_params best_p = p;
  for (const ml_sim_params& c : cands) {
    float t_rep[kTimed];
    bool ok = true;
    for (int rep = 0; rep <= kTimed && ok; ++rep) {
      cudaEventRecord(e0, stream);
      int r2 = ml_simulate(m, n, theta, x0, x0_per_traj, T, T_per_traj, &c, seed, 0, X, r, G,
                           stt, cnt, stream);
      if (r2 != ML_OK) ok = false;
      if (ok) {
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          cudaFree(out);
          return cuda_fail(cudaGetLastError(), "autotune run");
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep == 0 && t > 2.f * best_ms) ok = false;  // clearly slower: not timed further
        if (rep > 0) t_rep[rep - 1] = t;
      }
    }
    if (!ok) continue;
    std::sort(t_rep, t_rep + kTimed);
    const float ms = t_rep[kTimed / 2];
    if (ms < 0.97f * best_ms) {
      best_ms = ms;
      best_p = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (best_ms >= 1e30f) return fail(ML_ERR_CUDA, "no autotune candidate ran: %s", g_last_error.c_str());
  {
    std::lock_guard<std::mutex> lk(m->mu);
    DeviceState* st = nullptr;
    int dev = 0;
    rc = device_state(m, &st, &dev);
    if (rc != ML_OK) return rc;
    Tuned t;
    t.shape = best_p.shape;
    t.block = best_p.block_size;
    t.ctas_per_sm = best_p.ctas_per_sm;
    st->tuned[{p.precision, p.form}] = t;
  }
  if (best) {
    *best = best_p;
    best->use_graph = p.use_graph;
    best->queue_order = p.queue_order;
  }
  return ML_OK;
}

}  // extern "C"
