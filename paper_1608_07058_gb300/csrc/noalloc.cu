// Allocation-free simulate entry point (ml_simulate_noalloc).
//
// Some callers cannot let a library call cudaMalloc: code that runs under a device-memory
// pool owned by a host framework (a deep-learning runtime or an MPS client with a fixed
// memory cap), latency-bound loops for which cudaMalloc's implicit synchronization and
// unbounded cost are not acceptable, and code that must not take the CUDA allocator's
// lock.  For them this file keeps the only scratch the persistent kernel needs -- its
// work-queue counter and a copy of the model tables -- in a fixed device array instead of
// memory allocated on first use.  The caller still passes all inputs and outputs.
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "matleap.h"
#include "ml_internal.h"

namespace {

// Scratch layout: [0, 8) work-queue counter; [256, 4096) model tables.  Every GPU that
// loads the library holds these 4 KiB until the process exits.
constexpr size_t kScratchBytes = 4096;
constexpr size_t kTablesOffset = 256;
// The largest one-trajectory-per-thread table set (8 species x 16 reactions) is 944 bytes.
constexpr size_t kTableParamBytes = 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The model tables travel by value as a kernel parameter: the upload reads no pageable
// host memory, needs no copy engine and allocates nothing, and like the simulation launch
// after it, it is one kernel launch on the caller's stream.
struct TableParam {
  alignas(16) unsigned char b[kTableParamBytes];
};

// One CTA: zero the work-queue counter and write the tables behind it.
__global__ void k_noalloc_setup(unsigned char* scratch, const TableParam t, uint32_t bytes) {
  if (threadIdx.x == 0) *reinterpret_cast<unsigned long long*>(scratch) = 0ULL;
  for (uint32_t k = threadIdx.x; k < bytes; k += blockDim.x) scratch[kTablesOffset + k] = t.b[k];
}

// Device address of the scratch array for the current device's context (the array's name
// in host code is only a stand-in).  Looked up on every call: it is cheap, allocates
// nothing, and stays right if the context is re-created.  The first lookup on a device
// loads this module there.
int scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return mlk::set_error(ML_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
  *out = static_cast<unsigned char*>(p);
  return ML_OK;
}

}  // namespace

extern "C" int ml_simulate_noalloc(const ml_model* model, int64_t n_traj, const double* theta,
                                   const int64_t* x0, int32_t x0_per_traj, const double* T,
                                   int32_t T_per_traj, const ml_sim_params* p, uint64_t seed,
                                   uint64_t traj_id_base, int64_t* X_out, int64_t* r_out,
                                   double* G_out, uint32_t* status_out, int64_t* counters_out,
                                   void* cuda_stream) {
  mlk::NoAllocLaunch L;
  int rc = mlk::noalloc_prepare(model, n_traj, theta, x0, x0_per_traj, T, T_per_traj, p, seed,
                                traj_id_base, X_out, r_out, G_out, status_out, counters_out,
                                kTableParamBytes, &L);
  if (rc != ML_OK) return rc;
  if (n_traj == 0) return ML_OK;
  unsigned char* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != ML_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // The array keeps the previous call's contents: rewrite the tables and zero the counter.
  TableParam tp;
  std::memset(&tp, 0, sizeof tp);
  std::memcpy(tp.b, L.host_tables, L.table_bytes);
  k_noalloc_setup<<<1, 128, 0, s>>>(scratch, tp, (uint32_t)L.table_bytes);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mlk::set_error(ML_ERR_CUDA, cudaGetErrorString(e));
  L.args.queue = reinterpret_cast<unsigned long long*>(scratch);
  e = L.entry.launch(scratch + kTablesOffset, L.args, L.grid, L.block, 0, s);
  if (e != cudaSuccess) return mlk::set_error(ML_ERR_CUDA, cudaGetErrorString(e));
  return ML_OK;
}
