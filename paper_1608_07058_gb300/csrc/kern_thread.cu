// One thread-per-trajectory kernel variant, selected at compile time:
//   ML_FAST = 0: reference precision (compile with -fmad=false), 1: fast precision;
//   ML_VARIANT: index into the (species, reactions) capacity table;
//   ML_THREAD_MIN_BLOCKS = 2 (fast only): the occupancy build (at most 128 threads per
//   CTA, about 168 registers, more resident warps, some spilling), offered to the
//   autotuner as a separate shape.  The plain builds also carry the sequential driver
//   with time-grid output.
//   ML_PART (optional): build only the round-based driver (0), the sequential driver (1),
//   its time-grid build (2) or the pool driver (3) of this variant, so that the large
//   generic variant's kernels compile in parallel units; unset, the unit holds all of them.
#include "thread_core.cuh"

#ifndef ML_PART
#define ML_PART -1
#endif
#define ML_HAS_PART(k) (ML_PART < 0 || ML_PART == (k))

#ifndef ML_VARIANT
#error "ML_VARIANT must be defined"
#endif
#define ML_CAT_(a, b, c) a##b##_##c
#define ML_CAT(a, b, c) ML_CAT_(a, b, c)

namespace mlk {
#if ML_FAST && ML_THREAD_MIN_BLOCKS == 2
using Prec = PrecFast;
#define ML_PNAME fastocc
#elif ML_FAST
using Prec = PrecFast;
#define ML_PNAME fast
#else
using Prec = PrecRef;
#define ML_PNAME ref
#endif

namespace {
constexpr int kNM = kThreadN[ML_VARIANT];
constexpr int kMM = kThreadM[ML_VARIANT];
#if ML_HAS_PART(0)
cudaError_t launch(const void* dm, const SimArgs& a, int grid, int block, size_t smem,
                   cudaStream_t s) {
  k_thread<kNM, kMM, Prec><<<grid, block, smem, s>>>(
      static_cast<const ThreadModel<kNM, kMM>*>(dm), a);
  return cudaGetLastError();
}
#endif
#if ML_HAS_PART(1)
cudaError_t launch_seq(const void* dm, const SimArgs& a, int grid, int block, size_t smem,
                       cudaStream_t s) {
  k_thread_seq<kNM, kMM, Prec><<<grid, block, smem, s>>>(
      static_cast<const ThreadModel<kNM, kMM>*>(dm), a);
  return cudaGetLastError();
}
#endif
#if ML_HAS_PART(3)
cudaError_t launch_pool(const void* dm, const SimArgs& a, int grid, int block, size_t smem,
                        cudaStream_t s) {
  k_thread_pool<kNM, kMM, Prec><<<grid, block, smem, s>>>(
      static_cast<const ThreadModel<kNM, kMM>*>(dm), a);
  return cudaGetLastError();
}
#endif
#if !(ML_FAST && ML_THREAD_MIN_BLOCKS == 2) && ML_HAS_PART(2)
cudaError_t launch_seq_grid(const void* dm, const SimArgs& a, int grid, int block, size_t smem,
                            cudaStream_t s) {
  k_thread_seq<kNM, kMM, Prec, true><<<grid, block, smem, s>>>(
      static_cast<const ThreadModel<kNM, kMM>*>(dm), a);
  return cudaGetLastError();
}
#endif
}  // namespace

#if !(ML_FAST && ML_THREAD_MIN_BLOCKS == 2) && ML_HAS_PART(2)
KernelEntry ML_CAT(thread_seq_grid_entry_, ML_PNAME, ML_VARIANT)() {
  return KernelEntry{&launch_seq_grid,
                     reinterpret_cast<const void*>(&k_thread_seq<kNM, kMM, Prec, true>)};
}
#endif
#if ML_HAS_PART(0)
KernelEntry ML_CAT(thread_entry_, ML_PNAME, ML_VARIANT)() {
  return KernelEntry{&launch, reinterpret_cast<const void*>(&k_thread<kNM, kMM, Prec>)};
}
#endif
#if ML_HAS_PART(3)
KernelEntry ML_CAT(thread_pool_entry_, ML_PNAME, ML_VARIANT)() {
  return KernelEntry{&launch_pool, reinterpret_cast<const void*>(&k_thread_pool<kNM, kMM, Prec>),
                     ThreadLane<kNM, kMM, Prec>::kWords};
}
#endif
#if ML_HAS_PART(1)
KernelEntry ML_CAT(thread_seq_entry_, ML_PNAME, ML_VARIANT)() {
  return KernelEntry{&launch_seq, reinterpret_cast<const void*>(&k_thread_seq<kNM, kMM, Prec>)};
}
#endif
}  // namespace mlk
