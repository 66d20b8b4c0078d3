// One-trajectory-per-warp kernel for one arithmetic:
//   ML_FAST = 0: reference precision (compile with -fmad=false), 1: fast precision;
//   each with and without time-grid output.
#include "warp_core.cuh"

namespace mlk {
#if ML_FAST
using WPrec = PrecFast;
#else
using WPrec = PrecRef;
#endif

namespace {
cudaError_t launch(const void* dm, const SimArgs& a, int grid, int block, size_t smem,
                   cudaStream_t s) {
  k_warp<WPrec><<<grid, block, smem, s>>>(static_cast<const WarpModel*>(dm), a);
  return cudaGetLastError();
}
cudaError_t launch_grid(const void* dm, const SimArgs& a, int grid, int block, size_t smem,
                        cudaStream_t s) {
  k_warp<WPrec, true><<<grid, block, smem, s>>>(static_cast<const WarpModel*>(dm), a);
  return cudaGetLastError();
}
}  // namespace

#if ML_FAST
KernelEntry warp_entry_fast() {
  return KernelEntry{&launch, reinterpret_cast<const void*>(&k_warp<WPrec>)};
}
KernelEntry warp_grid_entry_fast() {
  return KernelEntry{&launch_grid, reinterpret_cast<const void*>(&k_warp<WPrec, true>)};
}
#else
KernelEntry warp_entry_ref() {
  return KernelEntry{&launch, reinterpret_cast<const void*>(&k_warp<WPrec>)};
}
KernelEntry warp_grid_entry_ref() {
  return KernelEntry{&launch_grid, reinterpret_cast<const void*>(&k_warp<WPrec, true>)};
}
size_t warp_smem_bytes(int warps, int N, int M, int precision, bool newton_fp32) {
  const bool fast = precision == ML_PREC_FAST_FP32;
  const int rbytes = fast ? 4 : 8;
  const int lbytes = fast && newton_fp32 ? 4 : 8;
  return (sizeof(WarpModel) + 15) / 16 * 16 + (size_t)warps * warp_slab_bytes(N, M, rbytes, lbytes);
}
#endif
}  // namespace mlk
