// One trajectory per warp (large networks).  Not built yet: the entries are empty and
// the host API reports such models as unsupported.
#include "ml_internal.h"

namespace mlk {
#if ML_FAST
KernelEntry warp_entry_fast() { return KernelEntry{nullptr, nullptr}; }
#else
KernelEntry warp_entry_ref() { return KernelEntry{nullptr, nullptr}; }
size_t warp_smem_bytes(int) { return 0; }
#endif
}  // namespace mlk
