// Model-specialized kernels (jit.cu): source generation and runtime compilation.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace mlk {

enum : int { kJitRounds = 0, kJitPool = 1, kJitSequential = 2 };

// What one specialized kernel is built for: the thread variant's capacities, the model
// (row-major [M][N] orders and net changes, rates, reversible partner of each reaction or
// -1, reactant flags and step-size flags per species, number of pairs), the arithmetic,
// the driver and the register budget (occupancy build).
struct JitSpec {
  int NM = 0, MM = 0;
  int N = 0, M = 0;
  const int32_t* ord = nullptr;
  const int32_t* nu = nullptr;
  const double* rates = nullptr;
  const int32_t* partner = nullptr;
  const uint8_t* isreact = nullptr;
  const uint8_t* hor = nullptr;
  int n_pairs = 0;
  bool precision_ref = false;
  int driver = kJitRounds;
  bool occ = false;
};

// CUDA source of the kernel `ml_jit_kernel(const void* tables, SimArgs)` for spec k.
std::string jit_source(const JitSpec& k);

// Compiles the source for sm_103a; 0 and the cubin on success, -1 and the log otherwise.
int jit_compile(const std::string& src, bool precision_ref, std::vector<char>* cubin,
                std::string* log);

}  // namespace mlk
