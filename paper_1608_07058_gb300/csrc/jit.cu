// Model-specialized thread-per-trajectory kernels, compiled at run time.
//
// The ahead-of-time kernels read the model (reactant orders, net changes, pair table,
// step-size flags) from shared memory, so every propensity, step-size and update loop
// carries a table load and a branch per (reaction, species) pair, and one kernel holds
// the code for every reaction order.  A model-specialized kernel is the same lane state
// machine (thread_core.cuh) instantiated with the model's tables as compile-time
// constants: the compiler drops the zero entries, the order dispatch and the unused
// features (partial equilibrium without reversible pairs, the implicit solve), leaving
// straight-line code a fraction of the size.  The source is the library's own kernel
// headers (embedded at build time) plus a generated table type; NVRTC compiles it for
// sm_103a and the CUDA runtime loads it as a library whose kernel launches like any other.
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "jit.h"
#include "jit_sources.h"  // generated by the build: the kernel headers as strings

namespace mlk {
namespace {

std::string hexd(double v) {
  char b[64];
  std::snprintf(b, sizeof b, "%a", v);
  return b;
}

template <class F>
std::string table2(const char* name, const char* type, int rows, int cols, F value) {
  std::string s = "  struct T_" + std::string(name) + " {\n    struct Row {\n      int j;\n";
  s += "      __device__ constexpr " + std::string(type) + " operator[](int c) const {\n";
  s += "        constexpr " + std::string(type) + " t[" + std::to_string(rows) + "][" +
       std::to_string(cols) + "] = {";
  for (int r = 0; r < rows; ++r) {
    s += r ? ", {" : "{";
    for (int c = 0; c < cols; ++c) s += (c ? ", " : "") + value(r, c);
    s += "}";
  }
  s += "};\n        return t[j][c];\n      }\n    };\n";
  s += "    __device__ constexpr Row operator[](int j) const { return Row{j}; }\n  } " +
       std::string(name) + ";\n";
  return s;
}

template <class F>
std::string table1(const char* name, const char* type, int n, F value) {
  std::string s = "  struct T_" + std::string(name) + " {\n";
  s += "    __device__ constexpr " + std::string(type) + " operator[](int i) const {\n";
  s += "      constexpr " + std::string(type) + " t[" + std::to_string(n) + "] = {";
  for (int i = 0; i < n; ++i) s += (i ? ", " : "") + value(i);
  s += "};\n      return t[i];\n    }\n  } " + std::string(name) + ";\n";
  return s;
}

}  // namespace

std::string jit_source(const JitSpec& k) {
  const int NM = k.NM, MM = k.MM;
  auto in = [&](int j, int s) { return j < k.M && s < k.N; };
  std::string src =
      "typedef signed char int8_t;\ntypedef unsigned char uint8_t;\n"
      "typedef short int16_t;\ntypedef unsigned short uint16_t;\n"
      "typedef int int32_t;\ntypedef unsigned int uint32_t;\n"
      "typedef long long int64_t;\ntypedef unsigned long long uint64_t;\n"
      "typedef unsigned long size_t;\n";
  src += "#define ML_THREAD_MIN_BLOCKS " + std::string(k.occ ? "2" : "1") + "\n";
  src += "#include \"thread_core.cuh\"\nnamespace mlk {\nstruct JitModel {\n";
  src += "  static constexpr bool kCompiled = true;\n";
  src += "  static constexpr int32_t n_pairs = " + std::to_string(k.n_pairs) +
         ", N = " + std::to_string(k.N) + ", M = " + std::to_string(k.M) + ";\n";
  src += table2("ord", "int8_t", MM, NM, [&](int j, int s) {
    return std::to_string(in(j, s) ? k.ord[j * k.N + s] : 0);
  });
  src += table2("nu", "int8_t", MM, NM, [&](int j, int s) {
    return std::to_string(in(j, s) ? k.nu[j * k.N + s] : 0);
  });
  src += table2("nuf", "float", MM, NM, [&](int j, int s) {
    return std::to_string(in(j, s) ? k.nu[j * k.N + s] : 0) + ".0f";
  });
  src += table1("partner", "int8_t", MM, [&](int j) {
    return std::to_string(j < k.M && k.partner[j] > j ? k.partner[j] : -1);
  });
  src += table1("isreact", "uint8_t", NM, [&](int s) {
    return std::to_string(s < k.N ? (int)k.isreact[s] : 0);
  });
  src += table1("hor", "uint8_t", NM, [&](int s) {
    return std::to_string(s < k.N ? (int)k.hor[s] : 0);
  });
  src += table1("rates", "double", MM, [&](int j) {
    return j < k.M ? hexd(k.rates[j]) : std::string("0.0");
  });
  src += "};\n}  // namespace mlk\n";
  const char* prec = k.precision_ref ? "mlk::PrecRef" : "mlk::PrecFast";
  const std::string tmpl = std::to_string(NM) + ", " + std::to_string(MM) + ", " + prec;
  src += "extern \"C\" __global__ void ML_THREAD_BOUNDS ml_jit_kernel(const void* tables, "
         "const mlk::SimArgs args) {\n  const mlk::JitModel md{};\n";
  if (k.driver == kJitPool) {
    src += "  extern __shared__ uint32_t pool_words[];\n";
    src += "  mlk::run_pool<" + tmpl + ">(md, true, args, pool_words);\n";
  } else if (k.driver == kJitSequential) {
    src += "  mlk::run_sequential<" + tmpl + ", false>(md, true, args);\n";
  } else {
    src += "  mlk::run_rounds<" + tmpl + ">(md, true, args);\n";
  }
  src += "}\n";
  return src;
}

int jit_compile(const std::string& src, bool precision_ref, std::vector<char>* cubin,
                std::string* log) {
  nvrtcProgram prog;
  std::vector<const char*> hdr, names;
  for (int i = 0; i < kJitHeaderCount; ++i) {
    hdr.push_back(kJitHeaderText[i]);
    names.push_back(kJitHeaderName[i]);
  }
  if (nvrtcCreateProgram(&prog, src.c_str(), "ml_jit.cu", kJitHeaderCount, hdr.data(),
                         names.data()) != NVRTC_SUCCESS) {
    *log = "nvrtcCreateProgram failed";
    return -1;
  }
  // -default-device: the public header's host declarations are read as device ones (unused)
  std::vector<const char*> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-DNDEBUG",
                                   "-default-device"};
  if (precision_ref) opts.push_back("--fmad=false");  // the reference order, no contraction
  const nvrtcResult rc = nvrtcCompileProgram(prog, (int)opts.size(), opts.data());
  size_t n = 0;
  nvrtcGetProgramLogSize(prog, &n);
  log->assign(n, '\0');
  if (n) nvrtcGetProgramLog(prog, &(*log)[0]);
  if (rc != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return -1;
  }
  size_t nb = 0;
  nvrtcGetCUBINSize(prog, &nb);
  cubin->resize(nb);
  nvrtcGetCUBIN(prog, cubin->data());
  nvrtcDestroyProgram(&prog);
  return nb ? 0 : -1;
}

}  // namespace mlk
