// Host-only check of the model-specialized kernel sources (built and run by
// tests/test_jit_sources.py, no GPU needed): for each model given on standard input,
// generate the source of the requested driver / precision / register-budget combinations
// and compile it with NVRTC for sm_103a.
//
// Input, one model per line:  K  (driver ref occ) x K  N M NM MM n_pairs  ord[M*N]
//                             nu[M*N]  partner[M]  isreact[N]  hor[N]  rates[M]
// Output: one line per compiled kernel, "ok <driver> <ref> <occ> <cubin bytes>", or
// "fail ..." followed by the compiler log; exit status 1 if any failed.
#include <cstdint>
#include <cstdio>
#include <iostream>
#include <string>
#include <vector>

#include "jit.h"

int main() {
  int K, N, M, NM, MM, n_pairs;
  int failed = 0, models = 0;
  while (std::cin >> K) {
    std::vector<int> combos(3 * K);
    for (auto& v : combos) std::cin >> v;
    std::cin >> N >> M >> NM >> MM >> n_pairs;
    std::vector<int32_t> ord(M * N), nu(M * N), partner(M);
    std::vector<uint8_t> isreact(N), hor(N);
    std::vector<double> rates(M);
    for (auto& v : ord) std::cin >> v;
    for (auto& v : nu) std::cin >> v;
    for (auto& v : partner) std::cin >> v;
    for (auto& v : isreact) {
      int b;
      std::cin >> b;
      v = (uint8_t)b;
    }
    for (auto& v : hor) {
      int b;
      std::cin >> b;
      v = (uint8_t)b;
    }
    for (auto& v : rates) std::cin >> v;
    ++models;
    for (int c = 0; c < K; ++c) {
      const int driver = combos[3 * c], ref = combos[3 * c + 1], occ = combos[3 * c + 2];
      mlk::JitSpec k;
      k.NM = NM;
      k.MM = MM;
      k.N = N;
      k.M = M;
      k.ord = ord.data();
      k.nu = nu.data();
      k.rates = rates.data();
      k.partner = partner.data();
      k.isreact = isreact.data();
      k.hor = hor.data();
      k.n_pairs = n_pairs;
      k.precision_ref = ref;
      k.driver = driver;
      k.occ = occ;
      std::vector<char> cubin;
      std::string log;
      if (mlk::jit_compile(mlk::jit_source(k), ref, &cubin, &log) == 0) {
        std::printf("ok %d %d %d %zu\n", driver, ref, occ, cubin.size());
      } else {
        std::printf("fail %d %d %d\n%s\n", driver, ref, occ, log.c_str());
        ++failed;
      }
    }
  }
  std::printf("models %d failed %d\n", models, failed);
  return failed || !models ? 1 : 0;
}
