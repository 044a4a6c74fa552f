// Host program: prints the compile-time triple-product tables of sg_gfix.cuh (one line per
// compiled PCE size: M p p_in P PI NNZ, then the (i, j, k) entries in table order), for the CPU
// test that compares them with the oracle.
#include <cstdio>
#include "../../paper_2512_23027_gb300/csrc/sg_gfix.cuh"

template <class C>
static void dump() {
  std::printf("%d %d %d %d %d %d\n", C::M, C::p, C::pin, C::P, C::PI, C::NNZ);
  for (int e = 0; e < C::NNZ; ++e) std::printf("%d %d %d\n", C::ti(e), C::tj(e), C::tk(e));
}

int main() {
  using namespace sgk::gfix;
  dump<C0>(); dump<C1>(); dump<C2>(); dump<C3>(); dump<C4>(); dump<C5>(); dump<C6>();
  return 0;
}
