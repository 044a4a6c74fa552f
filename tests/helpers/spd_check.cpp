// Host check of the coarse-matrix inverse (csrc/sg_host.cpp, sgh::spd_inverse): reads "n" and the n x n
// row-major matrix from stdin, prints "ok" (1 or 0) and, when ok, the inverse row-major.
#include <cstdio>
#include <vector>

#include "../../paper_2512_23027_gb300/csrc/sg_host.hpp"

int main() {
  int n;
  if (std::scanf("%d", &n) != 1 || n < 0) return 2;
  std::vector<double> A((size_t)n * n);
  for (auto& v : A)
    if (std::scanf("%lf", &v) != 1) return 2;
  const bool ok = sgh::spd_inverse(A, n);
  std::printf("%d\n", ok ? 1 : 0);
  if (ok)
    for (double v : A) std::printf("%.17g\n", v);
  return 0;
}
