// Prints the host set-up tables of one problem, built by the library's set-up code (sg_host.cpp),
// for comparison with the oracle (tests/test_host_setup.py).  Plain C++17, no GPU.
// Usage: host_dump N s M sigma bx by g0 p p_in dt kind x0 y0 width freq amp [kl_file]
// kl_file (optional): the caller's KL as whitespace-separated numbers, M lambdas then M x 2 N^2 mode
// values at the element centroids (mode-major).
// Output: one line per table, "name v0 v1 ...".
#include <cstdio>
#include <cstdlib>
#include <string>
#include <type_traits>
#include <vector>

#include "../../paper_2512_23027_gb300/csrc/sg_host.hpp"

template <typename T>
static void row(const char* name, const std::vector<T>& v) {
  std::printf("%s", name);
  for (const T& x : v) {
    if constexpr (std::is_floating_point_v<T>) std::printf(" %.17g", static_cast<double>(x));
    else std::printf(" %d", static_cast<int>(x));
  }
  std::printf("\n");
}

int main(int argc, char** argv) {
  if (argc != 17 && argc != 18) {
    std::fprintf(stderr, "usage: host_dump N s M sigma bx by g0 p p_in dt kind x0 y0 width freq amp [kl_file]\n");
    return 2;
  }
  const int N = std::atoi(argv[1]), s = std::atoi(argv[2]), M = std::atoi(argv[3]);
  const double sigma = std::atof(argv[4]), bx = std::atof(argv[5]), by = std::atof(argv[6]);
  const double g0 = std::atof(argv[7]), dt = std::atof(argv[10]);
  const int p = std::atoi(argv[8]), p_in = std::atoi(argv[9]);
  std::vector<double> modes, lambdas;
  if (argc == 18) {
    FILE* f = std::fopen(argv[17], "r");
    if (!f) return 2;
    double v;
    for (int n = 0; n < M && std::fscanf(f, "%lf", &v) == 1; ++n) lambdas.push_back(v);
    while (std::fscanf(f, "%lf", &v) == 1) modes.push_back(v);
    std::fclose(f);
    if ((int)lambdas.size() != M || modes.size() != (size_t)M * 2 * N * N) return 2;
  }
  sgh::Problem pr;
  const sgh::SourceDesc sd{std::atoi(argv[11]), std::atof(argv[12]), std::atof(argv[13]), std::atof(argv[14]),
                          std::atof(argv[15]), std::atof(argv[16])};
  const std::string msg = sgh::build_problem(pr, N, s, s, M, sigma, bx, by, g0, p, p_in, dt, 0.5445, 0.0174, sd,
                                             modes.empty() ? nullptr : modes.data(),
                                             lambdas.empty() ? nullptr : lambdas.data());
  if (!msg.empty()) {
    std::fprintf(stderr, "%s\n", msg.c_str());
    return 1;
  }
  std::printf("sizes %d %d %d %d %d %d %d %d\n", pr.L, pr.nl, pr.nsub, pr.P, pr.PI, pr.nG, pr.nC, pr.n_free);
  row("kl_lambda", pr.kl_lambda);
  std::vector<int> alpha;
  for (const auto& a : pr.alpha_out) alpha.insert(alpha.end(), a.begin(), a.end());
  row("alpha_out", alpha);
  row("gk_ptr", pr.gk_ptr);
  row("gk_i", pr.gk_i);
  row("gk_j", pr.gk_j);
  row("gk_v", pr.gk_v);
  row("cls", pr.cls);
  row("gidx", pr.gidx);
  row("Dw", pr.Dw);
  row("kapE", pr.kapE);
  row("kapN", pr.kapN);
  row("load_node", pr.load_node);
  row("load_w", pr.load_w);
  row("u0_local", pr.u0_local);
  return 0;
}
