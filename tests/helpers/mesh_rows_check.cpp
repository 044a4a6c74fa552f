// Runs the per-row arithmetic of the mesh kernels (sg_mesh_rows.h: the SG operator apply and the
// dense mean-operator preconditioner, the functions the CUDA kernels call) on the host over the
// device layout built by sg_host.cpp, for comparison with the oracle (tests/test_host_mesh.py).
// Plain C++17, no GPU.
// Usage: mesh_rows_check mesh_file layout_file x_file.  mesh_file and layout_file as mesh_dump;
// x_file holds "cm ck" and then two vectors of nsub * nl * P values, x and w (one local vector per
// subdomain, node-major).
// Output: "y v..." = cm (M (x) I) x + ck (sum_i K_i (x) G_i) x on every free row (0 on padding rows),
// "z0 v...", "z1 v..." = (I (x) A0^{-1}) x on patterns 0 and 1 (x restricted to the pattern's rows),
// "d1 v..." = the same operator as y applied to the direction x + 0.25 w formed on the fly
// (apply_row_dir), "d0 v..." = apply_row_dir with beta 0 and w replaced by NaN (never read).
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../paper_2512_23027_gb300/csrc/sg_host.hpp"
#include "../../paper_2512_23027_gb300/csrc/sg_mesh_rows.h"

static void row(const char* name, const std::vector<double>& v) {
  std::printf("%s", name);
  for (double x : v) std::printf(" %.17g", x);
  std::printf("\n");
}

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  FILE* f = std::fopen(argv[1], "r");
  if (!f) return 2;
  int nv, ne, M, p, p_in;
  double sigma, bx, by, g0;
  if (std::fscanf(f, "%d %d %d %lf %lf %lf %lf %d %d", &nv, &ne, &M, &sigma, &bx, &by, &g0, &p, &p_in) != 9) return 2;
  std::vector<double> xy(2 * (size_t)nv);
  std::vector<uint8_t> dir(nv);
  for (int v = 0; v < nv; ++v) {
    int d;
    if (std::fscanf(f, "%lf %lf %d", &xy[2 * v], &xy[2 * v + 1], &d) != 3) return 2;
    dir[v] = (uint8_t)d;
  }
  std::vector<int> tri(3 * (size_t)ne), part(ne);
  for (int e = 0; e < ne; ++e)
    if (std::fscanf(f, "%d %d %d %d", &tri[3 * e], &tri[3 * e + 1], &tri[3 * e + 2], &part[e]) != 4) return 2;
  std::fclose(f);
  FILE* g = std::fopen(argv[2], "r");
  if (!g) return 2;
  double dt, a0, a1, am, bk;
  sgh::SourceDesc src{};
  if (std::fscanf(g, "%lf %lf %lf %lf %lf %d %lf %lf %lf %lf %lf", &dt, &a0, &a1, &am, &bk, &src.kind, &src.x0, &src.y0,
                  &src.width, &src.freq, &src.amp) != 11)
    return 2;
  std::fclose(g);
  sgh::MeshProblem mp;
  std::string msg = sgh::build_mesh_problem(mp, nv, xy.data(), dir.data(), ne, tri.data(), part.data(), M, sigma, bx,
                                            by, g0, p, p_in);
  sgh::Problem pr;
  sgh::MeshRows mr;
  if (msg.empty()) msg = sgh::mesh_to_problem(pr, mr, mp, xy.data(), tri.data(), dt, a0, a1, src);
  if (!msg.empty()) {
    std::fprintf(stderr, "%s\n", msg.c_str());
    return 1;
  }
  const int nsub = pr.nsub, nl = pr.nl, P = pr.P;
  const long long len = (long long)nl * P;
  FILE* h = std::fopen(argv[3], "r");
  if (!h) return 2;
  double cm, ck;
  if (std::fscanf(h, "%lf %lf", &cm, &ck) != 2) return 2;
  std::vector<double> x((size_t)nsub * len), wv((size_t)nsub * len);
  for (auto& v : x)
    if (std::fscanf(h, "%lf", &v) != 1) return 2;
  for (auto& v : wv)
    if (std::fscanf(h, "%lf", &v) != 1) return 2;
  std::fclose(h);
  sgm::Rows<double> r;
  r.rp = mr.row_ptr.data(); r.col = mr.col.data(); r.kv = mr.kval.data(); r.mv = mr.mval.data();
  r.gk_ptr = pr.gk_ptr.data(); r.gk_i = pr.gk_i.data(); r.gk_j = pr.gk_j.data(); r.gk_v = pr.gk_v.data();
  r.nl = nl; r.P = P; r.PI = pr.PI;
  // the kernels' index decomposition: element idx of problem b (= subdomain b, R = 1)
  std::vector<double> y((size_t)nsub * len, 0.0);
  for (long long idx = 0; idx < nsub * len; ++idx) {
    const int b = (int)(idx / len);
    const long long t = idx - (long long)b * len;
    const int a = (int)(t / P), k = (int)(t - (long long)a * P);
    const long long rw = (long long)b * nl + a;
    if (pr.cls[rw] != sgh::DIRICHLET) y[idx] = sgm::apply_row(r, rw, k, x.data() + b * len, x.data() + b * len, cm, ck);
  }
  row("y", y);
  const std::vector<double> nanv((size_t)nsub * len, std::nan(""));
  for (int pass = 0; pass < 2; ++pass) {
    const double bet = pass == 0 ? 0.25 : 0.0;
    const double* pold = pass == 0 ? wv.data() : nanv.data();
    std::vector<double> d((size_t)nsub * len, 0.0);
    for (long long idx = 0; idx < nsub * len; ++idx) {
      const int b = (int)(idx / len);
      const long long t = idx - (long long)b * len;
      const int a = (int)(t / P), k = (int)(t - (long long)a * P);
      const long long rw = (long long)b * nl + a;
      if (pr.cls[rw] != sgh::DIRICHLET)
        d[idx] = sgm::apply_row_dir(r, rw, k, x.data() + b * len, pold + b * len, bet, cm, ck);
    }
    row(pass == 0 ? "d1" : "d0", d);
  }
  for (int pat = 0; pat < 2; ++pat) {
    std::vector<double> inv;
    if (!sgh::mesh_mean_inverse(pr, mr, pat, am, bk, inv)) return 1;
    std::vector<double> z((size_t)nsub * len, 0.0);
    for (long long idx = 0; idx < nsub * len; ++idx) {
      const int b = (int)(idx / len);
      const long long t = idx - (long long)b * len;
      const int a = (int)(t / P), k = (int)(t - (long long)a * P);
      const int n = mr.npat[(size_t)pat * nsub + b];
      if (a < n) z[idx] = sgm::dense_row(inv.data() + ((size_t)b * nl + a) * nl, x.data() + b * len, n, P, k);
    }
    row(pat == 0 ? "z0" : "z1", z);
  }
  return 0;
}
