// Prints the general-partition set-up tables of one mesh, built by the library's host code
// (sg_host.cpp, build_mesh_problem), for comparison with the oracle (tests/test_host_mesh.py).
// Plain C++17, no GPU.
// Usage: mesh_dump file.  The file holds: "nv ne M sigma bx by g0 p p_in", then nv lines
// "x y dirichlet", then ne lines "a b c subdomain".
// Output: one line per table, "name v0 v1 ..."; per subdomain s: "verts s ...", "edges s u v u v ...",
// "weights s ..." (PI per edge), "areas s ...".
#include <cstdio>
#include <string>
#include <type_traits>
#include <vector>

#include "../../paper_2512_23027_gb300/csrc/sg_host.hpp"

template <typename T>
static void row(const char* name, int s, const T* v, size_t n) {
  std::printf("%s", name);
  if (s >= 0) std::printf(" %d", s);
  for (size_t k = 0; k < n; ++k) {
    if constexpr (std::is_floating_point_v<T>) std::printf(" %.17g", static_cast<double>(v[k]));
    else std::printf(" %d", static_cast<int>(v[k]));
  }
  std::printf("\n");
}

int main(int argc, char** argv) {
  if (argc != 2) return 2;
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
  sgh::MeshProblem mp;
  const std::string msg = sgh::build_mesh_problem(mp, nv, xy.data(), dir.data(), ne, tri.data(), part.data(), M,
                                                  sigma, bx, by, g0, p, p_in);
  if (!msg.empty()) {
    std::fprintf(stderr, "%s\n", msg.c_str());
    return 1;
  }
  std::printf("sizes %d %d %d %d %d %d %d %d\n", mp.nv, mp.ne, mp.nsub, mp.P, mp.PI, mp.n_free, mp.nG, mp.nC);
  row("vclass", -1, mp.vclass.data(), mp.vclass.size());
  row("vmult", -1, mp.vmult.data(), mp.vmult.size());
  row("kl_lambda", -1, mp.kl_lambda.data(), mp.kl_lambda.size());
  for (int s = 0; s < mp.nsub; ++s) {
    const int v0 = mp.sub_vptr[s], v1 = mp.sub_vptr[s + 1];
    const int e0 = mp.sub_eptr[s], e1 = mp.sub_eptr[s + 1];
    const int t0 = mp.sub_tptr[s], t1 = mp.sub_tptr[s + 1];
    row("verts", s, mp.sub_verts.data() + v0, v1 - v0);
    std::vector<int> uv;
    for (int e = e0; e < e1; ++e) {
      uv.push_back(mp.sub_verts[v0 + mp.edge_u[e]]);
      uv.push_back(mp.sub_verts[v0 + mp.edge_v[e]]);
    }
    row("edges", s, uv.data(), uv.size());
    row("weights", s, mp.edge_w.data() + (size_t)e0 * mp.PI, (size_t)(e1 - e0) * mp.PI);
    row("areas", s, mp.tri_area.data() + t0, t1 - t0);
  }
  return 0;
}
