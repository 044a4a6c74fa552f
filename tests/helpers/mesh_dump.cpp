// Prints the general-partition set-up tables of one mesh, built by the library's host code
// (sg_host.cpp, build_mesh_problem, mesh_to_problem, mesh_mean_inverse), for comparison with the
// oracle (tests/test_host_mesh.py).  Plain C++17, no GPU.
// Usage: mesh_dump file [layout_file].  The file holds: "nv ne M sigma bx by g0 p p_in", then nv lines
// "x y dirichlet", then ne lines "a b c subdomain".  layout_file holds "dt alpha0 alpha1 am bk kind x0
// y0 width freq amp" and adds the device-layout tables.
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
  if (argc != 2 && argc != 3) return 2;
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
  if (argc == 3) {
    FILE* g = std::fopen(argv[2], "r");
    if (!g) return 2;
    double dt, a0, a1, am, bk;
    sgh::SourceDesc src{};
    if (std::fscanf(g, "%lf %lf %lf %lf %lf %d %lf %lf %lf %lf %lf", &dt, &a0, &a1, &am, &bk, &src.kind, &src.x0,
                    &src.y0, &src.width, &src.freq, &src.amp) != 11)
      return 2;
    std::fclose(g);
    sgh::Problem pr;
    sgh::MeshRows mr;
    const std::string m2 = sgh::mesh_to_problem(pr, mr, mp, xy.data(), tri.data(), dt, a0, a1, src);
    if (!m2.empty()) {
      std::fprintf(stderr, "%s\n", m2.c_str());
      return 1;
    }
    std::printf("layout %d %d %d %d %d %d %d %d\n", pr.nl, pr.mo, pr.mc, pr.nG, pr.nC, pr.n_free, pr.nGam,
                pr.max_corner);
    row("cls", -1, pr.cls.data(), pr.cls.size());
    row("gidx", -1, pr.gidx.data(), pr.gidx.size());
    row("cidx", -1, pr.cidx.data(), pr.cidx.size());
    row("owners", -1, pr.owners.data(), pr.owners.size());
    row("cowners", -1, pr.cowners.data(), pr.cowners.size());
    row("Dw", -1, pr.Dw.data(), pr.Dw.size());
    row("gam_ln", -1, pr.gam_ln.data(), pr.gam_ln.size());
    row("n_gam", -1, pr.n_gam.data(), pr.n_gam.size());
    row("loc_corner", -1, pr.loc_corner.data(), pr.loc_corner.size());
    row("n_loc_corner", -1, pr.n_loc_corner.data(), pr.n_loc_corner.size());
    row("free_owner", -1, pr.free_owner.data(), pr.free_owner.size());
    row("free_of_local", -1, pr.free_of_local.data(), pr.free_of_local.size());
    row("u0", -1, pr.u0_local.data(), pr.u0_local.size());
    row("load_node", -1, pr.load_node.data(), pr.load_node.size());
    row("load_w", -1, pr.load_w.data(), pr.load_w.size());
    row("gk_ptr", -1, pr.gk_ptr.data(), pr.gk_ptr.size());
    row("gk_i", -1, pr.gk_i.data(), pr.gk_i.size());
    row("gk_j", -1, pr.gk_j.data(), pr.gk_j.size());
    row("gk_v", -1, pr.gk_v.data(), pr.gk_v.size());
    row("npat", -1, mr.npat.data(), mr.npat.size());
    row("row_ptr", -1, mr.row_ptr.data(), mr.row_ptr.size());
    row("col", -1, mr.col.data(), mr.col.size());
    row("kval", -1, mr.kval.data(), mr.kval.size());
    row("mval", -1, mr.mval.data(), mr.mval.size());
    for (int pat = 0; pat < 3; ++pat) {
      std::vector<double> inv;
      if (!sgh::mesh_mean_inverse(pr, mr, pat, am, bk, inv)) {
        std::fprintf(stderr, "mean operator not positive definite\n");
        return 1;
      }
      const char* nm[3] = {"ainv0", "ainv1", "ainv2"};
      row(nm[pat], -1, inv.data(), inv.size());
    }
  }
  return 0;
}
