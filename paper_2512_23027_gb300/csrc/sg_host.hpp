// Host-side construction of the stochastic Galerkin problem data (set-up only).
//
// Everything here runs once in sg_setup: Hermite multi-indices and triple products (Sec. 4,
// G_ijk), the analytic KL eigenpairs of the separable exponential kernel (Sec. 4,
// Eqs. CovarKer2D, KLE), the log-normal PCE of c_s at element centroids (Eqs. c0pce, LNL0),
// the structured P1 stencils of each subdomain, the node classes of the partition (Sec. 3) and
// the interface / corner maps.  The per-step path never touches these host arrays.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace sgh {

enum NodeClass : uint8_t { DIRICHLET = 0, INTERIOR = 1, REMAINING = 2, CORNER = 3 };

struct SourceDesc { int kind; double x0, y0, width, freq, amp; };

struct Problem {
  // sizes
  int N = 0, s = 0, H = 0, L = 0, nl = 0, nsub = 0;
  int M = 0, p = 0, p_in = 0, P = 0, PI = 0;
  int gfix = -1;  // compiled triple-product table matching (M, p, p_in), or -1 (set by the CUDA set-up)
  double sigma = 0, bx = 0, by = 0, g0 = 0;
  double dt = 0, alpha0 = 0, alpha1 = 0;
  double h = 0;
  // Hermite triple products, grouped by the output mode k: entries [gk_ptr[k], gk_ptr[k+1])
  std::vector<int> gk_ptr;
  std::vector<int> gk_i, gk_j;
  std::vector<double> gk_v;
  // per subdomain, per local node (ln = lj * L + li)
  std::vector<uint8_t> cls;        // nsub * nl
  std::vector<double> kapE, kapN;  // nsub * nl * PI : stiffness edge weights to (li+1,lj), (li,lj+1)
  std::vector<uint8_t> cells;      // nsub * nl : bit0 cell(li-1,lj-1) bit1 cell(li,lj-1) bit2 cell(li-1,lj) bit3 cell(li,lj)
  // interface maps
  int nG = 0, nC = 0, nGam = 0;            // global interface nodes, corners, max local interface nodes
  std::vector<int> gidx;                   // nsub * nl : global interface index or -1
  std::vector<int> cidx;                   // nsub * nl : global corner index or -1
  std::vector<int> owners;                 // nG * mo : (sub * nl + ln) of owning subdomains, -1 padded
  std::vector<int> cowners;                // nC * mo : same for corners
  std::vector<double> Dw;                  // nG : 1 / multiplicity
  std::vector<int> gam_ln;                 // nsub * nGam : local interface nodes (ascending ln), -1 padded
  std::vector<int> n_gam;                  // nsub
  std::vector<int> loc_corner;             // nsub * mc : local corner ln, -1 padded
  std::vector<int> n_loc_corner;           // nsub
  int max_corner = 0;                      // max local corners per subdomain
  int mo = 4, mc = 4;                      // row strides of owners / cowners and of loc_corner
  // free nodes (global order) -> owning (sub * nl + ln) used for output
  int n_free = 0;
  std::vector<int> free_owner;             // n_free
  std::vector<int> free_of_local;          // nsub * nl : global free index or -1
  // initial displacement (local layout, mode 0) and point-load nodes
  std::vector<double> u0_local;            // nsub * nl
  std::vector<int> load_node;              // (sub * nl + ln) per entry
  std::vector<double> load_w;              // P1 value * partition weight
  SourceDesc src{};
  // KL / PCE diagnostics
  std::vector<double> kl_lambda;           // M
  std::vector<std::vector<int>> alpha_out; // P multi-indices
};

// Returns "" on success, else an error message.
// modes / lambdas: the caller's KL (modes[n * 2 N^2 + e] = phi_n at the centroid of element e), or
// both null for the analytic eigenpairs of the separable exponential kernel.
std::string build_problem(Problem& pr, int N, int sx, int sy, int M, double sigma, double bx,
                          double by, double g0, int p, int p_in, double dt, double alpha0,
                          double alpha1, const SourceDesc& src, const double* modes = nullptr,
                          const double* lambdas = nullptr);

// ---- general partitions of unstructured triangle meshes (host set-up of the general path) ----
// Vertex classes with the corner reading of Sec. 3 (free vertices of three or more subdomains, and
// end vertices of interface curves: a free vertex of exactly two subdomains A, B without exactly two
// A|B interface edges, an edge whose two triangles lie in A and B), interface and corner numbering,
// and per subdomain the local vertices, the edges with their P1 stiffness weights per PCE input mode
// (K_i = sum_edges w_i (e_a - e_b)(e_a - e_b)^T over the subdomain's triangles, w_i = -K_i[a][b])
// and the triangles with their areas (consistent mass area / 12 [2 1 1; 1 2 1; 1 1 2]).
struct MeshProblem {
  int nv = 0, ne = 0, nsub = 0;
  int M = 0, p = 0, p_in = 0, P = 0, PI = 0;
  std::vector<uint8_t> vclass;   // nv: DIRICHLET / INTERIOR / REMAINING / CORNER
  std::vector<int> vmult;        // nv: number of subdomains whose triangles contain the vertex
  int n_free = 0, nG = 0, nC = 0;
  std::vector<int> free_idx, iface_idx, corner_idx;  // nv: index in the free / interface / corner order, or -1
  // per subdomain s: local vertices [sub_vptr[s], sub_vptr[s+1]) of sub_verts (global ids; interior,
  // remaining, corners, then Dirichlet, each ascending), local edges [sub_eptr[s], sub_eptr[s+1]) as
  // local vertex indices (edge_u < edge_v) with PI weights each in edge_w, local triangles
  // [sub_tptr[s], sub_tptr[s+1]) as three local vertex indices with their areas
  std::vector<int> sub_vptr, sub_verts;
  std::vector<int> sub_eptr, edge_u, edge_v;
  std::vector<double> edge_w;
  std::vector<int> sub_tptr, tri_loc;
  std::vector<double> tri_area;
  std::vector<double> kl_lambda;  // M
};

// Device-layout problem of a mesh (the general-partition path of the solver).  The local layout of
// subdomain s holds its free vertices in the MeshProblem order (interior, remaining, corners), padded
// to nl = the largest free count with DIRICHLET rows; the generic tables of Problem (classes, interface
// and corner maps with strides mo / mc, output maps, initial displacement, point load) are filled for
// it, and MeshRows holds the operators as sparse rows of that layout.  L = N = 0 (no grid).
struct MeshRows {
  std::vector<int> row_ptr;    // nsub * nl + 1 (padding rows empty)
  std::vector<int> col;        // local column of each entry, same subdomain; the diagonal first in its row
  std::vector<double> kval;    // entries x PI: K_i[a][b] of the subdomain's own triangles
  std::vector<double> mval;    // entries: consistent mass M[a][b] of the subdomain's own triangles
  std::vector<int> npat;       // 3 * nsub, [pat * nsub + s]: local rows of pattern 0 (interior),
                               // 1 (interior + remaining: the Neumann problem), 2 (every free vertex)
};

// xy / tri: the mesh given to build_mesh_problem; dt, alpha0, alpha1: Newmark step and Rayleigh
// damping; src: the initial pulse (kind 1, at the free vertices) or the point source (kind 2: P1 values
// at (x0, y0) in the first triangle that contains it, split over the owning subdomains with D_s).
// Returns "" on success, else an error message.
std::string mesh_to_problem(Problem& pr, MeshRows& mr, const MeshProblem& mp, const double* xy, const int* tri,
                            double dt, double alpha0, double alpha1, const SourceDesc& src);

// Dense inverse of the mean operator am M + bk K_0 (K_0: the mean-coefficient stiffness, input mode
// 0) of every subdomain on the rows of pattern pat, in the local layout: out[(s * nl + a) * nl + c]
// for a, c < npat, zero elsewhere.  Returns false if a matrix is not positive definite.
bool mesh_mean_inverse(const Problem& pr, const MeshRows& mr, int pat, double am, double bk,
                       std::vector<double>& out);

// xy: nv x 2 vertex coordinates in the unit square; dirichlet: nv flags (homogeneous Dirichlet
// vertices, eliminated); tri: ne x 3 vertex ids; part: ne subdomain ids 0 .. nsub - 1 (every id
// used).  KL and PCE as build_problem (modes, when given, hold phi_n at the element centroids:
// modes[n * ne + e]).  Returns "" on success, else an error message.
std::string build_mesh_problem(MeshProblem& mp, int nv, const double* xy, const uint8_t* dirichlet, int ne,
                               const int* tri, const int* part, int M, double sigma, double bx, double by,
                               double g0, int p, int p_in, const double* modes = nullptr,
                               const double* lambdas = nullptr);

// Recursive coordinate bisection of the triangles by centroid: a set of triangles going to k subdomains
// is ordered along the longer extent of its centroids (ties by the other coordinate, then by triangle
// index) and split at floor(size * floor(k/2) / k) into floor(k/2) and k - floor(k/2) subdomains.
// part receives ne ids 0 .. nparts - 1.  Returns "" on success, else an error message.
std::string partition_rcb(int nv, const double* xy, int ne, const int* tri, int nparts, int* part);

std::vector<std::vector<int>> multi_indices(int M, int p);
double hermite_triple(int a, int b, int c);
double ricker(double t, double f);

// In-place inverse of a symmetric positive definite n x n row-major matrix (the coarse matrix
// F_cc, Eq. Fcc_2): blocked Cholesky A = L L^T, then A^{-1} = L^{-T} L^{-1} column by column, both
// spread over up to 16 host threads.  Returns false (A then undefined) if a pivot is not positive.
bool spd_inverse(std::vector<double>& A, int n);

}  // namespace sgh
