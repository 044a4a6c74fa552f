// Host-side set-up math (see sg_host.hpp).  Plain C++17, no architecture-specific code.
#include "sg_host.hpp"

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <thread>

namespace sgh {

static double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// Graded multi-indices |alpha| <= p; inside a degree, descending lexicographic order.
std::vector<std::vector<int>> multi_indices(int M, int p) {
  std::vector<std::vector<int>> out;
  for (int d = 0; d <= p; ++d) {
    std::vector<std::vector<int>> level;
    std::vector<int> a(M, 0);
    std::function<void(int, int)> rec = [&](int pos, int left) {
      if (pos == M - 1) {
        a[pos] = left;
        level.push_back(a);
        return;
      }
      for (int v = left; v >= 0; --v) {  // larger leading entries first
        a[pos] = v;
        rec(pos + 1, left - v);
      }
    };
    if (M > 0) rec(0, d);
    else if (d == 0) level.push_back({});
    out.insert(out.end(), level.begin(), level.end());
  }
  return out;
}

// <psi_a psi_b psi_c> for normalised probabilists' Hermite polynomials (Sec. 4, G_ijk):
// sqrt(a! b! c!) / ((s-a)! (s-b)! (s-c)!) with s = (a+b+c)/2 integral and >= max(a,b,c).
double hermite_triple(int a, int b, int c) {
  int t = a + b + c;
  if (t & 1) return 0.0;
  int s = t / 2;
  if (s < a || s < b || s < c) return 0.0;
  return std::sqrt(fact(a) * fact(b) * fact(c)) / (fact(s - a) * fact(s - b) * fact(s - c));
}

double ricker(double t, double f) {
  const double pi = 3.14159265358979323846;
  double tau = t - 1.0 / f;
  double a = (pi * f * tau) * (pi * f * tau);
  return (1.0 - 2.0 * a) * std::exp(-a);
}

// ---- KL of exp(-c|x-y|) on [-1/2, 1/2]: roots by bisection on the monotone branches ----
struct Eig1 { double lam, w; int parity; };

static double bisect(const std::function<double(double)>& f, double lo, double hi) {
  double flo = f(lo);
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double fm = f(mid);
    if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else { hi = mid; }
    if (hi - lo <= 1e-16 * std::max(1.0, std::fabs(mid))) break;
  }
  return 0.5 * (lo + hi);
}

static std::vector<Eig1> eig1d(double b, int n) {
  const double pi = 3.14159265358979323846;
  double c = 1.0 / b;
  std::vector<Eig1> out;
  for (int k = 0; (int)out.size() < n; ++k) {
    // even: c - w tan(w/2) = 0 on (2k pi, 2k pi + pi), decreasing
    double w = bisect([c](double x) { return c - x * std::tan(0.5 * x); },
                      2 * k * pi + 1e-10, 2 * k * pi + pi - 1e-10);
    out.push_back({2 * c / (w * w + c * c), w, 0});
    if ((int)out.size() == n) break;
    // odd: w + c tan(w/2) = 0 on (2k pi + pi, 2k pi + 2 pi), increasing
    w = bisect([c](double x) { return x + c * std::tan(0.5 * x); },
               2 * k * pi + pi + 1e-10, 2 * k * pi + 2 * pi - 1e-10);
    out.push_back({2 * c / (w * w + c * c), w, 1});
  }
  return out;
}

static double phi1(double x, const Eig1& e) {
  double u = x - 0.5;
  if (e.parity == 0) return std::cos(e.w * u) / std::sqrt(0.5 + std::sin(e.w) / (2 * e.w));
  return std::sin(e.w * u) / std::sqrt(0.5 - std::sin(e.w) / (2 * e.w));
}

// The top M 2-D KL modes of the separable exponential kernel: products of the 1-D eigenpairs (ex in x,
// ey in y, the first M + 1 of each), sorted by eigenvalue; ties go to the lower y index, then the lower
// x index.  A non-positive correlation length stands for 1 (its modes are then unused: caller KL).
struct KLCand { double lam; int ix, iy; };
static std::vector<KLCand> kl_select(int M, double bx, double by, std::vector<Eig1>& ex, std::vector<Eig1>& ey) {
  ex = eig1d(bx > 0 ? bx : 1.0, M + 1);
  ey = eig1d(by > 0 ? by : 1.0, M + 1);
  std::vector<KLCand> cand;
  for (int ix = 0; ix <= M; ++ix)
    for (int iy = 0; iy <= M; ++iy) cand.push_back({ex[ix].lam * ey[iy].lam, ix, iy});
  std::stable_sort(cand.begin(), cand.end(), [](const KLCand& a, const KLCand& b) {
    if (a.lam != b.lam) return a.lam > b.lam;
    if (a.iy != b.iy) return a.iy < b.iy;
    return a.ix < b.ix;
  });
  cand.resize(M);
  return cand;
}

// Runs f(i) for i in [i0, i1) on up to 16 host threads, rows assigned cyclically (thread t takes
// i0 + t, i0 + t + T, ...) so that triangular work stays balanced.
template <class F>
static void parallel_cyclic(int i0, int i1, F&& f) {
  const int n = i1 - i0;
  if (n <= 0) return;
  int T = (int)std::thread::hardware_concurrency();
  T = std::max(1, std::min({T, 16, n / 8}));
  if (T <= 1) {
    for (int i = i0; i < i1; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(T);
  for (int t = 0; t < T; ++t)
    th.emplace_back([&, t]() {
      for (int i = i0 + t; i < i1; i += T) f(i);
    });
  for (auto& x : th) x.join();
}

// Triple products <psi_i psi_j psi_k> (input mode i, output modes j, k), grouped by the output mode k.
static void triple_table(Problem& pr, const std::vector<std::vector<int>>& Ain,
                         const std::vector<std::vector<int>>& Aout) {
  const int P = (int)Aout.size(), PI = (int)Ain.size(), M = pr.M;
  pr.gk_ptr.assign(P + 1, 0);
  pr.gk_i.clear(); pr.gk_j.clear(); pr.gk_v.clear();
  for (int k = 0; k < P; ++k) {
    for (int i = 0; i < PI; ++i)
      for (int j = 0; j < P; ++j) {
        double v = 1.0;
        for (int d = 0; d < M && v != 0.0; ++d) v *= hermite_triple(Ain[i][d], Aout[j][d], Aout[k][d]);
        if (v != 0.0) { pr.gk_i.push_back(i); pr.gk_j.push_back(j); pr.gk_v.push_back(v); }
      }
    pr.gk_ptr[k + 1] = (int)pr.gk_v.size();
  }
}

std::string build_problem(Problem& pr, int N, int sx, int sy, int M, double sigma, double bx,
                          double by, double g0, int p, int p_in, double dt, double alpha0,
                          double alpha1, const SourceDesc& src, const double* modes,
                          const double* lambdas) {
  if (N < 2 || sx < 1 || sy < 1 || sx != sy) return "grid: N >= 2 and nsub_x == nsub_y >= 1 required";
  if (N % sx) return "grid: N must be divisible by the subdomain count";
  if (M < 0 || M > 12 || p < 0 || p_in < 0 || p > 10 || p_in > 20) return "pce/kl: unsupported M, p or p_in";
  if (!(dt > 0) || !(sigma >= 0)) return "params: dt > 0 and sigma >= 0 required";
  if (M > 0 && !modes && !(bx > 0 && by > 0)) return "kl: correlation lengths must be positive";
  if (modes && M > 0) {
    if (!lambdas) return "kl: modes given without lambdas";
    for (int n = 0; n < M; ++n)
      if (!(lambdas[n] > 0) || !std::isfinite(lambdas[n])) return "kl: lambdas must be positive and finite";
    const size_t ne = (size_t)2 * N * N * M;
    for (size_t e = 0; e < ne; ++e)
      if (!std::isfinite(modes[e])) return "kl: modes must be finite";
  }
  pr.N = N; pr.s = sx; pr.H = N / sx; pr.L = pr.H + 1; pr.nl = pr.L * pr.L; pr.nsub = sx * sx;
  pr.M = M; pr.p = p; pr.p_in = p_in; pr.sigma = sigma; pr.bx = bx; pr.by = by; pr.g0 = g0;
  pr.dt = dt; pr.alpha0 = alpha0; pr.alpha1 = alpha1; pr.h = 1.0 / N; pr.src = src;
  pr.mo = 4; pr.mc = 4;  // at most four subdomains meet at a node of the structured partition
  auto Aout = multi_indices(M, p);
  auto Ain = multi_indices(M, p_in);
  pr.P = (int)Aout.size();
  pr.PI = (int)Ain.size();
  pr.alpha_out = Aout;
  const int PI = pr.PI, H = pr.H, L = pr.L, nl = pr.nl, nsub = pr.nsub;

  triple_table(pr, Ain, Aout);

  // KL modes: products of 1-D eigenpairs, top M by lambda, ties -> lower y index, then x index
  std::vector<Eig1> ex, ey;
  const std::vector<KLCand> cand = kl_select(M, bx, by, ex, ey);
  pr.kl_lambda.resize(M);
  for (int n = 0; n < M; ++n) pr.kl_lambda[n] = modes ? lambdas[n] : cand[n].lam;

  // PCE coefficients of exp(g) at the element centroids (Eqs. c0pce, LNL0):
  //   c_alpha = exp(g0 + |g|^2 / 2) prod_n g_n^{a_n} / sqrt(a_n!),  g_n = sigma sqrt(lambda_n) phi_n(x) psi_n(y).
  // g_n is separable and the centroids of the T1 / T2 triangles lie on N column and N row positions,
  // so the 1-D factors are tabulated once per position (O(N M) trigonometric evaluations instead of
  // O(N^2 M)); the powers of g_n are formed by repeated products.
  const double h = pr.h;
  std::vector<double> fx1((size_t)M * N), fx2((size_t)M * N), fy1((size_t)M * N), fy2((size_t)M * N);
  for (int n = 0; n < M; ++n) {
    const double amp = sigma * std::sqrt(cand[n].lam);
    const Eig1& exn = ex[cand[n].ix];
    const Eig1& eyn = ey[cand[n].iy];
    for (int q = 0; q < N; ++q) {
      fx1[(size_t)n * N + q] = amp * phi1((q + 2.0 / 3.0) * h, exn);  // T1 centroid x
      fx2[(size_t)n * N + q] = amp * phi1((q + 1.0 / 3.0) * h, exn);  // T2 centroid x
      fy1[(size_t)n * N + q] = phi1((q + 1.0 / 3.0) * h, eyn);        // T1 centroid y
      fy2[(size_t)n * N + q] = phi1((q + 2.0 / 3.0) * h, eyn);        // T2 centroid y
    }
  }
  // per input mode i: prod_n 1 / sqrt(a_n!) and its nonzero exponents as (variable, exponent) pairs
  std::vector<double> kfac(PI);
  std::vector<int> mi_off(PI + 1, 0), mi_n, mi_a;
  for (int i = 0; i < PI; ++i) {
    double v = 1.0;
    for (int n = 0; n < M; ++n)
      if (Ain[i][n]) {
        v /= std::sqrt(fact(Ain[i][n]));
        mi_n.push_back(n);
        mi_a.push_back(Ain[i][n]);
      }
    kfac[i] = v;
    mi_off[i + 1] = (int)mi_n.size();
  }
  constexpr int MAXM = 12, MAXA = 20;  // limits checked above (M <= 12, p_in <= 20)
  auto coef_from = [&](const double* g, double* c) {
    double s2 = 0.0;
    double pw[MAXM][MAXA + 1];
    for (int n = 0; n < M; ++n) {
      s2 += g[n] * g[n];
      pw[n][0] = 1.0;
      for (int a = 1; a <= p_in; ++a) pw[n][a] = pw[n][a - 1] * g[n];
    }
    const double c0 = std::exp(g0 + 0.5 * s2);
    for (int i = 0; i < PI; ++i) {
      double v = c0 * kfac[i];
      for (int q = mi_off[i]; q < mi_off[i + 1]; ++q) v *= pw[mi_n[q]][mi_a[q]];
      c[i] = v;
    }
  };
  // element coefficients of the whole mesh: T1 centroid (i+2/3, j+1/3) h, T2 (i+1/3, j+2/3) h
  std::vector<double> cT1((size_t)N * N * PI), cT2((size_t)N * N * PI);
  std::vector<double> amp(M);
  for (int n = 0; n < M; ++n) amp[n] = modes ? sigma * std::sqrt(lambdas[n]) : 0.0;
  const size_t ne = (size_t)2 * N * N;
  parallel_cyclic(0, N, [&](int j) {  // grid rows are independent
    for (int i = 0; i < N; ++i) {
      double g[MAXM];
      const size_t e1 = 2 * ((size_t)j * N + i);  // element index of T1 (T2 is e1 + 1)
      for (int n = 0; n < M; ++n)
        g[n] = modes ? amp[n] * modes[(size_t)n * ne + e1] : fx1[(size_t)n * N + i] * fy1[(size_t)n * N + j];
      coef_from(g, &cT1[((size_t)j * N + i) * PI]);
      for (int n = 0; n < M; ++n)
        g[n] = modes ? amp[n] * modes[(size_t)n * ne + e1 + 1] : fx2[(size_t)n * N + i] * fy2[(size_t)n * N + j];
      coef_from(g, &cT2[((size_t)j * N + i) * PI]);
    }
  });

  // node classes and maps
  auto gfree = [&](int I, int J) { return I >= 1 && I <= N - 1 && J >= 1 && J <= N - 1; };
  auto on_iface = [&](int I, int J) { return gfree(I, J) && (I % H == 0 || J % H == 0); };
  auto is_corner = [&](int I, int J) { return gfree(I, J) && I % H == 0 && J % H == 0; };
  std::map<long long, int> gmap, cmap;  // global node id -> interface / corner index
  for (int J = 1; J <= N - 1; ++J)
    for (int I = 1; I <= N - 1; ++I) {
      if (on_iface(I, J)) gmap[(long long)J * (N + 1) + I] = (int)gmap.size();
      if (is_corner(I, J)) cmap[(long long)J * (N + 1) + I] = (int)cmap.size();
    }
  pr.nG = (int)gmap.size();
  pr.nC = (int)cmap.size();
  pr.cls.assign((size_t)nsub * nl, DIRICHLET);
  pr.gidx.assign((size_t)nsub * nl, -1);
  pr.cidx.assign((size_t)nsub * nl, -1);
  pr.cells.assign((size_t)nsub * nl, 0);
  pr.kapE.assign((size_t)nsub * nl * PI, 0.0);
  pr.kapN.assign((size_t)nsub * nl * PI, 0.0);
  pr.owners.assign((size_t)pr.nG * 4, -1);
  pr.cowners.assign((size_t)pr.nC * 4, -1);
  pr.Dw.assign(pr.nG, 0.0);
  pr.n_gam.assign(nsub, 0);
  pr.loc_corner.assign((size_t)nsub * 4, -1);
  pr.n_loc_corner.assign(nsub, 0);
  pr.free_of_local.assign((size_t)nsub * nl, -1);
  pr.n_free = (N - 1) * (N - 1);
  pr.free_owner.assign(pr.n_free, -1);
  pr.u0_local.assign((size_t)nsub * nl, 0.0);
  std::vector<int> mult(pr.nG, 0), cmult(pr.nC, 0);
  std::vector<std::vector<int>> gam(nsub);
  for (int sy_ = 0; sy_ < sx; ++sy_)
    for (int sx_ = 0; sx_ < sx; ++sx_) {
      int sub = sy_ * sx + sx_;
      for (int lj = 0; lj <= H; ++lj)
        for (int li = 0; li <= H; ++li) {
          int I = sx_ * H + li, J = sy_ * H + lj, ln = lj * L + li;
          size_t o = (size_t)sub * nl + ln;
          uint8_t cb = 0;
          if (li > 0 && lj > 0) cb |= 1;
          if (li < H && lj > 0) cb |= 2;
          if (li > 0 && lj < H) cb |= 4;
          if (li < H && lj < H) cb |= 8;
          pr.cells[o] = cb;
          if (!gfree(I, J)) continue;
          long long gid = (long long)J * (N + 1) + I;
          int fidx = (J - 1) * (N - 1) + (I - 1);
          pr.free_of_local[o] = fidx;
          if (pr.free_owner[fidx] < 0) pr.free_owner[fidx] = (int)o;
          if (is_corner(I, J)) {
            pr.cls[o] = CORNER;
            int c = cmap[gid];
            pr.cidx[o] = c;
            pr.cowners[(size_t)c * 4 + cmult[c]++] = (int)o;
            pr.loc_corner[(size_t)sub * 4 + pr.n_loc_corner[sub]++] = ln;
          } else if (on_iface(I, J)) {
            pr.cls[o] = REMAINING;
          } else {
            pr.cls[o] = INTERIOR;
          }
          if (on_iface(I, J)) {
            int g = gmap[gid];
            pr.gidx[o] = g;
            pr.owners[(size_t)g * 4 + mult[g]++] = (int)o;
            gam[sub].push_back(ln);
          }
          if (src.kind == 1) {
            double x = I * h - src.x0, y = J * h - src.y0;
            pr.u0_local[o] = src.amp * std::exp(-(x * x + y * y) / (src.width * src.width));
          }
        }
    }
  // stiffness edge weights from each subdomain's own elements (graph-Laplacian form of the P1
  // stiffness on right triangles: each leg carries half the element coefficient, the hypotenuse
  // none); subdomains write disjoint ranges and are filled in parallel
  parallel_cyclic(0, nsub, [&](int sub) {
    const int sy_ = sub / sx, sx_ = sub % sx;
    for (int lj = 0; lj <= H; ++lj)
      for (int li = 0; li <= H; ++li) {
        const int I = sx_ * H + li, J = sy_ * H + lj, ln = lj * L + li;
        double* kE = &pr.kapE[((size_t)sub * nl + ln) * PI];
        double* kN = &pr.kapN[((size_t)sub * nl + ln) * PI];
        for (int i = 0; i < PI; ++i) {
          double e = 0.0, n = 0.0;
          if (li < H) {
            if (lj < H) e += 0.5 * cT1[((size_t)J * N + I) * PI + i];
            if (lj > 0) e += 0.5 * cT2[((size_t)(J - 1) * N + I) * PI + i];
          }
          if (lj < H) {
            if (li > 0) n += 0.5 * cT1[((size_t)J * N + (I - 1)) * PI + i];
            if (li < H) n += 0.5 * cT2[((size_t)J * N + I) * PI + i];
          }
          kE[i] = e;
          kN[i] = n;
        }
      }
  });
  for (int g = 0; g < pr.nG; ++g) pr.Dw[g] = 1.0 / mult[g];
  pr.max_corner = 0;
  pr.nGam = 0;
  for (int s_ = 0; s_ < nsub; ++s_) {
    pr.n_gam[s_] = (int)gam[s_].size();
    pr.nGam = std::max(pr.nGam, pr.n_gam[s_]);
    pr.max_corner = std::max(pr.max_corner, pr.n_loc_corner[s_]);
  }
  pr.gam_ln.assign((size_t)nsub * std::max(pr.nGam, 1), -1);
  for (int s_ = 0; s_ < nsub; ++s_)
    for (int q = 0; q < pr.n_gam[s_]; ++q) pr.gam_ln[(size_t)s_ * pr.nGam + q] = gam[s_][q];

  // point load nodes: P1 values at the source point, split over owning subdomains with D_s
  pr.load_node.clear(); pr.load_w.clear();
  if (src.kind == 2) {
    int i = std::min((int)std::floor(src.x0 / h), N - 1);
    int j = std::min((int)std::floor(src.y0 / h), N - 1);
    double fx = src.x0 / h - i, fy = src.y0 / h - j;
    int vi[3], vj[3];
    double vw[3];
    if (fy <= fx) {
      vi[0] = i; vj[0] = j; vw[0] = 1.0 - fx;
      vi[1] = i + 1; vj[1] = j; vw[1] = fx - fy;
      vi[2] = i + 1; vj[2] = j + 1; vw[2] = fy;
    } else {
      vi[0] = i; vj[0] = j; vw[0] = 1.0 - fy;
      vi[1] = i + 1; vj[1] = j + 1; vw[1] = fx;
      vi[2] = i; vj[2] = j + 1; vw[2] = fy - fx;
    }
    for (int v = 0; v < 3; ++v) {
      if (vw[v] == 0.0 || !gfree(vi[v], vj[v])) continue;
      // every subdomain whose closed region contains the node receives D_s * value
      std::vector<int> own;
      for (int sy_ = 0; sy_ < sx; ++sy_)
        for (int sx_ = 0; sx_ < sx; ++sx_) {
          int li = vi[v] - sx_ * H, lj = vj[v] - sy_ * H;
          if (li < 0 || li > H || lj < 0 || lj > H) continue;
          own.push_back((sy_ * sx + sx_) * nl + lj * L + li);
        }
      for (int o : own) {
        pr.load_node.push_back(o);
        pr.load_w.push_back(src.amp * vw[v] / (double)own.size());
      }
    }
  }
  return "";
}

// ---- general partitions of unstructured triangle meshes ----
std::string build_mesh_problem(MeshProblem& mp, int nv, const double* xy, const uint8_t* dirichlet, int ne,
                               const int* tri, const int* part, int M, double sigma, double bx, double by,
                               double g0, int p, int p_in, const double* modes, const double* lambdas) {
  if (nv < 3 || ne < 1 || !xy || !dirichlet || !tri || !part) return "mesh: vertices, triangles and partition required";
  if (M < 0 || M > 12 || p < 0 || p_in < 0 || p > 10 || p_in > 20) return "pce/kl: unsupported M, p or p_in";
  if (!(sigma >= 0)) return "kl: sigma >= 0 required";
  if (M > 0 && !modes && !(bx > 0 && by > 0)) return "kl: correlation lengths must be positive";
  if (modes && M > 0) {
    if (!lambdas) return "kl: modes given without lambdas";
    for (int n = 0; n < M; ++n)
      if (!(lambdas[n] > 0) || !std::isfinite(lambdas[n])) return "kl: lambdas must be positive and finite";
    for (size_t q = 0; q < (size_t)M * ne; ++q)
      if (!std::isfinite(modes[q])) return "kl: modes must be finite";
  }
  int nsub = 0;
  for (int e = 0; e < ne; ++e) {
    for (int a = 0; a < 3; ++a)
      if (tri[3 * e + a] < 0 || tri[3 * e + a] >= nv) return "mesh: triangle vertex out of range";
    if (part[e] < 0) return "mesh: negative subdomain id";
    nsub = std::max(nsub, part[e] + 1);
  }
  {
    std::vector<char> used(nsub, 0);
    for (int e = 0; e < ne; ++e) used[part[e]] = 1;
    for (int s = 0; s < nsub; ++s)
      if (!used[s]) return "mesh: subdomain ids must be 0 .. nsub - 1, each used";
  }
  mp = MeshProblem{};
  mp.nv = nv; mp.ne = ne; mp.nsub = nsub; mp.M = M; mp.p = p; mp.p_in = p_in;
  const auto Ain = multi_indices(M, p_in);
  mp.P = (int)multi_indices(M, p).size();
  mp.PI = (int)Ain.size();
  const int PI = mp.PI;

  // element geometry: doubled signed area, unit-coefficient P1 stiffness from the barycentric
  // gradients grad(phi_a) = (y_b - y_c, x_c - x_b) / (2 area)
  std::vector<double> area(ne), Ke((size_t)ne * 9), cx(ne), cy(ne);
  for (int e = 0; e < ne; ++e) {
    const int* v = tri + 3 * e;
    const double x1 = xy[2 * v[0]], y1 = xy[2 * v[0] + 1], x2 = xy[2 * v[1]], y2 = xy[2 * v[1] + 1];
    const double x3 = xy[2 * v[2]], y3 = xy[2 * v[2] + 1];
    const double a2 = (x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1);
    if (!(std::fabs(a2) > 0)) return "mesh: degenerate triangle";
    area[e] = 0.5 * std::fabs(a2);
    const double b[3] = {y2 - y3, y3 - y1, y1 - y2}, c[3] = {x3 - x2, x1 - x3, x2 - x1};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Ke[(size_t)e * 9 + i * 3 + j] = (b[i] * b[j] + c[i] * c[j]) / (4.0 * area[e]);
    cx[e] = (x1 + x2 + x3) / 3.0;
    cy[e] = (y1 + y2 + y3) / 3.0;
  }

  // KL: top M products of the 1-D eigenpairs (ties: lower y index, then x index), or the caller's
  std::vector<Eig1> ex, ey;
  const std::vector<KLCand> cand = kl_select(M, bx, by, ex, ey);
  mp.kl_lambda.resize(M);
  for (int n = 0; n < M; ++n) mp.kl_lambda[n] = modes ? lambdas[n] : cand[n].lam;
  // PCE coefficients of exp(g) per element centroid: exp(g0 + |g|^2 / 2) prod_n g_n^{a_n} / sqrt(a_n!)
  std::vector<double> coef((size_t)ne * PI);
  for (int e = 0; e < ne; ++e) {
    std::vector<double> g(M);
    double s2 = 0.0;
    for (int n = 0; n < M; ++n) {
      g[n] = modes ? sigma * std::sqrt(lambdas[n]) * modes[(size_t)n * ne + e]
                   : sigma * std::sqrt(cand[n].lam) * phi1(cx[e], ex[cand[n].ix]) * phi1(cy[e], ey[cand[n].iy]);
      s2 += g[n] * g[n];
    }
    const double c0 = std::exp(g0 + 0.5 * s2);
    for (int i = 0; i < PI; ++i) {
      double v = c0;
      for (int n = 0; n < M; ++n)
        for (int a = 0; a < Ain[i][n]; ++a) v *= g[n] / std::sqrt((double)(a + 1));
      coef[(size_t)e * PI + i] = v;
    }
  }

  // subdomains of each vertex, interface edges (two triangles of different subdomains) per vertex
  std::vector<std::vector<int>> vsub(nv);
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a) {
      auto& l = vsub[tri[3 * e + a]];
      if (std::find(l.begin(), l.end(), part[e]) == l.end()) l.push_back(part[e]);
    }
  struct HalfEdge { int u, v, e; };
  std::vector<HalfEdge> he;
  he.reserve((size_t)3 * ne);
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a) {
      const int u = tri[3 * e + a], v = tri[3 * e + (a + 1) % 3];
      he.push_back({std::min(u, v), std::max(u, v), e});
    }
  std::sort(he.begin(), he.end(), [](const HalfEdge& a, const HalfEdge& b) {
    return a.u != b.u ? a.u < b.u : a.v != b.v ? a.v < b.v : a.e < b.e;
  });
  std::vector<std::vector<std::pair<long long, int>>> icount(nv);  // (pair key, interface edges)
  for (size_t q = 0; q < he.size();) {
    size_t r = q;
    while (r < he.size() && he[r].u == he[q].u && he[r].v == he[q].v) ++r;
    if (r - q > 2) return "mesh: an edge shared by more than two triangles";
    if (r - q == 2) {
      const int pa = part[he[q].e], pb = part[he[q + 1].e];
      if (pa != pb) {
        const long long key = (long long)std::min(pa, pb) * nsub + std::max(pa, pb);
        for (int x : {he[q].u, he[q].v}) {
          auto& l = icount[x];
          auto it = std::find_if(l.begin(), l.end(), [key](const std::pair<long long, int>& t) { return t.first == key; });
          if (it == l.end()) l.push_back({key, 1});
          else ++it->second;
        }
      }
    }
    q = r;
  }
  mp.vclass.assign(nv, DIRICHLET);
  mp.vmult.assign(nv, 0);
  mp.free_idx.assign(nv, -1);
  mp.iface_idx.assign(nv, -1);
  mp.corner_idx.assign(nv, -1);
  for (int v = 0; v < nv; ++v) {
    const int m = (int)vsub[v].size();
    mp.vmult[v] = m;
    if (dirichlet[v] || m == 0) continue;
    if (m == 1) {
      mp.vclass[v] = INTERIOR;
    } else if (m >= 3) {
      mp.vclass[v] = CORNER;
    } else {
      const long long key = (long long)std::min(vsub[v][0], vsub[v][1]) * nsub + std::max(vsub[v][0], vsub[v][1]);
      int cnt = 0;
      for (const auto& t : icount[v])
        if (t.first == key) cnt = t.second;
      mp.vclass[v] = cnt == 2 ? REMAINING : CORNER;
    }
  }
  for (int v = 0; v < nv; ++v) {
    if (mp.vclass[v] == DIRICHLET) continue;
    mp.free_idx[v] = mp.n_free++;
    if (mp.vclass[v] == REMAINING || mp.vclass[v] == CORNER) mp.iface_idx[v] = mp.nG++;
    if (mp.vclass[v] == CORNER) mp.corner_idx[v] = mp.nC++;
  }

  // per subdomain: local vertices (interior, remaining, corners, Dirichlet; ascending within a
  // class), edges with their weights per input mode, triangles
  std::vector<std::vector<int>> selems(nsub);
  for (int e = 0; e < ne; ++e) selems[part[e]].push_back(e);
  std::vector<int> loc(nv, -1);
  auto rank = [&](int v) { const int c = mp.vclass[v]; return c == DIRICHLET ? 4 : c; };
  mp.sub_vptr.assign(1, 0);
  mp.sub_eptr.assign(1, 0);
  mp.sub_tptr.assign(1, 0);
  for (int s = 0; s < nsub; ++s) {
    std::vector<int> verts;
    for (int e : selems[s])
      for (int a = 0; a < 3; ++a) verts.push_back(tri[3 * e + a]);
    std::sort(verts.begin(), verts.end());
    verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
    std::stable_sort(verts.begin(), verts.end(), [&](int a, int b) { return rank(a) < rank(b); });
    for (size_t k = 0; k < verts.size(); ++k) loc[verts[k]] = (int)k;
    std::map<std::pair<int, int>, std::vector<double>> edges;
    for (int e : selems[s]) {
      const int* v = tri + 3 * e;
      for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b) {
          const int la = loc[v[a]], lb = loc[v[b]];
          auto& w = edges[{std::min(la, lb), std::max(la, lb)}];
          if (w.empty()) w.assign(PI, 0.0);
          const double k = Ke[(size_t)e * 9 + a * 3 + b];
          for (int i = 0; i < PI; ++i) w[i] -= coef[(size_t)e * PI + i] * k;
        }
      for (int a = 0; a < 3; ++a) mp.tri_loc.push_back(loc[v[a]]);
      mp.tri_area.push_back(area[e]);
    }
    for (const auto& kv : edges) {
      mp.edge_u.push_back(kv.first.first);
      mp.edge_v.push_back(kv.first.second);
      mp.edge_w.insert(mp.edge_w.end(), kv.second.begin(), kv.second.end());
    }
    mp.sub_verts.insert(mp.sub_verts.end(), verts.begin(), verts.end());
    mp.sub_vptr.push_back((int)mp.sub_verts.size());
    mp.sub_eptr.push_back((int)mp.edge_u.size());
    mp.sub_tptr.push_back((int)mp.tri_area.size());
    for (int v : verts) loc[v] = -1;
  }
  return "";
}

// Every index the device kernels follow stays inside its table: local columns and owners inside the
// subdomain's rows, interface / corner indices inside their ranges, patterns inside nl.
static std::string check_mesh_tables(const Problem& pr, const MeshRows& mr) {
  const long long nloc = (long long)pr.nsub * pr.nl;
  if ((long long)mr.row_ptr.size() != nloc + 1 || mr.row_ptr[0] != 0) return "mesh tables: row pointers";
  for (long long r = 0; r < nloc; ++r) {
    if (mr.row_ptr[r + 1] < mr.row_ptr[r]) return "mesh tables: row pointers";
    for (int q = mr.row_ptr[r]; q < mr.row_ptr[r + 1]; ++q)
      if (mr.col[q] < 0 || mr.col[q] >= pr.nl || pr.cls[(size_t)(r / pr.nl) * pr.nl + mr.col[q]] == DIRICHLET)
        return "mesh tables: column outside the subdomain's free rows";
  }
  if ((long long)mr.col.size() != mr.row_ptr[nloc] || mr.mval.size() != mr.col.size() ||
      mr.kval.size() != mr.col.size() * (size_t)pr.PI)
    return "mesh tables: entry arrays";
  for (int s = 0; s < pr.nsub; ++s)
    for (int pat = 0; pat < 3; ++pat) {
      const int n = mr.npat[(size_t)pat * pr.nsub + s];
      if (n < 0 || n > pr.nl) return "mesh tables: pattern rows";
    }
  auto in_loc = [&](int o) { return o >= 0 && o < nloc; };
  for (long long o = 0; o < nloc; ++o) {
    const int c = pr.cls[o];
    if ((c == REMAINING || c == CORNER) != (pr.gidx[o] >= 0) || pr.gidx[o] >= pr.nG) return "mesh tables: gidx";
    if ((c == CORNER) != (pr.cidx[o] >= 0) || pr.cidx[o] >= pr.nC) return "mesh tables: cidx";
    if ((c != DIRICHLET) != (pr.free_of_local[o] >= 0) || pr.free_of_local[o] >= pr.n_free)
      return "mesh tables: free_of_local";
  }
  for (int g = 0; g < pr.nG; ++g)
    for (int q = 0; q < pr.mo; ++q) {
      const int o = pr.owners[(size_t)g * pr.mo + q];
      if (o != -1 && (!in_loc(o) || pr.gidx[o] != g)) return "mesh tables: owners";
    }
  for (int c = 0; c < pr.nC; ++c)
    for (int q = 0; q < pr.mo; ++q) {
      const int o = pr.cowners[(size_t)c * pr.mo + q];
      if (o != -1 && (!in_loc(o) || pr.cidx[o] != c)) return "mesh tables: cowners";
    }
  for (int s = 0; s < pr.nsub; ++s) {
    if (pr.n_gam[s] < 0 || pr.n_gam[s] > pr.nGam || pr.n_loc_corner[s] < 0 || pr.n_loc_corner[s] > pr.mc)
      return "mesh tables: local interface counts";
    for (int q = 0; q < pr.n_gam[s]; ++q) {
      const int a = pr.gam_ln[(size_t)s * pr.nGam + q];
      if (a < 0 || a >= pr.nl || pr.gidx[(size_t)s * pr.nl + a] < 0) return "mesh tables: gam_ln";
    }
    for (int q = 0; q < pr.n_loc_corner[s]; ++q) {
      const int a = pr.loc_corner[(size_t)s * pr.mc + q];
      if (a < 0 || a >= pr.nl || pr.cidx[(size_t)s * pr.nl + a] < 0) return "mesh tables: loc_corner";
    }
  }
  for (int f = 0; f < pr.n_free; ++f)
    if (!in_loc(pr.free_owner[f]) || pr.free_of_local[pr.free_owner[f]] != f) return "mesh tables: free_owner";
  for (int o : pr.load_node)
    if (!in_loc(o) || pr.cls[o] == DIRICHLET) return "mesh tables: load_node";
  return "";
}

std::string mesh_to_problem(Problem& pr, MeshRows& mr, const MeshProblem& mp, const double* xy, const int* tri,
                            double dt, double alpha0, double alpha1, const SourceDesc& src) {
  if (!(dt > 0)) return "params: dt > 0 required";
  if (mp.nsub < 1 || (int)mp.sub_vptr.size() != mp.nsub + 1) return "mesh: set-up tables missing";
  const int nsub = mp.nsub, PI = mp.PI, nv = mp.nv;
  pr = Problem{};
  pr.nsub = nsub; pr.M = mp.M; pr.p = mp.p; pr.p_in = mp.p_in; pr.P = mp.P; pr.PI = PI;
  pr.dt = dt; pr.alpha0 = alpha0; pr.alpha1 = alpha1; pr.src = src;
  pr.kl_lambda = mp.kl_lambda;
  pr.alpha_out = multi_indices(mp.M, mp.p);
  triple_table(pr, multi_indices(mp.M, mp.p_in), pr.alpha_out);

  // local layout: the free vertices of each subdomain (they come first in sub_verts)
  std::vector<int> nfree(nsub, 0), nint(nsub, 0), nrem(nsub, 0), ncor(nsub, 0);
  int nl = 1;
  for (int s = 0; s < nsub; ++s) {
    for (int q = mp.sub_vptr[s]; q < mp.sub_vptr[s + 1]; ++q) {
      const int c = mp.vclass[mp.sub_verts[q]];
      if (c == DIRICHLET) break;
      ++nfree[s];
      if (c == INTERIOR) ++nint[s];
      else if (c == REMAINING) ++nrem[s];
      else ++ncor[s];
    }
    nl = std::max(nl, nfree[s]);
  }
  pr.nl = nl;
  pr.nG = mp.nG; pr.nC = mp.nC; pr.n_free = mp.n_free;
  int mo = 1;
  for (int v = 0; v < nv; ++v)
    if (mp.iface_idx[v] >= 0) mo = std::max(mo, mp.vmult[v]);
  int mc = 1;
  for (int s = 0; s < nsub; ++s) mc = std::max(mc, ncor[s]);
  pr.mo = mo; pr.mc = mc;
  pr.cls.assign((size_t)nsub * nl, DIRICHLET);
  pr.gidx.assign((size_t)nsub * nl, -1);
  pr.cidx.assign((size_t)nsub * nl, -1);
  pr.owners.assign((size_t)std::max(pr.nG, 1) * mo, -1);
  pr.cowners.assign((size_t)std::max(pr.nC, 1) * mo, -1);
  pr.Dw.assign(std::max(pr.nG, 1), 0.0);
  pr.n_gam.assign(nsub, 0);
  pr.loc_corner.assign((size_t)nsub * mc, -1);
  pr.n_loc_corner.assign(nsub, 0);
  pr.free_of_local.assign((size_t)nsub * nl, -1);
  pr.free_owner.assign(std::max(pr.n_free, 1), -1);
  pr.u0_local.assign((size_t)nsub * nl, 0.0);
  std::vector<int> mult(std::max(pr.nG, 1), 0), cmult(std::max(pr.nC, 1), 0);
  pr.nGam = 1;
  for (int s = 0; s < nsub; ++s) {
    pr.n_gam[s] = nfree[s] - nint[s];
    pr.nGam = std::max(pr.nGam, pr.n_gam[s]);
  }
  pr.gam_ln.assign((size_t)nsub * pr.nGam, -1);
  for (int s = 0; s < nsub; ++s) {
    const int base = mp.sub_vptr[s];
    for (int a = 0; a < nfree[s]; ++a) {
      const int v = mp.sub_verts[base + a];
      const size_t o = (size_t)s * nl + a;
      const uint8_t c = mp.vclass[v];
      pr.cls[o] = c;
      const int f = mp.free_idx[v];
      if (f < 0 || f >= pr.n_free) return "mesh: free numbering inconsistent";
      pr.free_of_local[o] = f;
      if (pr.free_owner[f] < 0) pr.free_owner[f] = (int)o;
      if (c == REMAINING || c == CORNER) {
        const int g = mp.iface_idx[v];
        if (g < 0 || g >= pr.nG || mult[g] >= mo) return "mesh: interface numbering inconsistent";
        pr.gidx[o] = g;
        pr.owners[(size_t)g * mo + mult[g]++] = (int)o;
        pr.gam_ln[(size_t)s * pr.nGam + (a - nint[s])] = a;
      }
      if (c == CORNER) {
        const int cc = mp.corner_idx[v];
        if (cc < 0 || cc >= pr.nC || cmult[cc] >= mo) return "mesh: corner numbering inconsistent";
        pr.cidx[o] = cc;
        pr.cowners[(size_t)cc * mo + cmult[cc]++] = (int)o;
        pr.loc_corner[(size_t)s * mc + pr.n_loc_corner[s]++] = a;
      }
      if (src.kind == 1) {
        const double x = xy[2 * v] - src.x0, y = xy[2 * v + 1] - src.y0;
        pr.u0_local[o] = src.amp * std::exp(-(x * x + y * y) / (src.width * src.width));
      }
    }
  }
  for (int g = 0; g < pr.nG; ++g) {
    if (mult[g] < 2) return "mesh: interface vertex with fewer than two owners";
    pr.Dw[g] = 1.0 / mult[g];
  }
  pr.max_corner = 0;
  for (int s = 0; s < nsub; ++s) pr.max_corner = std::max(pr.max_corner, pr.n_loc_corner[s]);
  mr.npat.assign((size_t)3 * nsub, 0);
  for (int s = 0; s < nsub; ++s) {
    mr.npat[s] = nint[s];
    mr.npat[nsub + s] = nint[s] + nrem[s];
    mr.npat[2 * nsub + s] = nfree[s];
  }

  // sparse rows: stiffness K_i[a][a] = sum of the weights of a's edges (P1 element rows sum to zero),
  // K_i[a][b] = -w_i(a, b) between free vertices; mass area / 12 off the diagonal and area / 6 on it
  mr.row_ptr.assign((size_t)nsub * nl + 1, 0);
  mr.col.clear(); mr.kval.clear(); mr.mval.clear();
  for (int s = 0; s < nsub; ++s) {
    const int nf = nfree[s];
    std::vector<std::map<int, size_t>> rows(nf);   // column -> entry index in the row's buffer
    std::vector<std::vector<double>> kb(nf), mb(nf);
    auto entry = [&](int a, int b) -> size_t {
      auto it = rows[a].find(b);
      if (it != rows[a].end()) return it->second;
      const size_t q = mb[a].size();
      rows[a][b] = q;
      mb[a].push_back(0.0);
      kb[a].resize(kb[a].size() + PI, 0.0);
      return q;
    };
    for (int a = 0; a < nf; ++a) entry(a, a);
    for (int e = mp.sub_eptr[s]; e < mp.sub_eptr[s + 1]; ++e) {
      const int u = mp.edge_u[e], v = mp.edge_v[e];
      const double* w = &mp.edge_w[(size_t)e * PI];
      if (u < nf) { const size_t q = entry(u, u); for (int i = 0; i < PI; ++i) kb[u][q * PI + i] += w[i]; }
      if (v < nf) { const size_t q = entry(v, v); for (int i = 0; i < PI; ++i) kb[v][q * PI + i] += w[i]; }
      if (u < nf && v < nf) {
        const size_t q1 = entry(u, v), q2 = entry(v, u);
        for (int i = 0; i < PI; ++i) {
          kb[u][q1 * PI + i] -= w[i];
          kb[v][q2 * PI + i] -= w[i];
        }
      }
    }
    for (int t = mp.sub_tptr[s]; t < mp.sub_tptr[s + 1]; ++t) {
      const int* lv = &mp.tri_loc[(size_t)t * 3];
      const double ar = mp.tri_area[t];
      for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) {
          const int a = lv[x], b = lv[y];
          if (a >= nf || b >= nf) continue;
          mb[a][entry(a, b)] += (x == y ? ar / 6.0 : ar / 12.0);
        }
    }
    for (int a = 0; a < nl; ++a) {
      const size_t row = (size_t)s * nl + a;
      if (a < nf) {
        // diagonal first, then ascending columns
        std::vector<int> cols;
        cols.push_back(a);
        for (const auto& kv : rows[a])
          if (kv.first != a) cols.push_back(kv.first);
        for (int b : cols) {
          const size_t q = rows[a][b];
          mr.col.push_back(b);
          mr.mval.push_back(mb[a][q]);
          mr.kval.insert(mr.kval.end(), kb[a].begin() + q * PI, kb[a].begin() + (q + 1) * PI);
        }
      }
      mr.row_ptr[row + 1] = (int)mr.col.size();
    }
  }

  // point source: P1 values in the first triangle containing (x0, y0), split over the owning
  // subdomains with D_s
  pr.load_node.clear(); pr.load_w.clear();
  if (src.kind == 2) {
    int found = -1;
    double lam[3] = {0, 0, 0};
    for (int e = 0; e < mp.ne && found < 0; ++e) {
      const int* v = tri + 3 * e;
      const double ax = xy[2 * v[0]], ay = xy[2 * v[0] + 1], bx = xy[2 * v[1]], by = xy[2 * v[1] + 1];
      const double cx = xy[2 * v[2]], cy = xy[2 * v[2] + 1];
      const double det = (bx - ax) * (cy - ay) - (cx - ax) * (by - ay);
      const double l1 = ((src.x0 - ax) * (cy - ay) - (cx - ax) * (src.y0 - ay)) / det;
      const double l2 = ((bx - ax) * (src.y0 - ay) - (src.x0 - ax) * (by - ay)) / det;
      const double l0 = 1.0 - l1 - l2;
      if (l0 >= -1e-12 && l1 >= -1e-12 && l2 >= -1e-12) {
        found = e;
        lam[0] = l0; lam[1] = l1; lam[2] = l2;
      }
    }
    if (found < 0) return "source: the point (x0, y0) lies in no triangle of the mesh";
    for (int k = 0; k < 3; ++k) {
      const int v = tri[3 * found + k];
      if (lam[k] == 0.0 || mp.vclass[v] == DIRICHLET) continue;
      std::vector<int> own;
      for (int s = 0; s < nsub; ++s)
        for (int a = 0; a < nfree[s]; ++a)
          if (mp.sub_verts[mp.sub_vptr[s] + a] == v) own.push_back(s * nl + a);
      for (int o : own) {
        pr.load_node.push_back(o);
        pr.load_w.push_back(src.amp * lam[k] / (double)own.size());
      }
    }
  }
  return check_mesh_tables(pr, mr);
}

std::string partition_rcb(int nv, const double* xy, int ne, const int* tri, int nparts, int* part) {
  if (nv < 3 || ne < 1 || !xy || !tri || !part) return "partition: vertices and triangles required";
  if (nparts < 1 || nparts > ne) return "partition: 1 <= nparts <= triangles required";
  std::vector<double> cx(ne), cy(ne);
  for (int e = 0; e < ne; ++e) {
    const int a = tri[3 * e], b = tri[3 * e + 1], c = tri[3 * e + 2];
    if (a < 0 || a >= nv || b < 0 || b >= nv || c < 0 || c >= nv) return "partition: triangle vertex out of range";
    cx[e] = (xy[2 * a] + xy[2 * b] + xy[2 * c]) / 3.0;
    cy[e] = (xy[2 * a + 1] + xy[2 * b + 1] + xy[2 * c + 1]) / 3.0;
  }
  std::vector<int> ids(ne);
  for (int e = 0; e < ne; ++e) ids[e] = e;
  // explicit stack of (first, count, k, first id) ranges of ids
  struct Range { int lo, n, k, first; };
  std::vector<Range> todo{{0, ne, nparts, 0}};
  while (!todo.empty()) {
    const Range r = todo.back();
    todo.pop_back();
    if (r.k == 1) {
      for (int q = r.lo; q < r.lo + r.n; ++q) part[ids[q]] = r.first;
      continue;
    }
    double x0 = cx[ids[r.lo]], x1 = x0, y0 = cy[ids[r.lo]], y1 = y0;
    for (int q = r.lo; q < r.lo + r.n; ++q) {
      x0 = std::min(x0, cx[ids[q]]); x1 = std::max(x1, cx[ids[q]]);
      y0 = std::min(y0, cy[ids[q]]); y1 = std::max(y1, cy[ids[q]]);
    }
    const bool alongx = (x1 - x0) >= (y1 - y0);
    const std::vector<double>& major = alongx ? cx : cy;
    const std::vector<double>& minor = alongx ? cy : cx;
    std::stable_sort(ids.begin() + r.lo, ids.begin() + r.lo + r.n, [&](int a, int b) {
      if (major[a] != major[b]) return major[a] < major[b];
      return minor[a] < minor[b];
    });
    const int k0 = r.k / 2;
    const int n0 = (int)(((long long)r.n * k0) / r.k);
    todo.push_back({r.lo + n0, r.n - n0, r.k - k0, r.first + k0});
    todo.push_back({r.lo, n0, k0, r.first});
  }
  return "";
}

bool mesh_mean_inverse(const Problem& pr, const MeshRows& mr, int pat, double am, double bk,
                       std::vector<double>& out) {
  const int nsub = pr.nsub, nl = pr.nl, PI = pr.PI;
  out.assign((size_t)nsub * nl * nl, 0.0);
  for (int s = 0; s < nsub; ++s) {
    const int n = mr.npat[(size_t)pat * nsub + s];
    if (n == 0) continue;
    std::vector<double> A((size_t)n * n, 0.0);
    for (int a = 0; a < n; ++a) {
      const size_t row = (size_t)s * nl + a;
      for (int q = mr.row_ptr[row]; q < mr.row_ptr[row + 1]; ++q) {
        const int b = mr.col[q];
        if (b < n) A[(size_t)a * n + b] += am * mr.mval[q] + bk * mr.kval[(size_t)q * PI];
      }
    }
    if (!spd_inverse(A, n)) return false;
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) out[((size_t)s * nl + a) * nl + c] = A[(size_t)a * n + c];
  }
  return true;
}

bool spd_inverse(std::vector<double>& A, int n) {
  if (n <= 0) return true;
  if ((long long)A.size() < (long long)n * n) return false;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  // 1. Cholesky A = L L^T in place (lower triangle), blocked right-looking: factor the diagonal
  //    block, solve the panel below it (inner products over contiguous row segments), update the
  //    trailing lower triangle (row-parallel).
  constexpr int B = 64;
  bool spd = true;
  for (int k0 = 0; k0 < n && spd; k0 += B) {
    const int k1 = std::min(n, k0 + B);
    for (int j = k0; j < k1; ++j) {
      double d = a(j, j);
      for (int k = k0; k < j; ++k) d -= a(j, k) * a(j, k);
      if (!(d > 0.0)) { spd = false; break; }
      d = std::sqrt(d);
      a(j, j) = d;
      for (int i = j + 1; i < k1; ++i) {
        double s = a(i, j);
        for (int k = k0; k < j; ++k) s -= a(i, k) * a(j, k);
        a(i, j) = s / d;
      }
    }
    if (!spd) break;
    parallel_cyclic(k1, n, [&](int i) {
      for (int j = k0; j < k1; ++j) {  // panel row i: L[i, k0:k1] = A[i, k0:k1] L_kk^{-T}
        double s = a(i, j);
        for (int k = k0; k < j; ++k) s -= a(i, k) * a(j, k);
        a(i, j) = s / a(j, j);
      }
    });
    // trailing update A[i][j] -= L[i, k0:k1] . L[j, k0:k1] (k1 <= j <= i), after the whole panel is
    // known: with the panel transposed (Pt[k][j] = L[j][k0 + k]) row i is a sum of contiguous axpys
    // over j, one per panel column k
    const int nb = k1 - k0;
    std::vector<double> Pt((size_t)nb * n);
    for (int j = k1; j < n; ++j)
      for (int k = 0; k < nb; ++k) Pt[(size_t)k * n + j] = a(j, k0 + k);
    parallel_cyclic(k1, n, [&](int i) {
      double* ri = &A[(size_t)i * n];
      thread_local std::vector<double> acc;
      acc.assign((size_t)(i + 1), 0.0);
      for (int k = 0; k < nb; ++k) {
        const double l = ri[k0 + k];
        const double* pk = &Pt[(size_t)k * n];
        for (int j = k1; j <= i; ++j) acc[j] += l * pk[j];
      }
      for (int j = k1; j <= i; ++j) ri[j] -= acc[j];
    });
  }
  if (!spd) return false;
  // 2. A^{-1} = L^{-T} L^{-1}, in groups of MG consecutive columns c = c0 + t: Y = L^{-1} E (E the
  //    unit columns; rows above c0 are zero) and X = L^{-T} Y on rows c0..n-1, so that every row of
  //    L (forward) and of L^T (backward, copied row-major) is read once per group and serves MG
  //    right-hand sides (the inner loops run over the group's columns).  Only x[i] with i >= c is
  //    kept (the lower triangle); it is written to row c of `inv` and mirrored at the end.
  std::vector<double> U((size_t)n * n, 0.0);  // U = L^T, row-major
  for (int i = 0; i < n; ++i)
    for (int k = 0; k <= i; ++k) U[(size_t)k * n + i] = a(i, k);
  std::vector<double> inv((size_t)n * n, 0.0);
  constexpr int MG = 32;
  parallel_cyclic(0, (n + MG - 1) / MG, [&](int gi) {
    const int c0 = gi * MG, m = std::min(MG, n - c0), R = n - c0;
    std::vector<double> Y((size_t)R * MG, 0.0), X((size_t)R * MG, 0.0);
    double acc[MG];
    for (int i = c0; i < n; ++i) {  // forward: L y = e_c for the group's columns
      for (int t = 0; t < MG; ++t) acc[t] = 0.0;
      const double* li = &A[(size_t)i * n + c0];
      for (int k = 0; k < i - c0; ++k) {
        const double l = li[k];
        const double* yk = &Y[(size_t)k * MG];
        for (int t = 0; t < MG; ++t) acc[t] += l * yk[t];
      }
      const double d = a(i, i);
      double* yi = &Y[(size_t)(i - c0) * MG];
      for (int t = 0; t < MG; ++t) yi[t] = ((i == c0 + t ? 1.0 : 0.0) - acc[t]) / d;
    }
    for (int i = n - 1; i >= c0; --i) {  // backward: L^T x = y
      for (int t = 0; t < MG; ++t) acc[t] = 0.0;
      const double* ui = &U[(size_t)i * n];
      for (int k = i + 1; k < n; ++k) {
        const double u = ui[k];
        const double* xk = &X[(size_t)(k - c0) * MG];
        for (int t = 0; t < MG; ++t) acc[t] += u * xk[t];
      }
      const double d = ui[i];
      double* xi = &X[(size_t)(i - c0) * MG];
      const double* yi = &Y[(size_t)(i - c0) * MG];
      for (int t = 0; t < MG; ++t) xi[t] = (yi[t] - acc[t]) / d;
    }
    for (int t = 0; t < m; ++t)
      for (int i = c0 + t; i < n; ++i) inv[(size_t)(c0 + t) * n + i] = X[(size_t)(i - c0) * MG + t];
  });
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) A[(size_t)i * n + j] = A[(size_t)j * n + i] = inv[(size_t)i * n + j];
  return true;
}

}  // namespace sgh
