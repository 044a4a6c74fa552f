// SG-DD wave solver: device orchestration and the C ABI declared in include/sg.h.
//
// Per time step (Alg. 1, stochastic form of Sec. 5):
//   a1 effective load  f~ = f + M u~_m + C u~_c                     (Eqs. fparts, UmCm)
//   a2 condensed RHS   G = sum_s R_s^T (f~_G - K_GI K_II^{-1} f~_I)  (Eq. Sto_Schur)
//   a3 initial guess   previous step's interface solution            (Alg. 1)
//   a4 PCG on S u_G = G with the two-level NN preconditioner         (Eq. NNCP2)
//   a6 interior        u_I = K_II^{-1} (f~_I - K_IG u_G)
//   a7 Newmark update  a_{n+1}, v_{n+1}                               (Sec. 2)
// Subdomain Dirichlet / Neumann problems are solved by a batched CG over all subdomains (and
// right-hand sides) preconditioned by the exact mean operator I (x) A0^{-1} (line-block
// factorisation); the CG runs to a tight relative residual so the Schur operator is applied to
// full working precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sg.h"
#include "sg_host.hpp"
#include "sg_kernels.cuh"

using sgk::Op;

namespace {

constexpr double ZETA = 0.25, GAMMA = 0.5;

template <typename T>
struct InnerWS {
  T *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double *rz = nullptr, *rz_new = nullptr, *pq = nullptr, *rr = nullptr, *bb = nullptr;
  int *active = nullptr, *nactive = nullptr;
  int cap_nb = 0;
};

struct LineFactor {
  double* Sinv = nullptr;  // [sub][L][L][L]
  double* Bd = nullptr;    // [sub][L][L]
  double* Bu = nullptr;
  float* Sinv32 = nullptr;
  float* Bd32 = nullptr;
  float* Bu32 = nullptr;
};

}  // namespace

struct sg_handle_s {
  sgh::Problem pr;
  cudaStream_t st = nullptr;
  std::string err;
  int precision = SG_FP64, warm = SG_WARM_PREV;
  double tol = 1e-8, inner_tol = 1e-14;
  int max_iter = 500, inner_max = 400;
  double am = 0, bk = 0;
  long long step = 0;
  // device problem data
  uint8_t *cls = nullptr, *cells = nullptr;
  double *kapE = nullptr, *kapN = nullptr, *gk_v = nullptr;
  float *kapE32 = nullptr, *kapN32 = nullptr, *gk_v32 = nullptr;
  int *gk_ptr = nullptr, *gk_i = nullptr, *gk_j = nullptr;
  int *gidx = nullptr, *cidx = nullptr, *owners = nullptr, *cowners = nullptr, *gam_ln = nullptr;
  int *n_gam = nullptr, *loc_corner = nullptr, *n_loc_corner = nullptr, *free_owner = nullptr;
  int *free_of_local = nullptr;
  double *Dw = nullptr, *nodew = nullptr;
  int* load_node = nullptr;
  double* load_w = nullptr;
  int nload = 0;
  LineFactor lf[2];  // 0: Dirichlet (interior free), 1: Neumann (interior + remaining free)
  // coarse space
  double *Phi = nullptr, *Finv = nullptr;
  int nCd = 0, Rc = 0;
  // state and step work (local layout)
  double *U = nullptr, *V = nullptr, *A = nullptr, *um = nullptr, *uc = nullptr, *xm = nullptr;
  double *ft = nullptr, *Unew = nullptr, *wa = nullptr, *wb = nullptr, *wc = nullptr, *wd = nullptr;
  double* fext = nullptr;  // n_free
  double* outbuf = nullptr;
  // interface vectors
  double *xG = nullptr, *rG = nullptr, *zG = nullptr, *pG = nullptr, *qG = nullptr, *gG = nullptr;
  double *dC = nullptr, *uC = nullptr, *scal = nullptr;
  double* hscal = nullptr;  // pinned host scalars
  int* hint = nullptr;      // pinned host ints
  InnerWS<double> ws;
  std::vector<void*> allocs;
  long long bytes = 0;
  long long inner_iters = 0;
  std::vector<int> iters;
  std::vector<double> relres;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  Op<double> op64() const {
    Op<double> o;
    o.cls = cls; o.cells = cells; o.kapE = kapE; o.kapN = kapN;
    o.gk_ptr = gk_ptr; o.gk_i = gk_i; o.gk_j = gk_j; o.gk_v = gk_v;
    o.L = pr.L; o.nl = pr.nl; o.P = pr.P; o.PI = pr.PI; o.mass_h = pr.h * pr.h / 24.0;
    return o;
  }
  // operator restricted to subdomains [s0, ...)
  Op<double> op64_from(int s0) const {
    Op<double> o = op64();
    o.cls += (size_t)s0 * pr.nl;
    o.cells += (size_t)s0 * pr.nl;
    o.kapE += (size_t)s0 * pr.nl * pr.PI;
    o.kapN += (size_t)s0 * pr.nl * pr.PI;
    return o;
  }
  long long nloc() const { return (long long)pr.nsub * pr.nl; }
  long long nvec() const { return (long long)pr.nsub * pr.nl * pr.P; }
  long long nGd() const { return (long long)pr.nG * pr.P; }
};

static std::string g_setup_err;

#define CK(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);            \
      return SG_ECUDA;                                                        \
    }                                                                         \
  } while (0)

#define CKL()                                                                 \
  do {                                                                        \
    cudaError_t e_ = cudaPeekAtLastError();                                   \
    if (e_ != cudaSuccess) {                                                  \
      h->err = std::string("kernel launch: ") + cudaGetErrorString(e_);       \
      return SG_ECUDA;                                                        \
    }                                                                         \
  } while (0)

#define RET(x)                   \
  do {                           \
    int r_ = (x);                \
    if (r_ != SG_OK) return r_;  \
  } while (0)

static inline unsigned nblk(long long n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

template <typename T>
static int dalloc(sg_handle h, T** p, long long n) {
  if (n <= 0) n = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * (size_t)n);
  if (e != cudaSuccess) {
    h->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return SG_ENOMEM;
  }
  h->allocs.push_back(q);
  h->bytes += (long long)sizeof(T) * n;
  *p = (T*)q;
  return cudaMemsetAsync(q, 0, sizeof(T) * (size_t)n, h->st) == cudaSuccess ? SG_OK : SG_ECUDA;
}

template <typename T>
static int upload(sg_handle h, T** p, const std::vector<T>& v) {
  RET(dalloc(h, p, (long long)v.size()));
  if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->st));
  return SG_OK;
}

// ---------------------------------------------------------------------------------------------
// Batched inner CG on a subdomain pattern (0 Dirichlet, 1 Neumann): x = K_pat^{-1} rhs for nb
// problems (R per subdomain, subdomains from s0).  rhs must vanish outside the pattern's free
// nodes; x is returned in ws.x.  Returns the iteration count in *its.
// ---------------------------------------------------------------------------------------------
static int inner_solve(sg_handle h, int pat, int nb, int R, int s0, const double* rhs, int* its) {
  const auto& pr = h->pr;
  auto& ws = h->ws;
  const long long len = (long long)pr.nl * pr.P;
  const long long n = len * nb;
  Op<double> op = h->op64_from(s0);
  const int mask = pat == 0 ? sgk::MASK_I : sgk::MASK_N;
  const double cm = h->am, ck = h->bk;
  const int L = pr.L;
  const int G = std::max(1, std::min(pr.P, 256 / std::max(L, 1)));
  dim3 lb(L, G), lg(nb, (pr.P + G - 1) / G);
  const size_t lsm = sizeof(double) * 2 * L * G;
  const long long pstride = (long long)L * L * L;
  const double* Sinv = h->lf[pat].Sinv + (size_t)s0 * pstride;
  const double* Bd = h->lf[pat].Bd + (size_t)s0 * L * L;
  const double* Bu = h->lf[pat].Bu + (size_t)s0 * L * L;
  cudaStream_t st = h->st;
  CK(cudaMemcpyAsync(ws.r, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(ws.x, 0, sizeof(double) * n, st));
  sgk::k_line_solve<double><<<lg, lb, lsm, st>>>(L, pr.nl, pr.P, R, pstride, Sinv, Bd, Bu, ws.r, ws.z, nullptr);
  sgk::dot<double>(nb, len, ws.r, ws.z, ws.r, ws.rz, ws.bb, st);
  CK(cudaMemsetAsync(ws.nactive, 0, sizeof(int), st));
  sgk::k_cg_init<<<nblk(nb), 256, 0, st>>>(nb, ws.bb, ws.active, ws.nactive);
  CK(cudaMemcpyAsync(ws.p, ws.z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  CKL();
  const double tol2 = h->inner_tol * h->inner_tol;
  int it = 0;
  while (it < h->inner_max) {
    sgk::apply<double>(op, nb, R, ws.p, ws.p, ws.q, nullptr, cm, ck, mask, st);
    sgk::dot<double>(nb, len, ws.p, ws.q, nullptr, ws.pq, nullptr, st);
    sgk::k_cg_xr<double><<<nblk(n), 256, 0, st>>>(len, nb, ws.rz, ws.pq, ws.active, ws.p, ws.q, ws.x, ws.r);
    sgk::dot<double>(nb, len, ws.r, ws.r, nullptr, ws.rr, nullptr, st);
    CK(cudaMemsetAsync(ws.nactive, 0, sizeof(int), st));
    sgk::k_cg_check<<<nblk(nb), 256, 0, st>>>(nb, ws.rr, ws.bb, tol2, ws.active, ws.nactive, ws.pq);
    ++it;
    CK(cudaMemcpyAsync(h->hint, ws.nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h->hint[0] == 0) break;
    sgk::k_line_solve<double><<<lg, lb, lsm, st>>>(L, pr.nl, pr.P, R, pstride, Sinv, Bd, Bu, ws.r, ws.z,
                                                   ws.active);
    sgk::dot<double>(nb, len, ws.r, ws.z, nullptr, ws.rz_new, nullptr, st);
    sgk::k_cg_p<double><<<nblk(n), 256, 0, st>>>(len, nb, ws.rz_new, ws.rz, ws.active, ws.z, ws.p);
    sgk::k_copy_scalars<<<nblk(nb), 256, 0, st>>>(nb, ws.rz_new, ws.rz, ws.active);
    CKL();
  }
  CKL();
  h->inner_iters += it;
  if (its) *its = it;
  return SG_OK;
}

static int ensure_ws(sg_handle h, int nb) {
  auto& ws = h->ws;
  if (ws.cap_nb >= nb) return SG_OK;
  const long long len = (long long)h->pr.nl * h->pr.P * nb;
  RET(dalloc(h, &ws.x, len)); RET(dalloc(h, &ws.r, len)); RET(dalloc(h, &ws.z, len));
  RET(dalloc(h, &ws.p, len)); RET(dalloc(h, &ws.q, len));
  RET(dalloc(h, &ws.rz, nb)); RET(dalloc(h, &ws.rz_new, nb)); RET(dalloc(h, &ws.pq, nb));
  RET(dalloc(h, &ws.rr, nb)); RET(dalloc(h, &ws.bb, nb));
  RET(dalloc(h, &ws.active, nb)); RET(dalloc(h, &ws.nactive, 1));
  ws.cap_nb = nb;
  return SG_OK;
}

// ---------------------------------------------------------------------------------------------
// Interface operators
// ---------------------------------------------------------------------------------------------
// q = S p = sum_s R_s^T (K_GG - K_GI K_II^{-1} K_IG) R_s p
static int schur_apply(sg_handle h, const double* p, double* q) {
  const auto& pr = h->pr;
  cudaStream_t st = h->st;
  const int nsub = pr.nsub, nl = pr.nl, P = pr.P;
  const long long n = h->nvec();
  Op<double> op = h->op64();
  sgk::k_gather<double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, p, h->wa, sgk::MASK_G, 0);
  sgk::apply<double>(op, nsub, 1, h->wa, h->wa, h->wb, nullptr, -h->am, -h->bk, sgk::MASK_I, st);
  RET(inner_solve(h, 0, nsub, 1, 0, h->wb, nullptr));
  sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->wa, 1.0, h->ws.x, h->wd);
  sgk::apply<double>(op, nsub, 1, h->wd, h->wd, h->wb, nullptr, h->am, h->bk, sgk::MASK_G, st);
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, h->Dw, h->wb, q, 0);
  CKL();
  return SG_OK;
}

// z = M_NNC^{-1} r (Eq. NNCP2)
static int precond_apply(sg_handle h, const double* r, double* z) {
  const auto& pr = h->pr;
  cudaStream_t st = h->st;
  const int nsub = pr.nsub, nl = pr.nl, P = pr.P;
  const long long n = h->nvec();
  Op<double> op = h->op64();
  // w_s = D_s R_s r restricted to remaining nodes (Neumann RHS) and to corners
  sgk::k_gather<double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, r, h->wa, sgk::MASK_R, 1);
  sgk::k_gather<double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, r, h->wc, sgk::MASK_C, 1);
  RET(inner_solve(h, 1, nsub, 1, 0, h->wa, nullptr));  // v = [y; t], t = S_rr^{-1} w_r
  const double* v = h->ws.x;
  if (pr.nC > 0) {
    // S_cr t = (K~ [y; t; 0])_c ;  d = sum_s B^T (w_c - S_cr t) ;  u_c = F_cc^{-1} d
    sgk::apply<double>(op, nsub, 1, v, v, h->wd, nullptr, h->am, h->bk, sgk::MASK_C, st);
    sgk::k_corner_rhs<<<nblk((long long)pr.nC * P), 256, 0, st>>>(pr.nC, P, h->cowners, h->wc, h->wd, h->dC);
    sgk::k_gemv<<<nblk((long long)h->nCd * 32), 256, 0, st>>>(h->nCd, h->Finv, h->dC, h->uC);
  }
  sgk::k_coarse_extend<<<nblk((long long)nsub * pr.nGam * P), 256, 0, st>>>(
      nsub, nl, P, pr.nGam, pr.max_corner, h->cls, h->cidx, h->gam_ln, h->n_gam, h->loc_corner,
      h->n_loc_corner, h->Phi, h->uC, v, h->wd);
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, h->Dw, h->wd, z, 1);
  CKL();
  return SG_OK;
}

static int gdot(sg_handle h, const double* x, const double* y, double* out) {
  sgk::dot<double>(1, h->nGd(), x, y, nullptr, h->scal, nullptr, h->st);
  CK(cudaMemcpyAsync(h->hscal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  *out = h->hscal[0];
  return SG_OK;
}

// PCG on S x = g (Hestenes-Stiefel), x holds the initial guess; stops at ||r||/||g|| <= tol.
static int outer_pcg(sg_handle h, int* its, double* rel_out) {
  cudaStream_t st = h->st;
  const long long n = h->nGd();
  double gg, rr, rz, pq, rzn;
  *its = 0;
  RET(gdot(h, h->gG, h->gG, &gg));
  if (!std::isfinite(gg)) return SG_ENUMERIC;
  if (gg == 0.0) {
    CK(cudaMemsetAsync(h->xG, 0, sizeof(double) * n, st));
    *rel_out = 0.0;
    return SG_OK;
  }
  const double gn = std::sqrt(gg);
  RET(schur_apply(h, h->xG, h->qG));
  sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->gG, -1.0, h->qG, h->rG);
  RET(gdot(h, h->rG, h->rG, &rr));
  double rel = std::sqrt(rr) / gn;
  if (rel <= h->tol) { *rel_out = rel; return SG_OK; }
  RET(precond_apply(h, h->rG, h->zG));
  CK(cudaMemcpyAsync(h->pG, h->zG, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  RET(gdot(h, h->rG, h->zG, &rz));
  int it = 0;
  while (it < h->max_iter) {
    RET(schur_apply(h, h->pG, h->qG));
    RET(gdot(h, h->pG, h->qG, &pq));
    if (!(pq > 0.0) || !std::isfinite(pq)) { *its = it; *rel_out = rel; return SG_ENUMERIC; }
    const double alpha = rz / pq;
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->xG, alpha, h->pG, h->xG);
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->rG, -alpha, h->qG, h->rG);
    ++it;
    RET(gdot(h, h->rG, h->rG, &rr));
    rel = std::sqrt(rr) / gn;
    if (!std::isfinite(rel)) { *its = it; *rel_out = rel; return SG_ENUMERIC; }
    if (rel <= h->tol) break;
    RET(precond_apply(h, h->rG, h->zG));
    RET(gdot(h, h->rG, h->zG, &rzn));
    const double beta = rzn / rz;
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->zG, beta, h->pG, h->pG);
    rz = rzn;
  }
  CKL();
  *its = it;
  *rel_out = rel;
  return rel <= h->tol ? SG_OK : SG_ENOTCONV;
}

// ---------------------------------------------------------------------------------------------
// Set-up pieces
// ---------------------------------------------------------------------------------------------
// Mean operator stencils and line factorisation for both patterns.
static int build_line_factors(sg_handle h) {
  const auto& pr = h->pr;
  const int L = pr.L, nl = pr.nl, nsub = pr.nsub, H = pr.H, PI = pr.PI;
  const double mh = pr.h * pr.h / 24.0;
  for (int pat = 0; pat < 2; ++pat) {
    std::vector<double> Dd((size_t)nsub * L * L, 0.0), Du((size_t)nsub * L * L, 0.0);
    std::vector<double> Bd((size_t)nsub * L * L, 0.0), Bu((size_t)nsub * L * L, 0.0);
    for (int s = 0; s < nsub; ++s) {
      auto freep = [&](int li, int lj) {
        if (li < 0 || lj < 0 || li > H || lj > H) return false;
        int c = pr.cls[(size_t)s * nl + lj * L + li];
        return pat == 0 ? c == sgh::INTERIOR : (c == sgh::INTERIOR || c == sgh::REMAINING);
      };
      auto cellp = [&](int ci, int cj) { return ci >= 0 && cj >= 0 && ci < H && cj < H; };
      auto kapE0 = [&](int li, int lj) { return pr.kapE[((size_t)s * nl + lj * L + li) * PI]; };
      auto kapN0 = [&](int li, int lj) { return pr.kapN[((size_t)s * nl + lj * L + li) * PI]; };
      for (int lj = 0; lj <= H; ++lj)
        for (int li = 0; li <= H; ++li) {
          const size_t o = (size_t)s * L * L + (size_t)lj * L + li;
          if (!freep(li, lj)) { Dd[o] = 1.0; continue; }
          // mass: 2 h^2/24 per triangle containing the node on the diagonal, h^2/24 per shared
          // triangle off the diagonal; stiffness: graph Laplacian of the mode-0 edge weights
          int ntri = 2 * cellp(li - 1, lj - 1) + cellp(li, lj - 1) + cellp(li - 1, lj) + 2 * cellp(li, lj);
          double kd = 0.0;
          if (li < H) kd += kapE0(li, lj);
          if (li > 0) kd += kapE0(li - 1, lj);
          if (lj < H) kd += kapN0(li, lj);
          if (lj > 0) kd += kapN0(li, lj - 1);
          Dd[o] = h->am * mh * 2.0 * ntri + h->bk * kd;
          if (freep(li + 1, lj)) {
            double m = mh * (cellp(li, lj - 1) + cellp(li, lj));
            Du[o] = h->am * m - h->bk * kapE0(li, lj);
          }
          if (freep(li, lj + 1)) {
            double m = mh * (cellp(li - 1, lj) + cellp(li, lj));
            Bd[o] = h->am * m - h->bk * kapN0(li, lj);
          }
          if (freep(li + 1, lj + 1)) Bu[o] = h->am * mh * 2.0 * cellp(li, lj);
        }
    }
    double *dDd, *dDu;
    RET(upload(h, &dDd, Dd)); RET(upload(h, &dDu, Du));
    RET(upload(h, &h->lf[pat].Bd, Bd)); RET(upload(h, &h->lf[pat].Bu, Bu));
    RET(dalloc(h, &h->lf[pat].Sinv, (long long)nsub * L * L * L));
    int* dstat;
    RET(dalloc(h, &dstat, nsub));
    const size_t sm = sizeof(double) * ((size_t)L * L + 2 * L);
    if (sm > 48 * 1024) CK(cudaFuncSetAttribute(sgk::k_line_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    sgk::k_line_factor<<<nsub, 256, sm, h->st>>>(L, dDd, dDu, h->lf[pat].Bd, h->lf[pat].Bu, h->lf[pat].Sinv, dstat);
    CKL();
    std::vector<int> stat(nsub);
    CK(cudaMemcpyAsync(stat.data(), dstat, sizeof(int) * nsub, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int s = 0; s < nsub; ++s)
      if (stat[s]) { h->err = "mean operator not positive definite"; return SG_ENUMERIC; }
  }
  return SG_OK;
}

// Host inverse of a small SPD matrix by Cholesky (set-up only).
static bool spd_inverse(std::vector<double>& A, int n) {
  std::vector<double> Lm((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= Lm[(size_t)j * n + k] * Lm[(size_t)j * n + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    Lm[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= Lm[(size_t)i * n + k] * Lm[(size_t)j * n + k];
      Lm[(size_t)i * n + j] = s / d;
    }
  }
  // inverse = L^{-T} L^{-1}
  std::vector<double> Li((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    for (int i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= Lm[(size_t)i * n + k] * Li[(size_t)k * n + c];
      Li[(size_t)i * n + c] = s / Lm[(size_t)i * n + i];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int k = i; k < n; ++k) s += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
      A[(size_t)i * n + j] = s;
      A[(size_t)j * n + i] = s;
    }
  return true;
}

// Coarse basis Phi_s = -S_rr^{-1} S_rc (per local corner dof) and F_cc (Eq. Fcc_2), from one
// Neumann solve per local corner dof: v = -N^{-1} K_[ir],c e, F^s e = (K~ (v + e))_c.
static int build_coarse(sg_handle h) {
  const auto& pr = h->pr;
  const int P = pr.P, nl = pr.nl, nsub = pr.nsub;
  h->Rc = pr.max_corner * P;
  h->nCd = pr.nC * P;
  const int R = h->Rc;
  RET(dalloc(h, &h->Phi, (long long)nsub * std::max(R, 1) * pr.nGam * P));
  RET(dalloc(h, &h->dC, std::max(h->nCd, 1)));
  RET(dalloc(h, &h->uC, std::max(h->nCd, 1)));
  if (pr.nC == 0 || R == 0) return SG_OK;
  // chunk subdomains so that the batched solve holds at most ~2048 problems
  const int chunk = std::max(1, std::min(nsub, 2048 / R));
  const long long len = (long long)nl * P;
  RET(ensure_ws(h, chunk * R));
  double *e, *rhs, *ve, *y, *Fs;
  RET(dalloc(h, &e, len * chunk * R));
  RET(dalloc(h, &rhs, len * chunk * R));
  RET(dalloc(h, &ve, len * chunk * R));
  RET(dalloc(h, &y, len * chunk * R));
  RET(dalloc(h, &Fs, (long long)nsub * R * R));
  cudaStream_t st = h->st;
  for (int s0 = 0; s0 < nsub; s0 += chunk) {
    const int ns = std::min(chunk, nsub - s0);
    const int nb = ns * R;
    const long long n = len * nb;
    Op<double> op = h->op64_from(s0);
    CK(cudaMemsetAsync(e, 0, sizeof(double) * n, st));
    sgk::k_coarse_units<<<nblk((long long)nb), 256, 0, st>>>(ns, R, nl, P, s0, h->loc_corner, h->n_loc_corner, e);
    sgk::apply<double>(op, nb, R, e, e, rhs, nullptr, -h->am, -h->bk, sgk::MASK_N, st);
    RET(inner_solve(h, 1, nb, R, s0, rhs, nullptr));
    sgk::k_coarse_phi<<<nblk((long long)nb * pr.nGam * P), 256, 0, st>>>(ns, s0, R, nl, P, pr.nGam, h->cls,
                                                                         h->gam_ln, h->n_gam, h->ws.x, h->Phi);
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->ws.x, 1.0, e, ve);
    sgk::apply<double>(op, nb, R, ve, ve, y, nullptr, h->am, h->bk, sgk::MASK_C, st);
    sgk::k_coarse_fs<<<nblk((long long)nb * R), 256, 0, st>>>(ns, s0, R, nl, P, h->loc_corner, h->n_loc_corner, y, Fs);
    CKL();
  }
  std::vector<double> hFs((size_t)nsub * R * R);
  CK(cudaMemcpyAsync(hFs.data(), Fs, sizeof(double) * hFs.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int nCd = h->nCd;
  std::vector<double> F((size_t)nCd * nCd, 0.0);
  for (int s = 0; s < nsub; ++s) {
    const int nc = pr.n_loc_corner[s];
    for (int a = 0; a < nc; ++a) {
      const int ga = pr.cidx[(size_t)s * nl + pr.loc_corner[s * 4 + a]];
      for (int b = 0; b < nc; ++b) {
        const int gb = pr.cidx[(size_t)s * nl + pr.loc_corner[s * 4 + b]];
        for (int m = 0; m < P; ++m)
          for (int q = 0; q < P; ++q)
            F[(size_t)(ga * P + m) * nCd + gb * P + q] += hFs[((size_t)s * R + a * P + m) * R + b * P + q];
      }
    }
  }
  // symmetrise (the two triangles agree to rounding) and invert
  for (int i = 0; i < nCd; ++i)
    for (int j = 0; j < i; ++j) {
      double v = 0.5 * (F[(size_t)i * nCd + j] + F[(size_t)j * nCd + i]);
      F[(size_t)i * nCd + j] = F[(size_t)j * nCd + i] = v;
    }
  if (!spd_inverse(F, nCd)) { h->err = "coarse matrix F_cc not positive definite"; return SG_ENUMERIC; }
  RET(upload(h, &h->Finv, F));
  return SG_OK;
}

static int ldot_w(sg_handle h, const double* x, const double* y, double* out) {
  sgk::k_dot_w<<<1, 1024, 0, h->st>>>(h->nloc(), h->pr.P, h->nodew, x, y, h->scal);
  CK(cudaMemcpyAsync(h->hscal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  *out = h->hscal[0];
  return SG_OK;
}

// Initial state: U0 (pulse, mode 0), V0 = 0, consistent A0 from (M (x) I) A0 = F(0) - K U0,
// solved by CG on the globally assembled mass matrix in the local layout.
static int initial_state(sg_handle h) {
  const auto& pr = h->pr;
  cudaStream_t st = h->st;
  const long long n = h->nvec();
  const int P = pr.P;
  Op<double> op = h->op64();
  {
    std::vector<double> U0((size_t)n, 0.0);
    for (long long i = 0; i < h->nloc(); ++i) U0[(size_t)i * P] = pr.u0_local[(size_t)i];
    CK(cudaMemcpyAsync(h->U, U0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemsetAsync(h->V, 0, sizeof(double) * n, st));
  // rhs = F(0) - K U0 (local), assembled on the interface
  sgk::apply<double>(op, pr.nsub, 1, h->U, h->U, h->wa, nullptr, 0.0, -1.0, sgk::MASK_FREE, st);
  if (h->nload)
    sgk::k_point_load<<<nblk(h->nload), 256, 0, st>>>(h->nload, h->load_node, h->load_w, 0.0, pr.src.freq, P, h->wa);
  sgk::k_assemble_gamma<<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, h->wa);
  // CG on the assembled mass: x = A, r = wa, p = wb, q = wc
  CK(cudaMemsetAsync(h->A, 0, sizeof(double) * n, st));
  double rr, rr0, pq;
  RET(ldot_w(h, h->wa, h->wa, &rr));
  rr0 = rr;
  CK(cudaMemcpyAsync(h->wb, h->wa, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  for (int it = 0; it < 500 && rr > 1e-30 * rr0 && rr0 > 0.0; ++it) {
    sgk::apply<double>(op, pr.nsub, 1, h->wb, h->wb, h->wc, nullptr, 1.0, 0.0, sgk::MASK_FREE, st);
    sgk::k_assemble_gamma<<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, h->wc);
    RET(ldot_w(h, h->wb, h->wc, &pq));
    const double a = rr / pq;
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->A, a, h->wb, h->A);
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->wa, -a, h->wc, h->wa);
    double rn;
    RET(ldot_w(h, h->wa, h->wa, &rn));
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->wa, rn / rr, h->wb, h->wb);
    rr = rn;
  }
  CKL();
  // PCG warm start: interface restriction of U0
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, h->Dw, h->U, h->xG, 1);
  CKL();
  return SG_OK;
}

// ---------------------------------------------------------------------------------------------
// One time step
// ---------------------------------------------------------------------------------------------
static int do_step(sg_handle h, const double* fext_dev, int* its_out, double* rel_out) {
  const auto& pr = h->pr;
  cudaStream_t st = h->st;
  const long long n = h->nvec();
  const int nsub = pr.nsub, nl = pr.nl, P = pr.P;
  const double dt = pr.dt;
  const double t = (double)(h->step + 1) * dt;
  Op<double> op = h->op64();
  // a1: effective load f~ = M (u~_m + alpha0 u~_c) + alpha1 K u~_c + f
  sgk::k_newmark_pre<<<nblk(n), 256, 0, st>>>(n, dt, pr.alpha0, h->U, h->V, h->A, h->um, h->uc, h->xm);
  sgk::apply<double>(op, nsub, 1, h->xm, h->uc, h->ft, nullptr, 1.0, pr.alpha1, sgk::MASK_FREE, st);
  if (h->nload)
    sgk::k_point_load<<<nblk(h->nload), 256, 0, st>>>(h->nload, h->load_node, h->load_w, t, pr.src.freq, P, h->ft);
  if (fext_dev)
    sgk::k_ext_load<<<nblk(h->nloc()), 256, 0, st>>>(h->nloc(), P, h->free_of_local, h->cls, h->gidx, h->Dw,
                                                      fext_dev, h->ft);
  // a2: condensed RHS
  sgk::k_mask<double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->ft, h->wa, sgk::MASK_I);
  RET(inner_solve(h, 0, nsub, 1, 0, h->wa, nullptr));
  sgk::apply<double>(op, nsub, 1, h->ws.x, h->ws.x, h->wc, h->ft, -h->am, -h->bk, sgk::MASK_G, st);
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, h->Dw, h->wc, h->gG, 0);
  CKL();
  // a3-a5: PCG on the interface, warm-started from the previous solution in xG
  int its = 0;
  double rel = 0.0;
  int rc = outer_pcg(h, &its, &rel);
  if (rc != SG_OK && rc != SG_ENOTCONV) return rc;
  // a6: interior recovery
  sgk::k_gather<double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, h->xG, h->wa, sgk::MASK_G, 0);
  sgk::apply<double>(op, nsub, 1, h->wa, h->wa, h->wb, h->ft, -h->am, -h->bk, sgk::MASK_I, st);
  RET(inner_solve(h, 0, nsub, 1, 0, h->wb, nullptr));
  sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->ws.x, 1.0, h->wa, h->Unew);
  // a7: Newmark update
  sgk::k_newmark_post<<<nblk(n), 256, 0, st>>>(n, dt, h->Unew, h->um, h->U, h->V, h->A);
  CKL();
  h->step += 1;
  *its_out = its;
  *rel_out = rel;
  return rc;
}

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
static void free_all(sg_handle h) {
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->hscal) cudaFreeHost(h->hscal);
  if (h->hint) cudaFreeHost(h->hint);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
}

static int setup_impl(sg_handle h, const sg_grid* grid, const sg_kl* kl, const sg_pce* pce,
                      const sg_params* prm, const sg_source* src) {
  sgh::SourceDesc sd{src ? src->kind : 0, src ? src->x0 : 0.5, src ? src->y0 : 0.5,
                     src ? src->width : 0.05, src ? src->freq : 10.0, src ? src->amp : 1.0};
  if (sd.kind < 0 || sd.kind > 2) { h->err = "source kind"; return SG_EINVAL; }
  if (sd.kind == 1 && !(sd.width > 0)) { h->err = "pulse width must be positive"; return SG_EINVAL; }
  if (sd.kind == 2 && (!(sd.freq > 0) || sd.x0 < 0 || sd.x0 > 1 || sd.y0 < 0 || sd.y0 > 1)) {
    h->err = "ricker source outside the unit square or non-positive frequency";
    return SG_EINVAL;
  }
  std::string msg = sgh::build_problem(h->pr, grid->N, grid->nsub_x, grid->nsub_y, kl->M, kl->sigma, kl->bx,
                                       kl->by, kl->g0, pce->p, pce->p_in, prm->dt, prm->alpha0, prm->alpha1, sd);
  if (!msg.empty()) { h->err = msg; return SG_EINVAL; }
  auto& pr = h->pr;
  if (pr.L > 256) { h->err = "subdomains wider than 255 cells are not supported"; return SG_ENOTSUP; }
  h->precision = prm->precision;
  h->warm = prm->warm;
  h->tol = prm->tol > 0 ? prm->tol : 1e-8;
  h->max_iter = prm->max_iter > 0 ? prm->max_iter : 500;
  h->inner_tol = prm->inner_tol > 0 ? prm->inner_tol : 1e-14;
  h->inner_max = prm->inner_max_iter > 0 ? prm->inner_max_iter : 400;
  h->am = 1.0 / (ZETA * pr.dt * pr.dt) + pr.alpha0 * GAMMA / (ZETA * pr.dt);
  h->bk = 1.0 + pr.alpha1 * GAMMA / (ZETA * pr.dt);
  CK(cudaMallocHost(&h->hscal, sizeof(double) * 16));
  CK(cudaMallocHost(&h->hint, sizeof(int) * 16));
  CK(cudaEventCreate(&h->ev0));
  CK(cudaEventCreate(&h->ev1));
  // problem data
  RET(upload(h, &h->cls, pr.cls)); RET(upload(h, &h->cells, pr.cells));
  RET(upload(h, &h->kapE, pr.kapE)); RET(upload(h, &h->kapN, pr.kapN));
  RET(upload(h, &h->gk_ptr, pr.gk_ptr)); RET(upload(h, &h->gk_i, pr.gk_i)); RET(upload(h, &h->gk_j, pr.gk_j));
  RET(upload(h, &h->gk_v, pr.gk_v));
  RET(upload(h, &h->gidx, pr.gidx)); RET(upload(h, &h->cidx, pr.cidx));
  RET(upload(h, &h->owners, pr.owners)); RET(upload(h, &h->cowners, pr.cowners));
  RET(upload(h, &h->Dw, pr.Dw)); RET(upload(h, &h->gam_ln, pr.gam_ln)); RET(upload(h, &h->n_gam, pr.n_gam));
  RET(upload(h, &h->loc_corner, pr.loc_corner)); RET(upload(h, &h->n_loc_corner, pr.n_loc_corner));
  RET(upload(h, &h->free_owner, pr.free_owner)); RET(upload(h, &h->free_of_local, pr.free_of_local));
  RET(upload(h, &h->load_node, pr.load_node)); RET(upload(h, &h->load_w, pr.load_w));
  h->nload = (int)pr.load_node.size();
  RET(dalloc(h, &h->nodew, h->nloc()));
  sgk::k_node_weight<<<nblk(h->nloc()), 256, 0, h->st>>>((int)h->nloc(), h->cls, h->gidx, h->Dw, h->nodew);
  // state and work vectors
  const long long n = h->nvec();
  for (double** p : {&h->U, &h->V, &h->A, &h->um, &h->uc, &h->xm, &h->ft, &h->Unew, &h->wa, &h->wb, &h->wc, &h->wd})
    RET(dalloc(h, p, n));
  RET(dalloc(h, &h->fext, pr.n_free));
  RET(dalloc(h, &h->outbuf, (long long)pr.n_free * pr.P));
  for (double** p : {&h->xG, &h->rG, &h->zG, &h->pG, &h->qG, &h->gG}) RET(dalloc(h, p, h->nGd()));
  RET(dalloc(h, &h->scal, 16));
  RET(ensure_ws(h, pr.nsub));
  CKL();
  RET(build_line_factors(h));
  RET(build_coarse(h));
  RET(initial_state(h));
  CK(cudaStreamSynchronize(h->st));
  return SG_OK;
}

extern "C" {

int sg_setup(const sg_grid* grid, const sg_kl* kl, const sg_pce* pce, const sg_params* params,
             const sg_source* src, void* stream, sg_handle* out) {
  if (!out) return SG_EINVAL;
  *out = nullptr;
  if (!grid || !kl || !pce || !params) { g_setup_err = "null argument"; return SG_EINVAL; }
  sg_handle h = new (std::nothrow) sg_handle_s();
  if (!h) return SG_ENOMEM;
  h->st = (cudaStream_t)stream;
  int rc = setup_impl(h, grid, kl, pce, params, src);
  if (rc != SG_OK) {
    g_setup_err = h->err;
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return SG_OK;
}

int sg_step(sg_handle h, int nsteps, sg_stats* stats) {
  if (!h || nsteps < 0) return SG_EINVAL;
  h->iters.clear();
  h->relres.clear();
  const long long inner0 = h->inner_iters;
  CK(cudaEventRecord(h->ev0, h->st));
  int rc = SG_OK;
  long long tot = 0;
  int its = 0;
  double rel = 0.0;
  for (int s = 0; s < nsteps; ++s) {
    int r = do_step(h, nullptr, &its, &rel);
    h->iters.push_back(its);
    h->relres.push_back(rel);
    tot += its;
    if (r == SG_ENOTCONV) rc = SG_ENOTCONV;
    else if (r != SG_OK) return r;
  }
  CK(cudaEventRecord(h->ev1, h->st));
  CK(cudaEventSynchronize(h->ev1));
  if (stats) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    stats->steps = nsteps;
    stats->step_index = (int)h->step;
    stats->iters_last = its;
    stats->iters_total = tot;
    stats->inner_total = h->inner_iters - inner0;
    stats->relres_last = rel;
    stats->ms = ms;
  }
  return rc;
}

int sg_solve_batch(sg_handle* hs, int n, int nsteps, sg_stats* out_n) {
  if (!hs || n < 0) return SG_EINVAL;
  int rc = SG_OK;
  for (int i = 0; i < n; ++i) {
    int r = sg_step(hs[i], nsteps, out_n ? &out_n[i] : nullptr);
    if (r == SG_ENOTCONV) rc = r;
    else if (r != SG_OK) return r;
  }
  return rc;
}

int sg_get_field(sg_handle h, int mode, double* dst, int on_device) {
  if (!h || !dst || mode < -1 || mode >= h->pr.P) return SG_EINVAL;
  const auto& pr = h->pr;
  const long long cnt = mode < 0 ? (long long)pr.n_free * pr.P : pr.n_free;
  double* d = on_device ? dst : h->outbuf;
  sgk::k_gather_free<<<nblk(cnt), 256, 0, h->st>>>(pr.n_free, pr.P, mode, h->free_owner, h->U, d);
  CKL();
  if (!on_device) CK(cudaMemcpyAsync(dst, h->outbuf, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return SG_OK;
}

int sg_get_moments(sg_handle h, double* mean, double* var, int on_device) {
  if (!h) return SG_EINVAL;
  const auto& pr = h->pr;
  double* dm = on_device ? mean : (mean ? h->outbuf : nullptr);
  double* dv = on_device ? var : (var ? h->outbuf + pr.n_free : nullptr);
  sgk::k_moments<<<nblk(pr.n_free), 256, 0, h->st>>>(pr.n_free, pr.P, h->free_owner, h->U, dm, dv);
  CKL();
  if (!on_device) {
    if (mean) CK(cudaMemcpyAsync(mean, dm, sizeof(double) * pr.n_free, cudaMemcpyDeviceToHost, h->st));
    if (var) CK(cudaMemcpyAsync(var, dv, sizeof(double) * pr.n_free, cudaMemcpyDeviceToHost, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  return SG_OK;
}

int sg_get_state(sg_handle h, double* dst, int on_device) {
  if (!h || !dst) return SG_EINVAL;
  const auto& pr = h->pr;
  const long long cnt = (long long)pr.n_free * pr.P;
  const double* src[3] = {h->U, h->V, h->A};
  for (int q = 0; q < 3; ++q) {
    sgk::k_gather_free<<<nblk(cnt), 256, 0, h->st>>>(pr.n_free, pr.P, -1, h->free_owner, src[q], h->outbuf);
    CKL();
    CK(cudaMemcpyAsync(dst + q * cnt, h->outbuf, sizeof(double) * cnt,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  double stepd = (double)h->step;
  CK(cudaMemcpy(dst + 3 * cnt, &stepd, sizeof(double), on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
  return SG_OK;
}

int sg_set_state(sg_handle h, const double* src, int on_device) {
  if (!h || !src) return SG_EINVAL;
  const auto& pr = h->pr;
  const long long cnt = (long long)pr.n_free * pr.P;
  double* dst[3] = {h->U, h->V, h->A};
  for (int q = 0; q < 3; ++q) {
    CK(cudaMemcpyAsync(h->outbuf, src + q * cnt, sizeof(double) * cnt,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    sgk::k_scatter_free<<<nblk(h->nvec()), 256, 0, h->st>>>(h->nloc(), pr.P, h->free_of_local, h->outbuf, dst[q]);
    CKL();
  }
  double stepd = 0.0;
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemcpy(&stepd, src + 3 * cnt, sizeof(double), on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  if (!(stepd >= 0) || stepd != std::floor(stepd)) return SG_EINVAL;
  h->step = (long long)stepd;
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, h->st>>>(pr.nG, pr.P, h->owners, h->Dw, h->U, h->xG, 1);
  CKL();
  CK(cudaStreamSynchronize(h->st));
  return SG_OK;
}

int sg_step_host(sg_handle h, int nsteps, const double* f_host, double* u_host, sg_stats* stats) {
  if (!h || nsteps < 0) return SG_EINVAL;
  const auto& pr = h->pr;
  h->iters.clear();
  h->relres.clear();
  const long long inner0 = h->inner_iters;
  CK(cudaEventRecord(h->ev0, h->st));
  int rc = SG_OK, its = 0;
  long long tot = 0;
  double rel = 0.0;
  for (int s = 0; s < nsteps; ++s) {
    if (f_host)
      CK(cudaMemcpyAsync(h->fext, f_host + (size_t)s * pr.n_free, sizeof(double) * pr.n_free,
                         cudaMemcpyHostToDevice, h->st));
    int r = do_step(h, f_host ? h->fext : nullptr, &its, &rel);
    if (r == SG_ENOTCONV) rc = r;
    else if (r != SG_OK) return r;
    h->iters.push_back(its);
    h->relres.push_back(rel);
    tot += its;
    if (u_host) {
      sgk::k_gather_free<<<nblk(pr.n_free), 256, 0, h->st>>>(pr.n_free, pr.P, 0, h->free_owner, h->U, h->outbuf);
      CKL();
      CK(cudaMemcpyAsync(u_host + (size_t)s * pr.n_free, h->outbuf, sizeof(double) * pr.n_free,
                         cudaMemcpyDeviceToHost, h->st));
    }
  }
  CK(cudaEventRecord(h->ev1, h->st));
  CK(cudaEventSynchronize(h->ev1));
  if (stats) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    stats->steps = nsteps;
    stats->step_index = (int)h->step;
    stats->iters_last = its;
    stats->iters_total = tot;
    stats->inner_total = h->inner_iters - inner0;
    stats->relres_last = rel;
    stats->ms = ms;
  }
  return rc;
}

int sg_get_sizes(sg_handle h, sg_sizes* out) {
  if (!h || !out) return SG_EINVAL;
  const auto& pr = h->pr;
  out->N = pr.N; out->nsub = pr.nsub; out->P = pr.P; out->P_in = pr.PI; out->n_free = pr.n_free;
  out->n_gamma = pr.nG; out->n_corner = pr.nC; out->n_sub_nodes = pr.nl; out->device_bytes = h->bytes;
  return SG_OK;
}

int sg_get_iters(sg_handle h, int* iters, double* relres, int cap) {
  if (!h || cap < 0) return SG_EINVAL;
  int n = std::min(cap, (int)h->iters.size());
  for (int i = 0; i < n; ++i) {
    if (iters) iters[i] = h->iters[i];
    if (relres) relres[i] = h->relres[i];
  }
  return n;
}

int sg_destroy(sg_handle h) {
  if (!h) return SG_EINVAL;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return SG_OK;
}

const char* sg_strerror(int code) {
  switch (code) {
    case SG_OK: return "ok";
    case SG_EINVAL: return "invalid argument";
    case SG_ENOMEM: return "out of memory";
    case SG_ECUDA: return "CUDA error";
    case SG_ENOTCONV: return "PCG did not converge within max_iter";
    case SG_ENUMERIC: return "numerical breakdown (NaN/Inf or non-SPD)";
    case SG_ETIMEOUT: return "device wait timed out";
    case SG_ENOTSUP: return "unsupported configuration";
    default: return "unknown error";
  }
}

const char* sg_last_error(sg_handle h) { return h ? h->err.c_str() : g_setup_err.c_str(); }

}  // extern "C"
