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
// factorisation).  In FP64 mode every kernel computes in FP64 and the subdomain CG runs to a
// tight relative residual.  In mixed mode the subdomain CG runs in FP32; each Dirichlet solve
// inside the interface operator gets one FP64 residual correction, so the Schur matvec keeps
// FP64-level accuracy while the outer PCG (flexible beta), its dot products, residual
// recurrence and the coarse solve stay FP64.
//
// The whole step is one CUDA graph: the inner and outer loops are conditional WHILE nodes whose
// conditions are set on the device, so a step needs no host synchronisation.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/sg.h"
#include "sg_host.hpp"
#include "sg_kernels.cuh"
#include "sg_mesh.cuh"

using sgk::CgCtl;
using sgk::Op;
using sgk::OuterCtl;

namespace {

constexpr double ZETA = 0.25, GAMMA = 0.5;
constexpr int NB_OUT = 128;     // blocks of the outer vector kernels (= partial count)
constexpr int NSTREAMS = 6;     // capture depth of nested conditional bodies
constexpr int REC_CAP = 1 << 14;

template <typename T>
struct InnerWS {
  T *x = nullptr, *r = nullptr, *z = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
  int cap_nb = 0;
};

template <typename T>
struct LineFactor {
  T* Sinv = nullptr;  // [sub][L][L][L]
  T* Bd = nullptr;    // [sub][L][L]
  T* Bu = nullptr;
  T* Spad = nullptr;  // [sub][L][L][LS] rows zero-padded to a multiple of 4 (FP32 staged kernel)
};

struct Ctx {
  cudaStream_t st;
  int depth;
  bool capture;
};

}  // namespace

struct sg_handle_s {
  sgh::Problem pr;
  cudaStream_t st = nullptr;          // caller's stream (graph launches, copies)
  int dev = -1;                       // CUDA device current at sg_setup (the handle's memory lives there)
  bool own_st = false;
  cudaStream_t cs[NSTREAMS] = {};     // private capture streams
  std::string err;
  int precision = SG_FP64, warm = SG_WARM_PREV;
  int policy = SG_FP64;               // sg_params.precision as given (SG_FP32 / SG_BF16 select the preconditioner)
  double tol = 1e-8, inner_tol = 1e-14, inner_tol32 = 1e-6, prec_tol32 = 1e-3;
  int max_iter = 500, inner_max = 400;
  double am = 0, bk = 0;
  long long step = 0;
  bool eager = false;
  // device problem data
  uint8_t *cls = nullptr, *cells = nullptr;
  double *kapE = nullptr, *kapN = nullptr, *gk_v = nullptr;
  float *kapE32 = nullptr, *kapN32 = nullptr, *gk_v32 = nullptr;
  // float-float copies of the edge weights (hi, lo) for the float-float outer applies (apply_f2)
  float2 *kapE2 = nullptr, *kapN2 = nullptr;
  bool apply_f2 = false;
  int *gk_ptr = nullptr, *gk_i = nullptr, *gk_j = nullptr;
  unsigned* gk_pk = nullptr;  // gk_i | gk_j << 16
  int *gidx = nullptr, *cidx = nullptr, *owners = nullptr, *cowners = nullptr, *gam_ln = nullptr;
  int *n_gam = nullptr, *loc_corner = nullptr, *n_loc_corner = nullptr, *free_owner = nullptr;
  int *free_of_local = nullptr;
  double *Dw = nullptr, *nodew = nullptr;
  int* load_node = nullptr;
  double* load_w = nullptr;
  int nload = 0;
  // 0: Dirichlet (interior free), 1: Neumann (interior + remaining free), 2: all local free nodes
  // (one-level Neumann-Neumann preconditioner only)
  LineFactor<double> lf[3];
  LineFactor<float> lf32[3];
  int pc = SG_PC_NN2;                 // interface preconditioner
  // tensor-core mean preconditioner of the FP32 inner solves (mixed precision, small subdomains)
  bool mma = false;
  bool pdl = false;                // programmatic dependent launch inside the inner loop (opt-in)
  int mma_nb = 32;                 // N of the product: PCE modes padded to 16 or 32
  int Kp = 0, NC = 0, MT = 0;      // padded local node count, 64-node chunks, 128-row tiles
  // tensor-core line sweeps of the FP32 solves (k_line_tc): BF16 factor images of patterns 0 and 1,
  // their FP32 65th columns and TMA maps
  bool line_tc = false;
  __nv_bfloat16* limg[2] = {nullptr, nullptr};
  float* lcol[2] = {nullptr, nullptr};
  CUtensorMap tmL[2];
  __nv_bfloat16* ainv = nullptr;   // [pattern][subdomain][Kp][Kp] BF16 copy of A0^{-1}
  unsigned char* bimg = nullptr;   // [problem][chunk][hi, lo][NB x 64 swizzled] residual image
  int bimg_cap = 0;
  CUtensorMap tmA;                 // TMA map over ainv (64 x 128 boxes, 128-byte swizzle)
  // coarse space
  double *Phi = nullptr, *Finv = nullptr;
  int nCd = 0, Rc = 0;
  // state and step work (local layout)
  double *U = nullptr, *V = nullptr, *A = nullptr, *um = nullptr, *uc = nullptr, *xm = nullptr;
  double *ft = nullptr, *Unew = nullptr, *wa = nullptr, *wb = nullptr, *wc = nullptr, *wd = nullptr, *we = nullptr;
  float *fa = nullptr, *fb = nullptr;
  // mixed precision: interior solution accumulated from the Schur matvecs, W_I = K_II^{-1} f~_I +
  // sum of the PCG steps' Dirichlet extensions (replaces the two interior-recovery solves)
  double* Wrec = nullptr;
  bool a6_rec = false;
  double* fext = nullptr;  // n_free
  double* outbuf = nullptr;
  // surrogate sampling: multi-indices of the solution basis, staging of host inputs / outputs
  signed char* alpha_d = nullptr;
  double *samp_xi = nullptr, *samp_psi = nullptr, *samp_out = nullptr;
  int* samp_nodes = nullptr;
  long long samp_cap_s = 0, samp_cap_p = 0, samp_cap_out = 0;
  // interface vectors and outer control
  double *xG = nullptr, *rG = nullptr, *zG = nullptr, *pG = nullptr, *qG = nullptr, *gG = nullptr, *roG = nullptr;
  double *dC = nullptr, *uC = nullptr, *opart = nullptr, *opart2 = nullptr, *scal = nullptr;
  OuterCtl* octl = nullptr;
  int* omirror = nullptr;
  // inner CG control (shared by both precisions; solves are sequential)
  CgCtl ctl{};
  int ctl_cap_nb = 0, ctl_cap_nt = 0, ctl_cap_ng = 0;
  InnerWS<double> ws;
  InnerWS<float> ws32;
  // per-step records
  long long* stepctr = nullptr;
  int* rec_iters = nullptr;
  double* rec_rel = nullptr;
  int* rec_flags = nullptr;
  unsigned long long* nlaunch = nullptr;
  // graphs
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // [0] built-in load only, [1] + external load
  cudaGraph_t graph[2] = {nullptr, nullptr};
  double* hscal = nullptr;  // pinned host scalars
  int* hint = nullptr;      // pinned host ints
  std::vector<void*> allocs;
  long long bytes = 0;
  std::vector<int> iters;
  std::vector<double> relres;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // learned warm start
  sgk::WarmCtl wctl{};
  // learned warm start: predictor-error history (4 steps), interface velocity and acceleration,
  // predictor and feature scale per row
  double *wE0 = nullptr, *wE1 = nullptr, *wE2 = nullptr, *wE3 = nullptr, *vG = nullptr, *aG = nullptr;
  double *wpred = nullptr, *wscale = nullptr;
  float *wX = nullptr, *wy = nullptr, *wt = nullptr;
  int warm_train = 20, warm_epochs = 4;
  float warm_lr = 1e-3f;
  // general partitions of unstructured meshes (sg_setup_mesh): sparse rows of the local layout (FP64
  // and FP32 values), rows per pattern and subdomain, and the dense inverses of the subdomains' mean
  // operators per pattern (0 Dirichlet, 1 Neumann, 2 every free vertex) in the subdomain-solve type
  bool mesh = false;
  int *m_rp = nullptr, *m_col = nullptr, *m_npat = nullptr;
  double *m_kv = nullptr, *m_mv = nullptr;
  float *m_kv32 = nullptr, *m_mv32 = nullptr;
  double* m_ainv[3] = {nullptr, nullptr, nullptr};
  float* m_ainv32[3] = {nullptr, nullptr, nullptr};
  // per-kernel timing (host-driven enqueue only): 0 off, 1 line kernel, 2 fused apply kernel
  int kprof = 0;
  double kprof_ms = 0.0;
  long long kprof_n = 0;
  cudaEvent_t kev0 = nullptr, kev1 = nullptr;

  template <typename T>
  Op<T> op(int s0 = 0) const {
    Op<T> o;
    if (mesh) {  // the mesh apply reads the sparse rows; the Op only carries the first subdomain
      o.cls = cls + (size_t)s0 * pr.nl;
      o.nl = pr.nl; o.P = pr.P; o.PI = pr.PI;
      return o;
    }
    o.cls = cls + (size_t)s0 * pr.nl;
    o.cells = cells + (size_t)s0 * pr.nl;
    if constexpr (sizeof(T) == 8) {
      o.kapE = (const T*)kapE; o.kapN = (const T*)kapN; o.gk_v = (const T*)gk_v;
    } else {
      o.kapE = (const T*)kapE32; o.kapN = (const T*)kapN32; o.gk_v = (const T*)gk_v32;
    }

    o.kapE += (size_t)s0 * pr.nl * pr.PI;
    o.kapN += (size_t)s0 * pr.nl * pr.PI;
    o.gk_ptr = gk_ptr; o.gk_i = gk_i; o.gk_j = gk_j; o.gk_pk = gk_pk;
    o.L = pr.L; o.nl = pr.nl; o.P = pr.P; o.PI = pr.PI; o.mass_h = (T)(pr.h * pr.h / 24.0);
    o.fP = sgk::make_fd(pr.P); o.fPI = sgk::make_fd(pr.PI); o.fL = sgk::make_fd(pr.L);
    o.fLm1 = sgk::make_fd(pr.L - 1); o.fLP = sgk::make_fd(pr.L * pr.P);
    return o;
  }
  template <typename T>
  sgm::Rows<T> mrows() const {
    sgm::Rows<T> r;
    r.rp = m_rp; r.col = m_col;
    if constexpr (sizeof(T) == 8) {
      r.kv = (const T*)m_kv; r.mv = (const T*)m_mv; r.gk_v = (const T*)gk_v;
    } else {
      r.kv = (const T*)m_kv32; r.mv = (const T*)m_mv32; r.gk_v = (const T*)gk_v32;
    }
    r.gk_ptr = gk_ptr; r.gk_i = gk_i; r.gk_j = gk_j;
    r.nl = pr.nl; r.P = pr.P; r.PI = pr.PI;
    return r;
  }
  long long nloc() const { return (long long)pr.nsub * pr.nl; }
  long long nl_len() const { return (long long)pr.nl * pr.P; }
  long long nvec() const { return (long long)pr.nsub * pr.nl * pr.P; }
  long long nGd() const { return (long long)pr.nG * pr.P; }
};

static std::string g_setup_err;
static unsigned long long* g_nlaunch_dev = nullptr;

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

// release one allocation made by dalloc (set-up scratch)
template <typename T>
static void dfree(sg_handle h, T** p) {
  if (!*p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i] == (void*)*p) {
      h->allocs.erase(h->allocs.begin() + i);
      break;
    }
  cudaFree(*p);
  *p = nullptr;
}

// ---------------------------------------------------------------------------------------------
// Graph helpers: a conditional handle and a conditional node whose body is captured on the next
// capture stream.  In eager mode the same code runs the body as a host loop driven by a device
// mirror of the condition.
// ---------------------------------------------------------------------------------------------
static int make_handle(sg_handle h, Ctx& cx, cudaGraphConditionalHandle* out) {
  *out = 0;
  if (!cx.capture) return SG_OK;
  cudaStreamCaptureStatus status;
  cudaGraph_t g;
  CK(cudaStreamGetCaptureInfo(cx.st, &status, nullptr, &g, nullptr, nullptr, nullptr));
  CK(cudaGraphConditionalHandleCreate(out, g, 0, 0));
  return SG_OK;
}

static int cond_node(sg_handle h, Ctx& cx, cudaGraphConditionalHandle hnd, bool is_while, const int* mirror,
                     const std::function<int(Ctx&)>& body) {
  if (!cx.capture) {
    // eager: evaluate the device condition on the host
    for (int guard = 0; guard < 100000; ++guard) {
      CK(cudaMemcpyAsync(h->hint, mirror, sizeof(int), cudaMemcpyDeviceToHost, cx.st));
      CK(cudaStreamSynchronize(cx.st));
      if (!h->hint[0]) return SG_OK;
      RET(body(cx));
      if (!is_while) return SG_OK;
    }
    h->err = "loop guard exceeded";
    return SG_ETIMEOUT;
  }
  if (cx.depth + 1 >= NSTREAMS) { h->err = "conditional nesting too deep"; return SG_ENOTSUP; }
  cudaStreamCaptureStatus status;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(cx.st, &status, nullptr, &g, &deps, nullptr, &ndeps));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hnd;
  np.conditional.type = is_while ? cudaGraphCondTypeWhile : cudaGraphCondTypeIf;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
  CK(cudaStreamUpdateCaptureDependencies(cx.st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  Ctx child{h->cs[cx.depth + 1], cx.depth + 1, true};
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(child.st, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int rc = body(child);
  cudaGraph_t tmp;
  cudaError_t e = cudaStreamEndCapture(child.st, &tmp);
  if (rc != SG_OK) return rc;
  if (e != cudaSuccess) { h->err = std::string("body capture: ") + cudaGetErrorString(e); return SG_ECUDA; }
  return SG_OK;
}

// ---------------------------------------------------------------------------------------------
// Batched inner CG on a subdomain pattern (0 Dirichlet, 1 Neumann): x = K_pat^{-1} rhs for nb
// problems (R per subdomain, subdomains from s0).  rhs must vanish outside the pattern's free
// nodes; x is returned in ws.x (FP64) or ws32.x (FP32).
// ---------------------------------------------------------------------------------------------
template <typename T>
static InnerWS<T>& wsT(sg_handle h);
template <>
InnerWS<double>& wsT<double>(sg_handle h) { return h->ws; }
template <>
InnerWS<float>& wsT<float>(sg_handle h) { return h->ws32; }

template <typename T>
static const LineFactor<T>& lfT(sg_handle h, int pat);
template <>
const LineFactor<double>& lfT<double>(sg_handle h, int pat) { return h->lf[pat]; }
template <>
const LineFactor<float>& lfT<float>(sg_handle h, int pat) { return h->lf32[pat]; }

// ---- autotuned tile shapes (process-wide, keyed by the problem shape) ----
struct TuneKey {
  int kind, tsize, L, P, PI, nnz, nb;
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, tsize, L, P, PI, nnz, nb) < std::tie(o.kind, o.tsize, o.L, o.P, o.PI, o.nnz, o.nb);
  }
};
static std::map<TuneKey, int> g_tune;  // kind 0: apply lines per block; 1: line-solve modes per block

static int tuned(int kind, size_t tsize, const sgh::Problem& pr, int nb) {
  auto it = g_tune.find(TuneKey{kind, (int)tsize, pr.L, pr.P, pr.PI, (int)pr.gk_v.size(), nb});
  return it == g_tune.end() ? 0 : it->second;
}

// ---- compile-time triple-product tables (sg_gfix.cuh) ----
// Calls f(C{}) with the compiled size of index id; returns f's result (or r0 for an unknown id).
template <class R, class F>
static R with_gfix(int id, R r0, F&& f) {
  namespace gf = sgk::gfix;
  switch (id) {
    case 0: return f(gf::C0{});
    case 1: return f(gf::C1{});
    case 2: return f(gf::C2{});
    case 3: return f(gf::C3{});
    case 4: return f(gf::C4{});
    case 5: return f(gf::C5{});
    case 6: return f(gf::C6{});
    default: return r0;
  }
}

// the compiled table must list exactly the host's nonzero triples, in the host's order
template <class C>
static bool gfix_matches(const sgh::Problem& pr) {
  if (pr.M != C::M || pr.p != C::p || pr.p_in != C::pin) return false;
  if (pr.P != C::P || pr.PI != C::PI || (int)pr.gk_v.size() != C::NNZ) return false;
  for (int k = 0; k <= pr.P; ++k)
    if (pr.gk_ptr[k] != C::kptr(k)) return false;
  for (int e = 0; e < C::NNZ; ++e)
    if (pr.gk_i[e] != C::ti(e) || pr.gk_j[e] != C::tj(e)) return false;
  return true;
}

// FP64 applies use the compiled table too (SG_FP64_RT selects the runtime-table kernel).  With every
// subdomain problem active (1024^2 workload from step 200) the compiled FP64 apply takes 4.44 ms per
// launch against 5.77 ms for the runtime table (FP64 step 2471 -> 2229 ms, mixed step 176 -> 168 ms).
// An earlier measurement in the first steps of the 128^2 workload, where most subdomain problems are
// inactive and the launch is latency-bound, had favoured the runtime table.
template <class C>
constexpr bool gfix_fp64_ok() { return true; }

// compiled table usable for element type T (-1: runtime-table kernel): the table must match the PCE
// sizes and a one-line tile of the compiled kernel (input lines and fluxes) must fit shared memory
constexpr size_t SMEM_TILE_FIX = 200 * 1024;
template <typename T>
static int gfix_for(const sgh::Problem& pr) {
  if (pr.gfix < 0) return -1;
  if (sizeof(T) == 8 && std::getenv("SG_FP64_RT")) return -1;
  const size_t L = pr.L, P = pr.P, PS = pr.P | 1;
  const size_t one_line = sizeof(T) * (3 * L * P + ((L - 1) + 2 * L) * PS) + 16;
  return one_line <= SMEM_TILE_FIX ? pr.gfix : -1;
}

// Kernel launch that may overlap its prologue with the tail of the previous kernel in the stream
// (programmatic dependent launch); the kernels wait on griddepcontrol before reading its outputs.
template <typename... KA, typename... A>
static cudaError_t launch_k(bool pdl, void (*k)(KA...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// Dynamic shared-memory opt-in plus the maximum shared-memory carveout.  Every kernel of the inner
// loop asks for the same L1 / shared split, so consecutive launches never wait for the SM to drain
// and repartition its on-chip memory.
template <typename... A>
static int smem_attr(sg_handle h, void (*f)(A...), int lim) {
  CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  CK(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared));
  return SG_OK;
}

// apply tile configuration: lines per block, dynamic shared memory, kappa staging
constexpr size_t SMEM_MAX = 232448 - 1024;  // opt-in dynamic shared memory per block (static use below 1 KB)
constexpr size_t SMEM_TILE = 200 * 1024;    // dynamic shared memory the tile kernels are opted into

template <typename T>
static void apply_cfg(const sgh::Problem& pr, int nb, int* TL, int* NT, size_t* sm, int* stage, int* nods = nullptr) {
  if (nods) *nods = 0;
  const int L = pr.L, P = pr.P, PI = pr.PI;
  const int PS = P | 1, PIS = PI | 1;
  const size_t nnz = pr.gk_v.size();
  auto edges = [&](int t) { return (size_t)t * (L - 1) + (size_t)(t + 1) * L; };
  if (gfix_for<T>(pr) >= 0) {
    // compiled-table variant: input lines and fluxes only; the largest tile that still gives
    // about two blocks per SM
    auto bytes = [&](int t) { return sizeof(T) * ((size_t)(t + 2) * L * P + edges(t) * PS) + 16; };
    int best = 1;
    for (int t : {8, 4, 2, 1}) {
      if (t > L) continue;
      const long long blocks = (long long)nb * ((L + t - 1) / t);
      if (bytes(t) <= 100 * 1024 && blocks >= 256) { best = t; break; }
    }
    if (const int t = tuned(0, sizeof(T), pr, nb)) best = t;
    if (const char* f = std::getenv("SG_APPLY_LINES")) {  // explicit tile height (tuning)
      const int t = std::atoi(f);
      if (t >= 1 && t <= L && bytes(t) <= SMEM_TILE) best = t;
    }
    *TL = best;
    *NT = (L + best - 1) / best;
    *stage = 0;
    *sm = bytes(best);
    return;
  }
  auto base = [&](int t) {
    return sizeof(T) * ((size_t)(t + 2) * L * P + 2 * edges(t) * PS + nnz) + sizeof(unsigned) * nnz +
           sizeof(int) * (P + 1) + 16;
  };
  auto kap = [&](int t) { return sizeof(T) * edges(t) * PIS; };
  const char* force = std::getenv("SG_FORCE_NODS");
  if (base(1) > SMEM_TILE || force) {
    // widest subdomains: no staged edge differences (formed on the fly), no staged weights; when
    // even a one-line tile with the staged table exceeds 200 KB, the table is read from global
    // memory and the tile may use the whole opt-in shared memory (SG_FORCE_NODS=2 forces this)
    const bool gtab_forced = force && force[0] == '2';
    auto bytes = [&](int t, bool gtab) {
      return sizeof(T) * ((size_t)(t + 2) * L * P + edges(t) * PS) + 16 +
             (gtab ? 0 : sizeof(T) * nnz + sizeof(unsigned) * nnz + sizeof(int) * (P + 1));
    };
    const bool gtab = gtab_forced || bytes(1, false) > SMEM_TILE;
    const size_t cap = gtab ? SMEM_MAX : SMEM_TILE;
    int best = 1;
    for (int t : {4, 2, 1})
      if (t <= L && bytes(t, gtab) <= cap && (long long)nb * ((L + t - 1) / t) >= 128) { best = t; break; }
    *TL = best;
    *NT = (L + best - 1) / best;
    *stage = 0;
    *sm = bytes(best, gtab);
    if (nods) *nods = gtab ? 2 : 1;
    return;
  }
  int best = 1;
  for (int t : {8, 4, 2, 1}) {
    if (t > L) continue;
    const long long blocks = (long long)nb * ((L + t - 1) / t);
    if (base(t) + kap(t) <= 110 * 1024 && (blocks >= 128 || t == 1)) { best = t; break; }
  }
  while (best > 1 && base(best) > SMEM_TILE) best /= 2;
  if (const int t = tuned(0, sizeof(T), pr, nb)) best = t;
  *TL = best;
  *NT = (L + best - 1) / best;
  *stage = base(best) + kap(best) <= SMEM_TILE ? 1 : 0;
  *sm = base(best) + (*stage ? kap(best) : 0);
}

template <typename T, typename TO, bool FUSEDP, bool DOT>
static int launch_apply_k(sg_handle h, cudaStream_t st, const Op<T>& op, int nb, int R, const T* xm, const T* xk,
                          TO* y, const TO* add, double cm, double ck, int mask, T* p0, T* p1, const T* z) {
  if (h->mesh) {  // general partitions: sparse-row apply (the fused-CG forms belong to the line solvers)
    if constexpr (FUSEDP || DOT) {
      h->err = "fused CG apply on a mesh problem";
      return SG_ENOTSUP;
    } else {
      const int s0 = (int)((op.cls - h->cls) / h->pr.nl);
      const long long n = (long long)nb * h->pr.nl * h->pr.P;
      sgk::k_mapply<T, TO><<<nblk(n), 256, 0, st>>>(h->mrows<T>(), h->cls, s0, nb, R, xm, xk, y, add, (T)cm, (T)ck,
                                                     mask, nullptr);
      CKL();
      return SG_OK;
    }
  }
  int TL, NT, stage, nods;
  size_t sm;
  apply_cfg<T>(h->pr, nb, &TL, &NT, &sm, &stage, &nods);
  const int fx = gfix_for<T>(h->pr);
  const unsigned grid = (unsigned)((long long)nb * NT);
  const int nnz = (int)h->pr.gk_v.size();
  if constexpr (sizeof(T) == 8 && sizeof(TO) == 8 && !FUSEDP && !DOT) {
    if (h->apply_f2 && fx >= 0) {
      const size_t off = (size_t)(op.kapE - (const double*)h->kapE);  // the Op's first subdomain
      const bool ok = with_gfix(fx, false, [&](auto c) -> bool {
        using C = decltype(c);
        sgk::k_apply_f2<C><<<grid, 256, sm, st>>>(op, nb, R, TL, NT, xm, xk, y, add, cm, ck, mask, h->kapE2 + off,
                                                  h->kapN2 + off);
        return true;
      });
      if (ok) {
        CKL();
        return SG_OK;
      }
    }
  }
  bool done = with_gfix(fx, false, [&](auto c) -> bool {
    using C = decltype(c);
    if constexpr (sizeof(T) == 4 || gfix_fp64_ok<C>()) {
      sgk::k_apply<T, TO, FUSEDP, DOT, C><<<grid, 256, sm, st>>>(op, nb, R, TL, NT, nnz, stage, xm, xk, y, add, (T)cm,
                                                                 (T)ck, mask, p0, p1, z, h->ctl.parity, h->ctl.beta,
                                                                 h->ctl.active, h->ctl.part_pq);
      return true;
    } else {
      return false;
    }
  });
  if (!done && nods == 2) {
    sgk::k_apply<T, TO, FUSEDP, DOT, sgk::GDynNoDSG><<<grid, 256, sm, st>>>(
        op, nb, R, TL, NT, nnz, stage, xm, xk, y, add, (T)cm, (T)ck, mask, p0, p1, z, h->ctl.parity, h->ctl.beta,
        h->ctl.active, h->ctl.part_pq);
    done = true;
  }
  if (!done && nods) {
    sgk::k_apply<T, TO, FUSEDP, DOT, sgk::GDynNoDS><<<grid, 256, sm, st>>>(
        op, nb, R, TL, NT, nnz, stage, xm, xk, y, add, (T)cm, (T)ck, mask, p0, p1, z, h->ctl.parity, h->ctl.beta,
        h->ctl.active, h->ctl.part_pq);
    done = true;
  }
  if (!done) {
    auto kern = sgk::k_apply<T, TO, FUSEDP, DOT>;
    kern<<<grid, 256, sm, st>>>(op, nb, R, TL, NT, nnz, stage, xm, xk, y, add, (T)cm, (T)ck, mask, p0, p1, z,
                                h->ctl.parity, h->ctl.beta, h->ctl.active, h->ctl.part_pq);
  }
  CKL();
  return SG_OK;
}

// The apply launch; with kernel timing class 4 selected (sg_kernel_timing) the FP64-input applies
// (float-float in the mixed path) are bracketed by CUDA events on their stream, outside capture.
template <typename T, typename TO, bool FUSEDP, bool DOT>
static int launch_apply(sg_handle h, cudaStream_t st, const Op<T>& op, int nb, int R, const T* xm, const T* xk, TO* y,
                        const TO* add, double cm, double ck, int mask, T* p0 = nullptr, T* p1 = nullptr,
                        const T* z = nullptr) {
  bool timed = false;
  if constexpr (sizeof(T) == 8 && sizeof(TO) == 8 && !FUSEDP && !DOT) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (h->kprof == 4) CK(cudaStreamIsCapturing(st, &cs));
    timed = h->kprof == 4 && cs == cudaStreamCaptureStatusNone;
  }
  if (timed) CK(cudaEventRecord(h->kev0, st));
  RET((launch_apply_k<T, TO, FUSEDP, DOT>(h, st, op, nb, R, xm, xk, y, add, cm, ck, mask, p0, p1, z)));
  if (timed) {
    CK(cudaEventRecord(h->kev1, st));
    CK(cudaEventSynchronize(h->kev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->kev0, h->kev1));
    h->kprof_ms += ms;
    h->kprof_n += 1;
  }
  return SG_OK;
}

// line-solve block: G modes (fast thread index) x Lp rows, G * Lp a multiple of 32; FP32 covers
// the modes of a problem with about two blocks, FP64 spreads them over more blocks.
template <typename T>
static size_t line_smem(int L, int G) {
  return sizeof(T) * (2 * (size_t)L * L + 2 * (size_t)L * L * G + (size_t)L * G);
}
static int pad4(int L) { return (L + 3) & ~3; }
template <typename T>
static size_t team_smem(int L, int G) {
  const size_t LL = (size_t)L * L, LS = pad4(L);
  const size_t tstride = LS + 2 * LL + ((4 - ((2 * LL) & 3)) & 3);
  return sizeof(T) * (LL * LS + ((2 * LL + 3) & ~(size_t)3) + (size_t)G * tstride);
}
constexpr int TEAM_LS_MAX = 40;  // padded row length of the largest staged factor

struct LineCfg {
  bool team;      // warp-team kernel with the factor staged in shared memory
  bool gs;        // block kernel reading the factor from global memory (widest subdomains)
  bool wide;      // register-tiled kernel streaming the padded factor (wide subdomains)
  int G, NG;      // modes per block, blocks per problem
  int GS;         // wide kernel: modes per block rounded up to a multiple of 4
  dim3 block;
  size_t smem;
};

// Register-tiled line solve (k_line_w): shared memory for the double-buffered padded factor and the
// three [rows][GS] line buffers; threads for the 4 x 4 tiles and for the coalesced line I/O.
template <typename T>
static size_t wide_smem(int L, int GS) {
  const size_t LSP = pad4(L);
  return sizeof(T) * (2 * (size_t)L * LSP + (2 * (size_t)L + LSP) * GS + 6 * (size_t)L);
}
template <typename T>
static int wide_threads(int L, int G, int GS) {
  const int tiles = (pad4(L) / 2) * (GS / 4);                           // 2 x 4 tiles
  const int io = G * ((L + sgk::lw_npf<T>() - 1) / sgk::lw_npf<T>());  // G x rows per pass
  return 32 * ((std::max(tiles, io) + 31) / 32);
}

// line-solve launch shape: FP32 uses the warp-team kernel when the whole factor fits in shared
// memory; wider subdomains use the register-tiled kernel (modes grouped so that the blocks about
// fill the GPU, at most 32 modes per block); otherwise (or with SG_LINE_OLD) the block-synchronous
// kernel with a double-buffered factor (G modes x Lp rows, G * Lp a multiple of 32, FP64 spreads the
// modes over more blocks).
constexpr int WIDE_LMIN = 41;  // subdomains at least this many nodes wide use k_line_w
template <typename T>
static LineCfg line_cfg(const sgh::Problem& pr, int nb_hint) {
  const int L = pr.L, P = pr.P;
  LineCfg c{};
  if (sizeof(T) == 4) {
    int gmax = 0;
    for (int g = 1; g <= std::min(P, 15); ++g)
      if (pad4(L) <= TEAM_LS_MAX && team_smem<T>(L, g) <= SMEM_MAX && 32 * ((L + 31) / 32) * g <= 1024) gmax = g;
    if (gmax >= 1) {
      // one block per SM (the staged factor fills shared memory): pick the fewest modes per block
      // that keep the (problem, mode group) blocks within one wave of 152 SMs
      const int nbp = std::max(1, nb_hint);
      int g = std::max(1, (P * nbp + 151) / 152);
      g = std::min(g, gmax);
      if (const int t = tuned(1, sizeof(T), pr, nb_hint)) g = std::min(t, gmax);
      c.team = true;
      c.NG = (P + g - 1) / g;
      c.G = (P + c.NG - 1) / c.NG;
      c.block = dim3(32 * ((L + 31) / 32) * c.G);
      c.smem = team_smem<T>(L, c.G);
      return c;
    }
  }
  if (L >= WIDE_LMIN && !std::getenv("SG_LINE_OLD")) {
    const int nbp = std::max(1, nb_hint);
    int ng = std::max((P + 31) / 32, (4 * 152 / 5 + nbp - 1) / nbp);
    if (const int t = tuned(1, sizeof(T), pr, nb_hint)) ng = (P + std::min(t, 32) - 1) / std::min(t, 32);
    ng = std::min(ng, P);
    int G = (P + ng - 1) / ng;
    ng = (P + G - 1) / G;
    const int GS = pad4(G);
    if (wide_smem<T>(L, GS) <= SMEM_TILE && wide_threads<T>(L, G, GS) <= sgk::LW_MAXT) {
      c.wide = true;
      c.G = G;
      c.GS = GS;
      c.NG = ng;
      c.block = dim3(wide_threads<T>(L, G, GS));
      c.smem = wide_smem<T>(L, GS);
      return c;
    }
  }
  int g = sizeof(T) == 8 ? 2 : (P + 1) / 2;
  if (const int t = tuned(1, sizeof(T), pr, nb_hint)) g = t;
  g = std::max(1, std::min(g, 1024 / L));
  while (g > 1 && line_smem<T>(L, g) > SMEM_TILE) --g;
  c.gs = line_smem<T>(L, g) > SMEM_TILE || std::getenv("SG_FORCE_GLINE");
  if (c.gs) {  // factor and residual from global memory: solution slice only
    auto gsm = [&](int gg) { return sizeof(T) * ((size_t)L * L * gg + (size_t)L * gg); };
    g = std::max(1, std::min(g, 1024 / L));
    while (g > 1 && gsm(g) > SMEM_TILE) --g;
  }
  // rows padded so that the block is whole warps; keep the block within 1024 threads
  auto rows_for = [&](int gg) {
    int lp = L;
    while ((gg * lp) % 32) ++lp;
    return lp;
  };
  while (g > 1 && g * rows_for(g) > 1024) --g;
  const int lp = rows_for(g);
  c.team = false;
  c.G = g;
  c.NG = (P + g - 1) / g;
  c.block = dim3(g, lp);
  c.smem = c.gs ? sizeof(T) * ((size_t)L * L * g + (size_t)L * g) : line_smem<T>(L, g);
  return c;
}

// Tensor-core line sweeps (k_line_tc) for the FP32 solves of subdomains of WIDE_LMIN .. 65 nodes per
// side whose line plan is the register-tiled kernel (at most 32 modes per block): the SG_BF16 policy
// (BF16 mean-operator products on the tensor cores).  SG_MIXED keeps the FP32 products of k_line_w,
// which measured faster: on the 1024^2 workload with every subdomain active 597 us per launch against
// 631 us, since the line product is not what bounds a line step (input phase, barriers and the
// dependent sweep are).
constexpr int LTC_LMAX = 65;
static bool line_tc_eligible(const sgh::Problem& pr, int policy) {
  if (policy != SG_BF16) return false;
  if (pr.L < WIDE_LMIN || pr.L > LTC_LMAX) return false;
  const LineCfg lc = line_cfg<float>(pr, pr.nsub);
  return lc.wide && lc.G <= 32;
}
static int ltc_nb(int G) { return G <= 16 ? 16 : 32; }
// threads: four warps for the 128 accumulator lanes, and G x ceil(L / 8) for the line I/O
static int ltc_threads(int L, int G) { return 32 * ((std::max(128, G * ((L + 7) / 8)) + 31) / 32); }

static int ensure_ctl(sg_handle h, int nb, int nt, int ng) {
  if (h->ctl_cap_nb >= nb && h->ctl_cap_nt >= nt && h->ctl_cap_ng >= ng) return SG_OK;
  nb = std::max(nb, h->ctl_cap_nb);
  nt = std::max(nt, h->ctl_cap_nt);
  ng = std::max(ng, h->ctl_cap_ng);
  auto& c = h->ctl;
  RET(dalloc(h, &c.rz, nb)); RET(dalloc(h, &c.bb, nb)); RET(dalloc(h, &c.beta, nb));
  RET(dalloc(h, &c.active, nb));
  RET(dalloc(h, &c.part_pq, (long long)nb * nt));
  RET(dalloc(h, &c.part_rz, (long long)nb * ng)); RET(dalloc(h, &c.part_rr, (long long)nb * ng));
  if (!c.counter) {
    RET(dalloc(h, &c.counter, 1)); RET(dalloc(h, &c.parity, 1)); RET(dalloc(h, &c.it, 1));
    RET(dalloc(h, &c.it_total, 1)); RET(dalloc(h, &c.cond, 1)); RET(dalloc(h, &c.breakdown, 1));
  }
  h->ctl_cap_nb = nb; h->ctl_cap_nt = nt; h->ctl_cap_ng = ng;
  return SG_OK;
}

// residual image of the tensor-core preconditioner for nb right-hand sides
static int ensure_bimg(sg_handle h, int nb) {
  if (!h->mma || h->bimg_cap >= nb) return SG_OK;
  RET(dalloc(h, &h->bimg, (long long)nb * h->NC * 2 * h->mma_nb * 128));
  h->bimg_cap = nb;
  return SG_OK;
}

template <typename T>
static int ensure_ws(sg_handle h, int nb) {
  auto& w = wsT<T>(h);
  if (sizeof(T) == 4) RET(ensure_bimg(h, nb));
  if (w.cap_nb < nb) {
    const long long len = (long long)h->pr.nl * h->pr.P * nb;
    RET(dalloc(h, &w.x, len)); RET(dalloc(h, &w.r, len)); RET(dalloc(h, &w.z, len));
    RET(dalloc(h, &w.p0, len)); RET(dalloc(h, &w.p1, len)); RET(dalloc(h, &w.q, len));
    w.cap_nb = nb;
  }
  if (h->mesh) {
    // one p.q, r.z, r.r per problem; the tensor-core loop keeps per-block p.q and per-row-tile partials
    const int nt = h->mma ? (int)((h->nl_len() + 255) / 256) : 1;
    return ensure_ctl(h, nb, nt, h->mma ? std::max(h->pr.P, h->MT) : 1);
  }
  int TL, NT, stage;
  size_t sm;
  apply_cfg<T>(h->pr, nb, &TL, &NT, &sm, &stage);
  // capacities cover every tile shape the tuner may pick: NT <= L, NG <= max(P, row tiles)
  (void)NT;
  return ensure_ctl(h, nb, h->pr.L, std::max(h->pr.P, h->MT));
}

// CUDA-event timing of one kernel launch on its stream (host-driven enqueue only)
static int kprof_begin(sg_handle h, Ctx& cx, int which) {
  if (h->kprof != which || cx.capture) return SG_OK;
  CK(cudaEventRecord(h->kev0, cx.st));
  return SG_OK;
}
static int kprof_end(sg_handle h, Ctx& cx, int which) {
  if (h->kprof != which || cx.capture) return SG_OK;
  CK(cudaEventRecord(h->kev1, cx.st));
  CK(cudaEventSynchronize(h->kev1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, h->kev0, h->kev1));
  h->kprof_ms += ms;
  h->kprof_n += 1;
  return SG_OK;
}

template <typename T>
static int enq_inner_mesh(sg_handle h, Ctx& cx, int pat, int nb, int R, int s0, const T* rhs, double tol_override);

template <typename T>
static int enq_inner(sg_handle h, Ctx& cx, int pat, int nb, int R, int s0, const T* rhs, double tol_override = 0.0) {
  if (h->mesh) return enq_inner_mesh<T>(h, cx, pat, nb, R, s0, rhs, tol_override);
  const auto& pr = h->pr;
  auto& w = wsT<T>(h);
  const long long n = (long long)pr.nl * pr.P * nb;
  const Op<T> op = h->op<T>(s0);
  const int mask = pat == 0 ? sgk::MASK_I : pat == 1 ? sgk::MASK_N : sgk::MASK_FREE;
  const int L = pr.L;
  const LineCfg lc = line_cfg<T>(pr, nb);
  const int NG = lc.NG;
  int TL, NT, stage;
  size_t asm_;
  apply_cfg<T>(pr, nb, &TL, &NT, &asm_, &stage);
  const long long pstride = (long long)L * L * L;
  const auto& lf = lfT<T>(h, pat);
  const T* Sinv = lf.Sinv + (size_t)s0 * pstride;
  const T* Bd = lf.Bd + (size_t)s0 * L * L;
  const T* Bu = lf.Bu + (size_t)s0 * L * L;
  const double tol = tol_override > 0.0 ? tol_override : (sizeof(T) == 8 ? h->inner_tol : h->inner_tol32);
  const double tol2 = tol * tol;
  // right-hand sides whose squared norm is at the underflow level of T are left at x = 0
  const double bb_min = sizeof(T) == 8 ? 1e-280 : 1e-60;
  const int imax = sizeof(T) == 8 ? h->inner_max : std::min(h->inner_max, 120);
  const unsigned lg = (unsigned)nb * NG;
  const int LSp = pad4(L);
  const long long pstride_pad = (long long)L * L * LSp;
  const T* Sinv_pad = lf.Spad ? lf.Spad + (size_t)s0 * pstride_pad : nullptr;
  auto line = [&](cudaStream_t s, int init, cudaGraphConditionalHandle hh, int use) {
    if (lc.team) {
#define SG_TEAM(LSV)                                                                                              \
  case LSV:                                                                                                       \
    sgk::k_line_team<T, LSV><<<lg, lc.block, lc.smem, s>>>(L, pr.nl, pr.P, R, NG, NT, lc.G, pstride_pad, Sinv_pad, \
                                                           Bd, Bu, nb, w.x, w.r, w.z, w.p0, w.p1, w.q, h->ctl, init, \
                                                           tol2, bb_min, imax, hh, use);                         \
    break;
      switch (LSp) {
        SG_TEAM(4) SG_TEAM(8) SG_TEAM(12) SG_TEAM(16) SG_TEAM(20) SG_TEAM(24) SG_TEAM(28) SG_TEAM(32) SG_TEAM(36)
        SG_TEAM(40)
        default: break;
      }
#undef SG_TEAM
    } else if (lc.wide) {
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        if (h->line_tc && pat < 2) {
          const int nbv = ltc_nb(lc.G);
          const dim3 thr((unsigned)ltc_threads(L, lc.G));
          const size_t smb = sgk::ltc_smem(L, lc.G, nbv);
          const long long row0 = (long long)s0 * L * L;
          const float* colp = h->lcol[pat] + (size_t)s0 * L * sgk::LTC_COLN;
          if (nbv == 16)
            sgk::k_line_tc<16><<<lg, thr, smb, s>>>(h->tmL[pat], L, pr.nl, pr.P, R, NG, NT, lc.G, row0, colp, Bd, Bu,
                                                    nb, w.x, w.r, w.z, w.p0, w.p1, w.q, h->ctl, init, tol2, bb_min,
                                                    imax, hh, use);
          else
            sgk::k_line_tc<32><<<lg, thr, smb, s>>>(h->tmL[pat], L, pr.nl, pr.P, R, NG, NT, lc.G, row0, colp, Bd, Bu,
                                                    nb, w.x, w.r, w.z, w.p0, w.p1, w.q, h->ctl, init, tol2, bb_min,
                                                    imax, hh, use);
          done = true;
        }
      }
      if (!done)
        sgk::k_line_w<T><<<lg, lc.block, lc.smem, s>>>(L, LSp, pr.nl, pr.P, R, NG, NT, lc.G, lc.GS, pstride_pad,
                                                       Sinv_pad, Bd, Bu, nb, w.x, w.r, w.z, w.p0, w.p1, w.q, h->ctl,
                                                       init, tol2, bb_min, imax, hh, use);
    } else if (lc.gs)
      sgk::k_line<T, true><<<lg, lc.block, lc.smem, s>>>(L, pr.nl, pr.P, R, NG, NT, pstride, Sinv, Bd, Bu, nb, w.x,
                                                         w.r, w.z, w.p0, w.p1, w.q, h->ctl, init, tol2, bb_min, imax,
                                                         hh, use);
    else
      sgk::k_line<T><<<lg, lc.block, lc.smem, s>>>(L, pr.nl, pr.P, R, NG, NT, pstride, Sinv, Bd, Bu, nb, w.x, w.r,
                                                   w.z, w.p0, w.p1, w.q, h->ctl, init, tol2, bb_min, imax, hh, use);
  };
  // tensor-core preconditioner (FP32 solves of small subdomains): CG update + residual image, then
  // the dense product with the inner-CG control
  const bool use_mma = sizeof(T) == 4 && h->mma && pat < 2;  // the dense inverses cover patterns 0 and 1
  const int row0 = (pat * pr.nsub + s0) * h->Kp;
  auto pre_mma = [&](Ctx& cc, int init, cudaGraphConditionalHandle hh, int use) -> int {
    cudaStream_t s = cc.st;
    float* wx = (float*)w.x;
    float* wr = (float*)w.r;
    float* wz = (float*)w.z;
    const float* p0 = (const float*)w.p0;
    const float* p1 = (const float*)w.p1;
    const float* wq = (const float*)w.q;
    const unsigned gp = (unsigned)nb * h->NC, gm = (unsigned)nb * h->MT;
    // inside the loop body the pack follows the apply and the product follows the pack: both may
    // start early (PDL); the first pack of a solve follows a copy and launches normally
    const bool pdl_pack = h->pdl && !init && h->kprof == 0;
    const bool pdl_mma = h->pdl && h->kprof == 0;
    if (h->mma_nb == 32)
      CK(launch_k(pdl_pack, sgk::k_cg_pack<32, 2>, dim3(gp), dim3(256), 0, s, L, pr.nl, pr.P, h->NC, NT, wx, wr, p0,
                  p1, wq, h->ctl, init, h->bimg));
    else
      CK(launch_k(pdl_pack, sgk::k_cg_pack<16, 2>, dim3(gp), dim3(256), 0, s, L, pr.nl, pr.P, h->NC, NT, wx, wr, p0,
                  p1, wq, h->ctl, init, h->bimg));
    RET(kprof_begin(h, cc, 3));
#define SG_PRE(NBV, SMEMV)                                                                                      \
  CK(launch_k(pdl_mma, sgk::k_pre_mma<NBV>, dim3(gm), dim3(256), (size_t)SMEMV, s, h->tmA, L, pr.nl, pr.P, R,     \
              h->MT, h->NC, NT, h->Kp, row0, nb, (const unsigned char*)h->bimg, (const float*)wr, wz, h->ctl, init, \
              tol2, bb_min, imax, hh, use, h->ctl.breakdown))
    if (h->mma_nb == 32) SG_PRE(32, (sgk::PreShape<32, 2>::SMEM));
    else SG_PRE(16, (sgk::PreShape<16, 2>::SMEM));
#undef SG_PRE
    RET(kprof_end(h, cc, 3));
    return SG_OK;
  };
  if (use_mma && h->bimg_cap < nb) {
    h->err = "residual image smaller than the batch of inner solves";
    return SG_EINVAL;
  }
  CK(cudaMemcpyAsync(w.r, rhs, sizeof(T) * n, cudaMemcpyDeviceToDevice, cx.st));
  CK(cudaMemsetAsync(w.x, 0, sizeof(T) * n, cx.st));
  cudaGraphConditionalHandle hnd;
  RET(make_handle(h, cx, &hnd));
  if (use_mma) {
    RET(pre_mma(cx, 1, hnd, cx.capture ? 1 : 0));
    CKL();
    return cond_node(h, cx, hnd, true, h->ctl.cond, [&](Ctx& c2) -> int {
      RET(kprof_begin(h, c2, 2));
      RET((launch_apply<T, T, true, true>(h, c2.st, op, nb, R, nullptr, nullptr, w.q, nullptr, h->am, h->bk, mask,
                                          w.p0, w.p1, w.z)));
      RET(kprof_end(h, c2, 2));
      RET(kprof_begin(h, c2, 1));
      RET(pre_mma(c2, 0, hnd, c2.capture ? 1 : 0));
      CKL();
      RET(kprof_end(h, c2, 1));
      return SG_OK;
    });
  }
  line(cx.st, 1, hnd, cx.capture ? 1 : 0);
  CKL();
  return cond_node(h, cx, hnd, true, h->ctl.cond, [&](Ctx& c2) -> int {
    RET(kprof_begin(h, c2, 2));
    RET((launch_apply<T, T, true, true>(h, c2.st, op, nb, R, nullptr, nullptr, w.q, nullptr, h->am, h->bk, mask,
                                        w.p0, w.p1, w.z)));
    RET(kprof_end(h, c2, 2));
    RET(kprof_begin(h, c2, 1));
    line(c2.st, 0, hnd, c2.capture ? 1 : 0);
    CKL();
    RET(kprof_end(h, c2, 1));
    return SG_OK;
  });
}

// FP32 mesh solves with the mean-operator inverse on the tensor cores (SG_BF16 on a mesh): the loop of
// the structured tensor-core path (k_cg_pack: CG update and BF16 residual image; k_pre_mma: the product
// and the loop control) behind the mesh's fused direction-and-apply kernel.  The inverse image holds
// patterns 0 and 1.
static int enq_inner_mesh_mma(sg_handle h, Ctx& cx, int pat, int nb, int R, int s0, const float* rhs, double tol2,
                              double bb_min, int imax, int mask) {
  const auto& pr = h->pr;
  auto& w = h->ws32;
  const long long len = h->nl_len(), n = len * nb;
  const int NT = (int)((len + 255) / 256);
  if (h->bimg_cap < nb || h->ctl_cap_nt < NT || h->ctl_cap_ng < h->MT) {
    h->err = "mesh tensor-core solve: residual image or control arrays smaller than the batch";
    return SG_EINVAL;
  }
  const sgm::Rows<float> rows = h->mrows<float>();
  const int row0 = (pat * pr.nsub + s0) * h->Kp;
  auto pre = [&](Ctx& cc, int init, cudaGraphConditionalHandle hh, int use) -> int {
    cudaStream_t s = cc.st;
    const unsigned gp = (unsigned)nb * h->NC, gm = (unsigned)nb * h->MT;
    if (h->mma_nb == 32)
      sgk::k_cg_pack<32, 2><<<gp, 256, 0, s>>>(0, pr.nl, pr.P, h->NC, NT, w.x, w.r, w.p0, w.p1, w.q, h->ctl, init,
                                                h->bimg);
    else
      sgk::k_cg_pack<16, 2><<<gp, 256, 0, s>>>(0, pr.nl, pr.P, h->NC, NT, w.x, w.r, w.p0, w.p1, w.q, h->ctl, init,
                                                h->bimg);
    if (h->mma_nb == 32)
      sgk::k_pre_mma<32><<<gm, 256, (size_t)sgk::PreShape<32, 2>::SMEM, s>>>(
          h->tmA, 0, pr.nl, pr.P, R, h->MT, h->NC, NT, h->Kp, row0, nb, h->bimg, w.r, w.z, h->ctl, init, tol2, bb_min,
          imax, hh, use, h->ctl.breakdown);
    else
      sgk::k_pre_mma<16><<<gm, 256, (size_t)sgk::PreShape<16, 2>::SMEM, s>>>(
          h->tmA, 0, pr.nl, pr.P, R, h->MT, h->NC, NT, h->Kp, row0, nb, h->bimg, w.r, w.z, h->ctl, init, tol2, bb_min,
          imax, hh, use, h->ctl.breakdown);
    CKL();
    return SG_OK;
  };
  CK(cudaMemcpyAsync(w.r, rhs, sizeof(float) * n, cudaMemcpyDeviceToDevice, cx.st));
  CK(cudaMemsetAsync(w.x, 0, sizeof(float) * n, cx.st));
  cudaGraphConditionalHandle hnd;
  RET(make_handle(h, cx, &hnd));
  RET(pre(cx, 1, hnd, cx.capture ? 1 : 0));
  return cond_node(h, cx, hnd, true, h->ctl.cond, [&](Ctx& c2) -> int {
    RET(kprof_begin(h, c2, 2));   // kernel timing class 2: the operator apply of the inner loop
    sgk::k_mapply_cg<float><<<(unsigned)nb * NT, 256, 0, c2.st>>>(rows, h->cls, s0, R, NT, w.z, w.p0, w.p1, w.q,
                                                                  (float)h->am, (float)h->bk, mask, h->ctl);
    CKL();
    RET(kprof_end(h, c2, 2));
    RET(kprof_begin(h, c2, 1));   // class 1: the preconditioner step (pack and tensor-core product)
    RET(pre(c2, 0, hnd, c2.capture ? 1 : 0));
    return kprof_end(h, c2, 1);
  });
}

// The same batched solve on the sparse rows of a mesh problem: CG preconditioned by the dense inverse
// of each subdomain's mean operator on the pattern's rows; per iteration the apply (active problems),
// p.q, the update, the preconditioner, r.r and r.z, the control (loop condition) and the new
// direction.  Same stopping rule, tolerances and iteration cap as the line solvers.
template <typename T>
static int enq_inner_mesh(sg_handle h, Ctx& cx, int pat, int nb, int R, int s0, const T* rhs, double tol_override) {
  const auto& pr = h->pr;
  auto& w = wsT<T>(h);
  const T* Ainv = pat < 0 || pat > 2 ? nullptr : sizeof(T) == 8 ? (const T*)h->m_ainv[pat] : (const T*)h->m_ainv32[pat];
  if (pat < 0 || pat > 2 || !Ainv || nb < 1 || R < 1 || s0 < 0 || w.cap_nb < nb || h->ctl_cap_nb < nb ||
      s0 + (nb + R - 1) / R > pr.nsub) {
    h->err = "mesh subdomain solve: pattern, workspace or batch out of range";
    return SG_EINVAL;
  }
  const long long len = (long long)pr.nl * pr.P, n = len * nb;
  const int mask = pat == 0 ? sgk::MASK_I : pat == 1 ? sgk::MASK_N : sgk::MASK_FREE;
  const double tol = tol_override > 0.0 ? tol_override : (sizeof(T) == 8 ? h->inner_tol : h->inner_tol32);
  const double tol2 = tol * tol;
  const double bb_min = sizeof(T) == 8 ? 1e-280 : 1e-60;
  const int imax = sizeof(T) == 8 ? h->inner_max : std::min(h->inner_max, 120);
  const int* npat = h->m_npat + (size_t)pat * pr.nsub;
  const sgm::Rows<T> rows = h->mrows<T>();
  const T am = (T)h->am, bk = (T)h->bk;
  cudaStream_t st = cx.st;
  if constexpr (sizeof(T) == 4) {
    if (h->mma && pat < 2) return enq_inner_mesh_mma(h, cx, pat, nb, R, s0, rhs, tol2, bb_min, imax, mask);
  }
  CK(cudaMemcpyAsync(w.r, rhs, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(w.x, 0, sizeof(T) * n, st));
  sgk::k_mdense<T><<<nblk(n), 256, 0, st>>>(Ainv, npat, s0, nb, R, pr.nl, pr.P, w.r, w.z, nullptr);
  sgk::k_mdot2<T><<<nb, sgk::MDOT_THREADS, 0, st>>>(len, w.r, w.r, h->ctl.part_rr, w.r, w.z, h->ctl.part_rz, nullptr);
  cudaGraphConditionalHandle hnd;
  RET(make_handle(h, cx, &hnd));
  sgk::k_mcg_ctl<<<1, 256, 0, st>>>(nb, h->ctl, 1, tol2, bb_min, imax, hnd, cx.capture ? 1 : 0);
  sgk::k_mcg_dir<T><<<nblk(n), 256, 0, st>>>(len, nb, h->ctl, 1, w.z, w.p0);
  CKL();
  return cond_node(h, cx, hnd, true, h->ctl.cond, [&](Ctx& c2) -> int {
    cudaStream_t s = c2.st;
    RET(kprof_begin(h, c2, 2));   // kernel timing class 2: the operator apply of the inner loop
    sgk::k_mapply<T, T><<<nblk(n), 256, 0, s>>>(rows, h->cls, s0, nb, R, w.p0, w.p0, w.q, nullptr, am, bk, mask,
                                                 h->ctl.active);
    RET(kprof_end(h, c2, 2));
    sgk::k_mdot2<T><<<nb, sgk::MDOT_THREADS, 0, s>>>(len, w.p0, w.q, h->ctl.part_pq, nullptr, nullptr, nullptr,
                                                      h->ctl.active);
    sgk::k_mcg_upd<T><<<nblk(n), 256, 0, s>>>(len, nb, h->ctl, w.x, w.r, w.p0, w.q);
    RET(kprof_begin(h, c2, 1));   // class 1: the preconditioner step
    sgk::k_mdense<T><<<nblk(n), 256, 0, s>>>(Ainv, npat, s0, nb, R, pr.nl, pr.P, w.r, w.z, h->ctl.active);
    RET(kprof_end(h, c2, 1));
    sgk::k_mdot2<T><<<nb, sgk::MDOT_THREADS, 0, s>>>(len, w.r, w.r, h->ctl.part_rr, w.r, w.z, h->ctl.part_rz,
                                                      h->ctl.active);
    sgk::k_mcg_ctl<<<1, 256, 0, s>>>(nb, h->ctl, 0, tol2, bb_min, imax, hnd, c2.capture ? 1 : 0);
    sgk::k_mcg_dir<T><<<nblk(n), 256, 0, s>>>(len, nb, h->ctl, 0, w.z, w.p0);
    CKL();
    return SG_OK;
  });
}

// ---------------------------------------------------------------------------------------------
// Interface operators
// ---------------------------------------------------------------------------------------------
// q = S p = sum_s R_s^T (K_GG - K_GI K_II^{-1} K_IG) R_s p
static int enq_schur(sg_handle h, Ctx& cx, const double* p, double* q) {
  const auto& pr = h->pr;
  cudaStream_t st = cx.st;
  const int nsub = pr.nsub, nl = pr.nl, P = pr.P;
  const long long n = h->nvec();
  const Op<double> op = h->op<double>();
  if (h->precision == SG_FP64) {
    sgk::k_gather<double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, p, h->wa, sgk::MASK_G, 0);
    RET((launch_apply<double, double, false, false>(h, st, op, nsub, 1, h->wa, h->wa, h->wb, nullptr, -h->am, -h->bk,
                                                    sgk::MASK_I)));
    RET(enq_inner<double>(h, cx, 0, nsub, 1, 0, h->wb));
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->wa, 1.0, h->ws.x, h->wd);
    RET((launch_apply<double, double, false, false>(h, st, op, nsub, 1, h->wd, h->wd, h->wb, nullptr, h->am, h->bk,
                                                    sgk::MASK_G)));
  } else {
    const Op<float> o32 = h->op<float>();
    // b32 = -(K32 [0; p])_I, first FP32 solve
    sgk::k_gather<float><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, p, h->fa, sgk::MASK_G, 0);
    RET((launch_apply<float, float, false, false>(h, st, o32, nsub, 1, h->fa, h->fa, h->fb, nullptr, -h->am, -h->bk,
                                                  sgk::MASK_I)));
    RET(enq_inner<float>(h, cx, 0, nsub, 1, 0, h->fb));
    // y1 = K64 [w0; p] on all free rows; residual r_I = -y1_I
    sgk::k_gather<double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, p, h->wa, sgk::MASK_G, 0);
    sgk::k_add_conv<float><<<nblk(n), 256, 0, st>>>(n, h->ws32.x, h->wa, h->wd);
    RET((launch_apply<double, double, false, false>(h, st, op, nsub, 1, h->wd, h->wd, h->wb, nullptr, h->am, h->bk,
                                                    sgk::MASK_FREE)));
    sgk::k_conv_mask<double, float><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->wb, h->fb, sgk::MASK_I, -1.0);
    RET(enq_inner<float>(h, cx, 0, nsub, 1, 0, h->fb));
    // y2_G = y1_G + (K32 [e; 0])_G
    RET((launch_apply<float, double, false, false>(h, st, o32, nsub, 1, h->ws32.x, h->ws32.x, h->wb, h->wb, h->am,
                                                   h->bk, sgk::MASK_G)));
  }
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, pr.mo, h->Dw, h->wb, q, 0);
  CKL();
  return SG_OK;
}

// z = M_NNC^{-1} r (Eq. NNCP2)
template <typename T>
static int enq_precond_t(sg_handle h, Ctx& cx, const double* r, double* z) {
  const auto& pr = h->pr;
  cudaStream_t st = cx.st;
  const int nsub = pr.nsub, nl = pr.nl, P = pr.P;
  const long long n = h->nvec();
  const Op<T> op = h->op<T>();
  T* wr = sizeof(T) == 8 ? (T*)h->wa : (T*)h->fa;
  T* wy = sizeof(T) == 8 ? (T*)h->wd : (T*)h->fb;
  // w_s = D_s R_s r on remaining nodes (Neumann RHS) and on corners
  sgk::k_gather<T><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, r, wr, sgk::MASK_R, 1);
  sgk::k_gather<double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, r, h->wc, sgk::MASK_C, 1);
  // v = [y; t], t = S_rr^{-1} w_r; in mixed mode the preconditioner solve is approximate (the outer
  // PCG uses the flexible beta)
  RET(enq_inner<T>(h, cx, 1, nsub, 1, 0, wr, sizeof(T) == 8 ? 0.0 : h->prec_tol32));
  const T* v = wsT<T>(h).x;
  if (pr.nC > 0) {
    // S_cr t = (K~ [y; t; 0])_c ;  d = sum_s B^T (w_c - S_cr t) ;  u_c = F_cc^{-1} d  (FP64)
    RET((launch_apply<T, T, false, false>(h, st, op, nsub, 1, v, v, wy, nullptr, h->am, h->bk, sgk::MASK_C)));
    sgk::k_corner_rhs<T><<<nblk((long long)pr.nC * P), 256, 0, st>>>(pr.nC, P, h->cowners, pr.mo, h->wc, wy, h->dC);
    sgk::k_gemv<<<nblk((long long)h->nCd * 32), 256, 0, st>>>(h->nCd, h->Finv, h->dC, h->uC);
  }
  sgk::k_coarse_extend<T><<<nblk((long long)nsub * pr.nGam * P), 256, 0, st>>>(
      nsub, nl, P, pr.nGam, pr.max_corner, h->cls, h->cidx, h->gam_ln, h->n_gam, h->loc_corner, pr.mc,
      h->n_loc_corner, h->Phi, h->uC, v, h->we);
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, pr.mo, h->Dw, h->we, z, 1);
  CKL();
  return SG_OK;
}

// One-level preconditioners of the comparison (Sec. 6.1), textbook forms:
//   lumped:  z = sum_s R_s^T D_s K~_GG^s D_s R_s r  (one FP64 apply restricted to the interface)
//   NN1:     z = sum_s R_s^T D_s S_s^{-1} D_s R_s r, S_s^{-1} w the interface part of the local Neumann
//            solve with the whole local interface free (line-factor pattern 2; no coarse space)
static int enq_precond_lumped(sg_handle h, Ctx& cx, const double* r, double* z) {
  const auto& pr = h->pr;
  cudaStream_t st = cx.st;
  const long long n = h->nvec();
  sgk::k_gather<double><<<nblk(n), 256, 0, st>>>(pr.nsub, 1, pr.nl, pr.P, h->cls, h->gidx, h->Dw, r, h->wa,
                                                  sgk::MASK_G, 1);
  RET((launch_apply<double, double, false, false>(h, st, h->op<double>(), pr.nsub, 1, h->wa, h->wa, h->we, nullptr,
                                                  h->am, h->bk, sgk::MASK_G)));
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, pr.P, h->owners, pr.mo, h->Dw, h->we, z, 1);
  CKL();
  return SG_OK;
}

template <typename T>
static int enq_precond_nn1(sg_handle h, Ctx& cx, const double* r, double* z) {
  const auto& pr = h->pr;
  cudaStream_t st = cx.st;
  const long long n = h->nvec();
  T* wr = sizeof(T) == 8 ? (T*)h->wa : (T*)h->fa;
  sgk::k_gather<T><<<nblk(n), 256, 0, st>>>(pr.nsub, 1, pr.nl, pr.P, h->cls, h->gidx, h->Dw, r, wr, sgk::MASK_G, 1);
  RET(enq_inner<T>(h, cx, 2, pr.nsub, 1, 0, wr, sizeof(T) == 8 ? 0.0 : h->prec_tol32));
  sgk::k_scatter<T><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, pr.P, h->owners, pr.mo, h->Dw, wsT<T>(h).x, z, 1);
  CKL();
  return SG_OK;
}

static int enq_precond(sg_handle h, Ctx& cx, const double* r, double* z) {
  if (h->pc == SG_PC_LUMPED) return enq_precond_lumped(h, cx, r, z);
  if (h->pc == SG_PC_NN1)
    return h->precision == SG_FP64 ? enq_precond_nn1<double>(h, cx, r, z) : enq_precond_nn1<float>(h, cx, r, z);
  return h->precision == SG_FP64 ? enq_precond_t<double>(h, cx, r, z) : enq_precond_t<float>(h, cx, r, z);
}

// PCG on S x = G (Hestenes-Stiefel; flexible Polak-Ribiere beta in mixed mode); x holds the
// initial guess; stops at ||r|| / ||G|| <= tol.
static int enq_outer(sg_handle h, Ctx& cx) {
  const long long n = h->nGd();
  const int nbo = (int)std::min<long long>(NB_OUT, std::max<long long>(1, (n + 255) / 256));
  cudaStream_t st = cx.st;
  const int flex = h->precision != SG_FP64;
  sgk::k_odot<<<nbo, 256, 0, st>>>(n, h->gG, h->gG, nullptr, nullptr, h->opart, nullptr);
  sgk::k_octl<<<1, 32, 0, st>>>(sgk::OP_INIT_G, nbo, h->opart, nullptr, h->octl, h->tol, h->max_iter, 0, 0, 0, h->omirror);
  sgk::k_ozero_if<<<nbo, 256, 0, st>>>(n, h->octl, h->xG);
  CKL();
  RET(enq_schur(h, cx, h->xG, h->qG));
  const long long nl_all = h->nvec();
  if (h->a6_rec)  // W_I += K_II^{-1}(-K_IG x0): interior part of the extension just computed
    sgk::k_wacc<<<nblk(nl_all), 256, 0, st>>>(nl_all, h->pr.P, h->cls, nullptr, 0, h->wd, h->ws32.x, h->Wrec);
  sgk::k_ores0<<<nbo, 256, 0, st>>>(n, h->gG, h->qG, h->rG, h->opart);
  cudaGraphConditionalHandle hw, hif;
  RET(make_handle(h, cx, &hw));
  RET(make_handle(h, cx, &hif));
  sgk::k_octl<<<1, 32, 0, st>>>(sgk::OP_RES0, nbo, h->opart, nullptr, h->octl, h->tol, h->max_iter, hw, hif,
                                cx.capture ? 1 : 0, h->omirror);
  CKL();
  RET(cond_node(h, cx, hif, false, h->omirror + 1, [&](Ctx& c) -> int {
    RET(enq_precond(h, c, h->rG, h->zG));
    sgk::k_op<<<nbo, 256, 0, c.st>>>(n, h->octl, h->zG, h->pG, 1);
    sgk::k_odot<<<nbo, 256, 0, c.st>>>(n, h->rG, h->zG, nullptr, nullptr, h->opart, nullptr);
    sgk::k_octl<<<1, 32, 0, c.st>>>(sgk::OP_RZ0, nbo, h->opart, nullptr, h->octl, h->tol, h->max_iter, 0, 0, 0,
                                    h->omirror);
    CKL();
    return SG_OK;
  }));
  return cond_node(h, cx, hw, true, h->omirror, [&](Ctx& c) -> int {
    RET(enq_schur(h, c, h->pG, h->qG));
    sgk::k_odot<<<nbo, 256, 0, c.st>>>(n, h->pG, h->qG, nullptr, nullptr, h->opart, nullptr);
    sgk::k_octl<<<1, 32, 0, c.st>>>(sgk::OP_ALPHA, nbo, h->opart, nullptr, h->octl, h->tol, h->max_iter, 0, 0, 0,
                                    h->omirror);
    if (flex) CK(cudaMemcpyAsync(h->roG, h->rG, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.st));
    sgk::k_oupd<<<nbo, 256, 0, c.st>>>(n, h->octl, h->pG, h->qG, h->xG, h->rG, h->opart);
    if (h->a6_rec)  // W_I += alpha K_II^{-1}(-K_IG p), with the alpha that just updated x
      sgk::k_wacc<<<nblk(nl_all), 256, 0, c.st>>>(nl_all, h->pr.P, h->cls, h->octl, 0, h->wd, h->ws32.x, h->Wrec);
    cudaGraphConditionalHandle hif2;
    RET(make_handle(h, c, &hif2));
    sgk::k_octl<<<1, 32, 0, c.st>>>(sgk::OP_CHECK, nbo, h->opart, nullptr, h->octl, h->tol, h->max_iter, hw, hif2,
                                    c.capture ? 1 : 0, h->omirror);
    CKL();
    return cond_node(h, c, hif2, false, h->omirror + 1, [&](Ctx& c2) -> int {
      RET(enq_precond(h, c2, h->rG, h->zG));
      if (flex) {
        sgk::k_odot<<<nbo, 256, 0, c2.st>>>(n, h->rG, h->zG, h->roG, h->zG, h->opart, h->opart2);
        sgk::k_octl<<<1, 32, 0, c2.st>>>(sgk::OP_BETA_FLEX, nbo, h->opart, h->opart2, h->octl, h->tol, h->max_iter, 0,
                                         0, 0, h->omirror);
      } else {
        sgk::k_odot<<<nbo, 256, 0, c2.st>>>(n, h->rG, h->zG, nullptr, nullptr, h->opart, nullptr);
        sgk::k_octl<<<1, 32, 0, c2.st>>>(sgk::OP_BETA, nbo, h->opart, nullptr, h->octl, h->tol, h->max_iter, 0, 0, 0,
                                         h->omirror);
      }
      sgk::k_op<<<nbo, 256, 0, c2.st>>>(n, h->octl, h->zG, h->pG, 0);
      CKL();
      return SG_OK;
    });
  });
}

// ---------------------------------------------------------------------------------------------
// Learned warm start (extension): guess before the PCG, online training after it
// ---------------------------------------------------------------------------------------------
static int enq_warm_guess(sg_handle h, Ctx& cx) {
  const auto& pr = h->pr;
  cudaStream_t st = cx.st;
  const int nr = (int)h->nGd();
  sgk::k_scatter<double><<<nblk(nr), 256, 0, st>>>(pr.nG, pr.P, h->owners, pr.mo, h->Dw, h->V, h->vG, 1);
  sgk::k_scatter<double><<<nblk(nr), 256, 0, st>>>(pr.nG, pr.P, h->owners, pr.mo, h->Dw, h->A, h->aG, 1);
  sgk::k_wfeat<<<nblk(nr), 256, 0, st>>>(nr, pr.dt, h->xG, h->wE0, h->wE1, h->wE2, h->wE3, h->vG, h->aG, h->wX,
                                         h->wpred, h->wscale);
  sgk::k_mlp<false><<<(nr + sgk::NN_ROWS - 1) / sgk::NN_ROWS, sgk::NN_ROWS, 0, st>>>(nr, h->wX, nullptr, h->wctl.wb, h->wy,
                                                                                    nullptr, nullptr, nullptr);
  sgk::k_wguess<<<nblk(nr), 256, 0, st>>>(nr, h->wctl, h->wy, h->wpred, h->wscale, h->wE0, h->wE1, h->wE2, h->wE3,
                                          h->xG);
  CKL();
  return SG_OK;
}

static int enq_warm_train(sg_handle h, Ctx& cx) {
  cudaStream_t st = cx.st;
  const int nr = (int)h->nGd();
  const int nb = (nr + sgk::NN_ROWS - 1) / sgk::NN_ROWS;
  sgk::k_wstats<<<nblk(nr), 256, 0, st>>>(nr, h->wctl, h->xG, h->wpred, h->wscale, h->wy, h->wE0, h->wE1, h->wE2,
                                          h->wE3, h->wt);
  sgk::k_wsolve<<<1, 256, 0, st>>>((int)nblk(nr), h->wctl);
  for (int e = 0; e < h->warm_epochs; ++e) {
    sgk::k_mlp<true><<<nb, sgk::NN_ROWS, 0, st>>>(nr, h->wX, h->wt, h->wctl.wb, nullptr, h->wctl.part, h->wctl.loss_part,
                                                  h->wctl.train_left);
    sgk::k_mlp_adam<<<1, 256, 0, st>>>(nb, nr, h->wctl, h->warm_lr, h->wctl.train_left);
  }
  sgk::k_wdone<<<1, 32, 0, st>>>(h->wctl);
  sgk::k_wshift<<<nblk(nr), 256, 0, st>>>(nr, h->wE0, h->wE1, h->wE2, h->wE3, h->xG, h->wpred);
  CKL();
  return SG_OK;
}

// initial weights: SplitMix64 stream (seed 1), uniform in +-sqrt(6 / (fan_in + fan_out)); the output
// layer starts at 1/10 of that scale so the first guesses stay close to the predictor
static std::vector<float> warm_init_weights() {
  std::vector<float> th(sgk::NN_NP, 0.f);
  unsigned long long s = 1ULL;
  auto u01 = [&]() {
    s += 0x9E3779B97F4A7C15ULL;
    unsigned long long z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int off, int n, int fin, int fout, double scale) {
    const double a = scale * std::sqrt(6.0 / (fin + fout));
    for (int i = 0; i < n; ++i) th[off + i] = (float)((2.0 * u01() - 1.0) * a);
  };
  fill(sgk::NN_OW1, sgk::NN_H * sgk::NN_F, sgk::NN_F, sgk::NN_H, 1.0);
  fill(sgk::NN_OW2, sgk::NN_H * sgk::NN_H, sgk::NN_H, sgk::NN_H, 1.0);
  fill(sgk::NN_OW3, sgk::NN_H, sgk::NN_H, 1, 0.1);
  return th;
}

static int warm_setup(sg_handle h) {
  const int nr = (int)h->nGd();
  auto& wc = h->wctl;
  RET(dalloc(h, &wc.theta, sgk::NN_NP)); RET(dalloc(h, &wc.m, sgk::NN_NP)); RET(dalloc(h, &wc.v, sgk::NN_NP));
  RET(dalloc(h, &wc.wb, sgk::NN_NP));
  const int nb = std::max(1, (nr + sgk::NN_ROWS - 1) / sgk::NN_ROWS);
  RET(dalloc(h, &wc.part, (long long)nb * sgk::NN_NP)); RET(dalloc(h, &wc.loss_part, nb));
  RET(dalloc(h, &wc.loss, 1)); RET(dalloc(h, &wc.train_left, 1)); RET(dalloc(h, &wc.trained, 1));
  RET(dalloc(h, &wc.adam_it, 1));
  RET(dalloc(h, &wc.arw, 4)); RET(dalloc(h, &wc.use_net, 1));
  RET(dalloc(h, &wc.spart, (long long)nblk(nr) * sgk::WS_NSTAT));
  for (double** p : {&h->wE0, &h->wE1, &h->wE2, &h->wE3, &h->vG, &h->aG, &h->wpred, &h->wscale}) RET(dalloc(h, p, nr));
  RET(dalloc(h, &h->wX, 4LL * nr)); RET(dalloc(h, &h->wy, nr)); RET(dalloc(h, &h->wt, nr));
  const std::vector<float> th = warm_init_weights();
  CK(cudaMemcpyAsync(wc.theta, th.data(), sizeof(float) * th.size(), cudaMemcpyHostToDevice, h->st));
  sgk::k_to_bf16<<<nblk(sgk::NN_NP), 256, 0, h->st>>>(sgk::NN_NP, wc.theta, wc.wb);
  CK(cudaMemcpyAsync(wc.train_left, &h->warm_train, sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  CKL();
  return SG_OK;
}

// the predictor-error history starts empty (guesses are the plain predictor until it fills)
static int warm_reset_history(sg_handle h) {
  if (h->warm != SG_WARM_LEARNED) return SG_OK;
  const size_t nb = sizeof(double) * (size_t)h->nGd();
  for (double* e : {h->wE0, h->wE1, h->wE2, h->wE3}) CK(cudaMemsetAsync(e, 0, nb, h->st));
  CK(cudaMemsetAsync(h->wctl.arw, 0, 4 * sizeof(double), h->st));
  CK(cudaMemsetAsync(h->wctl.use_net, 0, sizeof(int), h->st));
  return SG_OK;
}

// One time step (a1 .. a7), enqueued on cx.
static int enq_step(sg_handle h, Ctx& cx, bool ext) {
  const auto& pr = h->pr;
  cudaStream_t st = cx.st;
  const long long n = h->nvec();
  const int nsub = pr.nsub, nl = pr.nl, P = pr.P;
  const double dt = pr.dt;
  const Op<double> op = h->op<double>();
  // a1: effective load f~ = M (u~_m + alpha0 u~_c) + alpha1 K u~_c + f
  sgk::k_newmark_pre<<<nblk(n), 256, 0, st>>>(n, dt, pr.alpha0, h->U, h->V, h->A, h->um, h->uc, h->xm);
  RET((launch_apply<double, double, false, false>(h, st, op, nsub, 1, h->xm, h->uc, h->ft, nullptr, 1.0, pr.alpha1,
                                                  sgk::MASK_FREE)));
  if (h->nload)
    sgk::k_point_load<<<nblk(h->nload), 256, 0, st>>>(h->nload, h->load_node, h->load_w, h->stepctr, dt, 1.0,
                                                       pr.src.freq, P, h->ft);
  if (ext)
    sgk::k_ext_load<<<nblk(h->nloc()), 256, 0, st>>>(h->nloc(), P, h->free_of_local, h->cls, h->gidx, h->Dw, h->fext,
                                                      h->ft);
  CKL();
  // a2: condensed RHS G = sum_s R_s^T (f~_G - K_GI K_II^{-1} f~_I)
  if (h->precision == SG_FP64) {
    sgk::k_conv_mask<double, double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->ft, h->wa, sgk::MASK_I, 1.0);
    RET(enq_inner<double>(h, cx, 0, nsub, 1, 0, h->wa));
    RET((launch_apply<double, double, false, false>(h, st, op, nsub, 1, h->ws.x, h->ws.x, h->wc, h->ft, -h->am, -h->bk,
                                                    sgk::MASK_G)));
  } else {
    const Op<float> o32 = h->op<float>();
    sgk::k_conv_mask<double, float><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->ft, h->fb, sgk::MASK_I, 1.0);
    RET(enq_inner<float>(h, cx, 0, nsub, 1, 0, h->fb));
    sgk::k_conv_mask<float, double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->ws32.x, h->wd, sgk::MASK_I, 1.0);
    // wa = f~ - K64 [w0; 0] (all free rows): interior part is the residual of the first solve
    RET((launch_apply<double, double, false, false>(h, st, op, nsub, 1, h->wd, h->wd, h->wa, h->ft, -h->am, -h->bk,
                                                    sgk::MASK_FREE)));
    sgk::k_conv_mask<double, float><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->wa, h->fb, sgk::MASK_I, 1.0);
    RET(enq_inner<float>(h, cx, 0, nsub, 1, 0, h->fb));
    // g_s = f~_G - K_GI (w0 + e) = wa_G - (K32 [e; 0])_G
    RET((launch_apply<float, double, false, false>(h, st, o32, nsub, 1, h->ws32.x, h->ws32.x, h->wc, h->wa, -h->am,
                                                   -h->bk, sgk::MASK_G)));
    // interior accumulator: W_I = K_II^{-1} f~_I = w0 + e
    if (h->a6_rec)
      sgk::k_wacc<<<nblk(n), 256, 0, st>>>(n, P, h->cls, nullptr, 1, h->wd, h->ws32.x, h->Wrec);
  }
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, pr.mo, h->Dw, h->wc, h->gG, 0);
  CKL();
  // a3: initial guess -- previous solution in xG (Alg. 1), or the learned predictor
  if (h->warm == SG_WARM_LEARNED) RET(enq_warm_guess(h, cx));
  // a4-a5: PCG on the interface
  RET(enq_outer(h, cx));
  sgk::k_record<<<1, 32, 0, st>>>(h->octl, h->stepctr, REC_CAP, h->rec_iters, h->rec_rel, h->rec_flags);
  if (h->warm == SG_WARM_LEARNED) RET(enq_warm_train(h, cx));
  // a6: interior recovery u_I = K_II^{-1} (f~_I - K_IG u_G)
  sgk::k_gather<double><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->gidx, h->Dw, h->xG, h->wa, sgk::MASK_G, 0);
  if (!h->a6_rec)
    RET((launch_apply<double, double, false, false>(h, st, op, nsub, 1, h->wa, h->wa, h->wb, h->ft, -h->am, -h->bk,
                                                    sgk::MASK_I)));
  if (h->precision == SG_FP64) {
    RET(enq_inner<double>(h, cx, 0, nsub, 1, 0, h->wb));
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->ws.x, 1.0, h->wa, h->Unew);
  } else if (h->a6_rec) {
    // u = [W_I; u_G]: the interior part was accumulated along the PCG (k_wacc)
    sgk::k_axpby<double><<<nblk(n), 256, 0, st>>>(n, 1.0, h->Wrec, 1.0, h->wa, h->Unew);
  } else {
    sgk::k_conv_mask<double, float><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->wb, h->fb, sgk::MASK_I, 1.0);
    RET(enq_inner<float>(h, cx, 0, nsub, 1, 0, h->fb));
    sgk::k_add_conv<float><<<nblk(n), 256, 0, st>>>(n, h->ws32.x, h->wa, h->wc);   // v = [w0; u_G]
    RET((launch_apply<double, double, false, false>(h, st, op, nsub, 1, h->wc, h->wc, h->wb, h->ft, -h->am, -h->bk,
                                                    sgk::MASK_I)));                  // r_I = f~_I - (K v)_I
    sgk::k_conv_mask<double, float><<<nblk(n), 256, 0, st>>>(nsub, 1, nl, P, h->cls, h->wb, h->fb, sgk::MASK_I, 1.0);
    RET(enq_inner<float>(h, cx, 0, nsub, 1, 0, h->fb));
    sgk::k_add_conv<float><<<nblk(n), 256, 0, st>>>(n, h->ws32.x, h->wc, h->Unew);
  }
  // a7: Newmark update
  sgk::k_newmark_post<<<nblk(n), 256, 0, st>>>(n, dt, h->Unew, h->um, h->U, h->V, h->A);
  CKL();
  return SG_OK;
}

static int build_graph(sg_handle h, int which) {
  if (h->gexec[which]) return SG_OK;
  Ctx cx{h->cs[0], 0, true};
  CK(cudaStreamBeginCapture(cx.st, cudaStreamCaptureModeThreadLocal));
  int rc = enq_step(h, cx, which == 1);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cx.st, &g);
  if (rc != SG_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) { h->err = std::string("step capture: ") + cudaGetErrorString(e); return SG_ECUDA; }
  h->graph[which] = g;
  CK(cudaGraphInstantiate(&h->gexec[which], g, 0));
  return SG_OK;
}

// ---------------------------------------------------------------------------------------------
// Set-up pieces
// ---------------------------------------------------------------------------------------------
// Mean operator stencils and line factorisation for both patterns (FP64, plus FP32 copies).
static int build_line_factors(sg_handle h) {
  const auto& pr = h->pr;
  const int L = pr.L, nl = pr.nl, nsub = pr.nsub, H = pr.H, PI = pr.PI;
  const double mh = pr.h * pr.h / 24.0;
  const int npat = h->pc == SG_PC_NN1 ? 3 : 2;
  for (int pat = 0; pat < npat; ++pat) {
    std::vector<double> Dd((size_t)nsub * L * L, 0.0), Du((size_t)nsub * L * L, 0.0);
    std::vector<double> Bd((size_t)nsub * L * L, 0.0), Bu((size_t)nsub * L * L, 0.0);
    for (int s = 0; s < nsub; ++s) {
      auto freep = [&](int li, int lj) {
        if (li < 0 || lj < 0 || li > H || lj > H) return false;
        int c = pr.cls[(size_t)s * nl + lj * L + li];
        if (pat == 0) return c == sgh::INTERIOR;
        if (pat == 1) return c == sgh::INTERIOR || c == sgh::REMAINING;
        return c != sgh::DIRICHLET;
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
          if (freep(li + 1, lj)) Du[o] = h->am * mh * (cellp(li, lj - 1) + cellp(li, lj)) - h->bk * kapE0(li, lj);
          if (freep(li, lj + 1)) Bd[o] = h->am * mh * (cellp(li - 1, lj) + cellp(li, lj)) - h->bk * kapN0(li, lj);
          if (freep(li + 1, lj + 1)) Bu[o] = h->am * mh * 2.0 * cellp(li, lj);
        }
    }
    double *dDd, *dDu;
    RET(upload(h, &dDd, Dd)); RET(upload(h, &dDu, Du));
    RET(upload(h, &h->lf[pat].Bd, Bd)); RET(upload(h, &h->lf[pat].Bu, Bu));
    const long long ns = (long long)nsub * L * L * L;
    RET(dalloc(h, &h->lf[pat].Sinv, ns));
    int* dstat;
    RET(dalloc(h, &dstat, nsub));
    const size_t sm = sizeof(double) * ((size_t)L * L + 2 * L);
    if (sm > 48 * 1024) CK(cudaFuncSetAttribute(sgk::k_line_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    sgk::k_line_factor<<<nsub, 256, sm, h->st>>>(L, dDd, dDu, h->lf[pat].Bd, h->lf[pat].Bu, h->lf[pat].Sinv, dstat);
    CKL();
    // FP32 copies for the mixed-precision subdomain solves
    RET(dalloc(h, &h->lf32[pat].Sinv, ns));
    RET(dalloc(h, &h->lf32[pat].Bd, (long long)nsub * L * L));
    RET(dalloc(h, &h->lf32[pat].Bu, (long long)nsub * L * L));
    sgk::k_cvt<double, float><<<nblk(ns), 256, 0, h->st>>>(ns, h->lf[pat].Sinv, h->lf32[pat].Sinv);
    {
      // rows padded to pad4(L) values: the staged FP32 team kernel and the register-tiled kernel
      // (FP32 and FP64 copies) read 16-byte pieces
      const long long nrows = (long long)nsub * L * L;
      RET(dalloc(h, &h->lf32[pat].Spad, nrows * pad4(L)));
      sgk::k_pad_factor<float><<<nblk(nrows * pad4(L)), 256, 0, h->st>>>(nrows, L, pad4(L), h->lf[pat].Sinv,
                                                                        h->lf32[pat].Spad);
      if (L >= WIDE_LMIN) {
        RET(dalloc(h, &h->lf[pat].Spad, nrows * pad4(L)));
        sgk::k_pad_factor<double><<<nblk(nrows * pad4(L)), 256, 0, h->st>>>(nrows, L, pad4(L), h->lf[pat].Sinv,
                                                                           h->lf[pat].Spad);
      }
    }
    sgk::k_cvt<double, float><<<nblk((long long)nsub * L * L), 256, 0, h->st>>>((long long)nsub * L * L, h->lf[pat].Bd,
                                                                               h->lf32[pat].Bd);
    sgk::k_cvt<double, float><<<nblk((long long)nsub * L * L), 256, 0, h->st>>>((long long)nsub * L * L, h->lf[pat].Bu,
                                                                               h->lf32[pat].Bu);
    CKL();
    std::vector<int> stat(nsub);
    CK(cudaMemcpyAsync(stat.data(), dstat, sizeof(int) * nsub, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int s = 0; s < nsub; ++s)
      if (stat[s]) { h->err = "mean operator not positive definite"; return SG_ENUMERIC; }
  }
  return SG_OK;
}

// Tensor-core mean preconditioner (mixed precision): A0^{-1} of both patterns in BF16 and its TMA
// map.  Used when the subdomains have at most MMA_LMAX nodes per side and P <= 32; larger subdomains
// keep the line-sweep preconditioner (a dense inverse would grow as L^4).
constexpr int MMA_LMAX = 40;
static bool mma_applies(const sgh::Problem& pr) { return pr.L <= MMA_LMAX && pr.P <= 32; }
static bool mma_eligible(const sgh::Problem& pr, int precision) {
  return (precision == SG_MIXED || precision == SG_BF16) && mma_applies(pr) && !std::getenv("SG_NO_MMA");
}

static int build_mma_precond(sg_handle h) {
  const auto& pr = h->pr;
  if (!mma_eligible(pr, h->policy)) return SG_OK;
  const int L = pr.L, LL = L * L;
  h->Kp = (LL + sgk::MMA_M - 1) / sgk::MMA_M * sgk::MMA_M;
  h->NC = h->Kp / sgk::MMA_KC;
  h->MT = h->Kp / sgk::MMA_M;
  h->mma_nb = pr.P <= 16 ? 16 : 32;
  const long long per = (long long)pr.nsub * h->Kp * h->Kp;
  RET(dalloc(h, &h->ainv, 2 * per));
  const size_t sm = sizeof(double) * ((size_t)sgk::INV_CB * LL + sgk::INV_CB * 64);
  RET(smem_attr(h, sgk::k_inv_cols, (int)sm));
  const int ngrp = (LL + sgk::INV_CB - 1) / sgk::INV_CB;
  for (int pat = 0; pat < 2; ++pat) {
    const int mask = pat == 0 ? sgk::MASK_I : sgk::MASK_N;
    sgk::k_inv_cols<<<(unsigned)(pr.nsub * ngrp), dim3(64, sgk::INV_CB), sm, h->st>>>(
        L, pr.nl, h->Kp, mask, h->cls, h->lf[pat].Sinv, h->lf[pat].Bd, h->lf[pat].Bu, h->ainv + pat * per);
    CKL();
  }
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  cudaDriverEntryPointQueryResult qr;
  CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&enc, 12000, cudaEnableDefault, &qr));
  if (!enc || qr != cudaDriverEntryPointSuccess) {
    h->err = "cuTensorMapEncodeTiled is not available from the driver";
    return SG_ECUDA;
  }
  // rows [pattern][subdomain][Kp] x Kp BF16 columns; 64 x 128 boxes with the 128-byte swizzle
  const cuuint64_t dims[2] = {(cuuint64_t)h->Kp, (cuuint64_t)(2LL * pr.nsub * h->Kp)};
  const cuuint64_t strides[1] = {(cuuint64_t)h->Kp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)sgk::MMA_KC, (cuuint32_t)sgk::MMA_M};
  const cuuint32_t es[2] = {1, 1};
  const CUresult cr = enc(&h->tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, h->ainv, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    h->err = "tensor map encoding of the mean-operator inverse failed";
    return SG_ECUDA;
  }
  RET(smem_attr(h, sgk::k_pre_mma<32>, sgk::PreShape<32, 2>::SMEM));
  RET(smem_attr(h, sgk::k_pre_mma<16>, sgk::PreShape<16, 2>::SMEM));
  h->mma = true;
  RET(ensure_bimg(h, pr.nsub));
  return ensure_ctl(h, pr.nsub, pr.L, std::max(pr.P, h->MT));
}

// BF16 images of the line factors (patterns 0 and 1) and their TMA maps for k_line_tc: rows
// (subdomain, line, a) of 64 BF16 columns, boxes of 64 x L with the 128-byte swizzle.
static int build_line_tc(sg_handle h) {
  const auto& pr = h->pr;
  if (!line_tc_eligible(pr, h->policy)) return SG_OK;
  const int L = pr.L;
  const long long nmat = (long long)pr.nsub * L;
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  cudaDriverEntryPointQueryResult qr;
  CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&enc, 12000, cudaEnableDefault, &qr));
  if (!enc || qr != cudaDriverEntryPointSuccess) {
    h->err = "cuTensorMapEncodeTiled is not available from the driver";
    return SG_ECUDA;
  }
  for (int pat = 0; pat < 2; ++pat) {
    RET(dalloc(h, &h->limg[pat], nmat * L * 64));
    RET(dalloc(h, &h->lcol[pat], nmat * sgk::LTC_COLN));
    sgk::k_line_img<<<nblk(nmat * L * 64), 256, 0, h->st>>>(nmat, L, h->lf[pat].Sinv, h->limg[pat], h->lcol[pat]);
    CKL();
    const cuuint64_t dims[2] = {64, (cuuint64_t)(nmat * L)};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {64, (cuuint32_t)L};
    const cuuint32_t es[2] = {1, 1};
    const CUresult cr = enc(&h->tmL[pat], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, h->limg[pat], dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
      h->err = "tensor map encoding of the line-factor image failed";
      return SG_ECUDA;
    }
  }
  const int lim = (int)sgk::ltc_smem(L, 32, 32);
  RET(smem_attr(h, sgk::k_line_tc<16>, lim));
  RET(smem_attr(h, sgk::k_line_tc<32>, lim));
  h->line_tc = true;
  return SG_OK;
}

// Coarse basis Phi_s = -S_rr^{-1} S_rc (per local corner dof) and F_cc (Eq. Fcc_2), from one
// Neumann solve per local corner dof: v = -N^{-1} K_[ir],c e, F^s e = (K~ (v + e))_c.  The right-hand
// sides and F^s are formed in FP64; the Neumann solves run in T (FP64 in FP64 mode, FP32 in mixed
// mode, where the coarse space only enters the preconditioner).  The batched-solve workspace is
// set-up scratch and is released afterwards.
template <typename T>
static int build_coarse_t(sg_handle h) {
  const auto& pr = h->pr;
  const int P = pr.P, nl = pr.nl, nsub = pr.nsub;
  const int R = h->Rc;
  const int chunk = std::max(1, std::min(nsub, 1024 / R));
  const long long len = (long long)nl * P;
  RET(ensure_ws<T>(h, chunk * R));
  double *e, *rhs, *ve, *y, *Fs;
  T* rhsT = nullptr;
  RET(dalloc(h, &e, len * chunk * R));
  RET(dalloc(h, &rhs, len * chunk * R));
  RET(dalloc(h, &ve, len * chunk * R));
  RET(dalloc(h, &y, len * chunk * R));
  RET(dalloc(h, &Fs, (long long)nsub * R * R));
  if (sizeof(T) != 8) RET(dalloc(h, &rhsT, len * chunk * R));
  Ctx cx{h->st, 0, false};
  cudaStream_t st = h->st;
  for (int s0 = 0; s0 < nsub; s0 += chunk) {
    const int ns = std::min(chunk, nsub - s0);
    const int nb = ns * R;
    const long long n = len * nb;
    const Op<double> op = h->op<double>(s0);
    CK(cudaMemsetAsync(e, 0, sizeof(double) * n, st));
    sgk::k_coarse_units<<<nblk((long long)nb), 256, 0, st>>>(ns, R, nl, P, s0, h->loc_corner, pr.mc, h->n_loc_corner, e);
    RET((launch_apply<double, double, false, false>(h, st, op, nb, R, e, e, rhs, nullptr, -h->am, -h->bk, sgk::MASK_N)));
    const T* rhs_in = reinterpret_cast<const T*>(rhs);
    if (sizeof(T) != 8) {
      sgk::k_cvt<double, float><<<nblk(n), 256, 0, st>>>(n, rhs, reinterpret_cast<float*>(rhsT));
      rhs_in = rhsT;
    }
    RET(enq_inner<T>(h, cx, 1, nb, R, s0, rhs_in));
    const T* v = wsT<T>(h).x;
    sgk::k_coarse_phi<T><<<nblk((long long)nb * pr.nGam * P), 256, 0, st>>>(ns, s0, R, nl, P, pr.nGam, h->cls,
                                                                            h->gam_ln, h->n_gam, v, h->Phi);
    sgk::k_add_conv<T><<<nblk(n), 256, 0, st>>>(n, v, e, ve);
    RET((launch_apply<double, double, false, false>(h, st, op, nb, R, ve, ve, y, nullptr, h->am, h->bk, sgk::MASK_C)));
    sgk::k_coarse_fs<<<nblk((long long)nb * R), 256, 0, st>>>(ns, s0, R, nl, P, h->loc_corner, pr.mc, h->n_loc_corner, y, Fs);
    CKL();
  }
  std::vector<double> hFs((size_t)nsub * R * R);
  CK(cudaMemcpyAsync(hFs.data(), Fs, sizeof(double) * hFs.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  dfree(h, &e); dfree(h, &rhs); dfree(h, &ve); dfree(h, &y); dfree(h, &Fs);
  if (rhsT) dfree(h, &rhsT);
  // shrink the batched workspace back to one problem per subdomain
  auto& w = wsT<T>(h);
  dfree(h, &w.x); dfree(h, &w.r); dfree(h, &w.z); dfree(h, &w.p0); dfree(h, &w.p1); dfree(h, &w.q);
  w.cap_nb = 0;
  RET(ensure_ws<T>(h, nsub));
  const int nCd = h->nCd;
  std::vector<double> F((size_t)nCd * nCd, 0.0);
  for (int s = 0; s < nsub; ++s) {
    const int nc = pr.n_loc_corner[s];
    for (int a = 0; a < nc; ++a) {
      const int ga = pr.cidx[(size_t)s * nl + pr.loc_corner[s * pr.mc + a]];
      for (int b = 0; b < nc; ++b) {
        const int gb = pr.cidx[(size_t)s * nl + pr.loc_corner[s * pr.mc + b]];
        for (int m = 0; m < P; ++m)
          for (int q = 0; q < P; ++q)
            F[(size_t)(ga * P + m) * nCd + gb * P + q] += hFs[((size_t)s * R + a * P + m) * R + b * P + q];
      }
    }
  }
  for (int i = 0; i < nCd; ++i)
    for (int j = 0; j < i; ++j) {
      double v = 0.5 * (F[(size_t)i * nCd + j] + F[(size_t)j * nCd + i]);
      F[(size_t)i * nCd + j] = F[(size_t)j * nCd + i] = v;
    }
  if (!sgh::spd_inverse(F, nCd)) { h->err = "coarse matrix F_cc not positive definite"; return SG_ENUMERIC; }
  RET(upload(h, &h->Finv, F));
  return SG_OK;
}

static int build_coarse(sg_handle h) {
  const auto& pr = h->pr;
  h->Rc = pr.max_corner * pr.P;
  h->nCd = pr.nC * pr.P;
  RET(dalloc(h, &h->Phi, (long long)pr.nsub * std::max(h->Rc, 1) * pr.nGam * pr.P));
  RET(dalloc(h, &h->dC, std::max(h->nCd, 1)));
  RET(dalloc(h, &h->uC, std::max(h->nCd, 1)));
  if (pr.nC == 0 || h->Rc == 0) return SG_OK;
  return h->precision == SG_FP64 ? build_coarse_t<double>(h) : build_coarse_t<float>(h);
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
  const Op<double> op = h->op<double>();
  {
    std::vector<double> U0((size_t)n, 0.0);
    for (long long i = 0; i < h->nloc(); ++i) U0[(size_t)i * P] = pr.u0_local[(size_t)i];
    CK(cudaMemcpyAsync(h->U, U0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemsetAsync(h->V, 0, sizeof(double) * n, st));
  RET((launch_apply<double, double, false, false>(h, st, op, pr.nsub, 1, h->U, h->U, h->wa, nullptr, 0.0, -1.0,
                                                  sgk::MASK_FREE)));
  if (h->nload)
    sgk::k_point_load<<<nblk(h->nload), 256, 0, st>>>(h->nload, h->load_node, h->load_w, nullptr, pr.dt, 0.0,
                                                       pr.src.freq, P, h->wa);
  sgk::k_assemble_gamma<<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, pr.mo, h->wa);
  CK(cudaMemsetAsync(h->A, 0, sizeof(double) * n, st));
  double rr, rr0, pq;
  RET(ldot_w(h, h->wa, h->wa, &rr));
  rr0 = rr;
  CK(cudaMemcpyAsync(h->wb, h->wa, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  for (int it = 0; it < 500 && rr > 1e-30 * rr0 && rr0 > 0.0; ++it) {
    RET((launch_apply<double, double, false, false>(h, st, op, pr.nsub, 1, h->wb, h->wb, h->wc, nullptr, 1.0, 0.0,
                                                    sgk::MASK_FREE)));
    sgk::k_assemble_gamma<<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, pr.mo, h->wc);
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
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, st>>>(pr.nG, P, h->owners, pr.mo, h->Dw, h->U, h->xG, 1);
  CKL();
  return SG_OK;
}

// Run nsteps steps (graph launches, or eager enqueue when SG_EAGER is set).
static int run_steps(sg_handle h, int nsteps, const double* f_host, double* u_host, int* rc_out) {
  const auto& pr = h->pr;
  const bool ext = f_host != nullptr;
  if (!h->eager) RET(build_graph(h, ext ? 1 : 0));
  CK(cudaMemsetAsync(h->rec_flags, 0, sizeof(int), h->st));
  long long first = h->step;
  for (int s = 0; s < nsteps; ++s) {
    if (ext)
      CK(cudaMemcpyAsync(h->fext, f_host + (size_t)s * pr.n_free, sizeof(double) * pr.n_free, cudaMemcpyHostToDevice,
                         h->st));
    if (h->eager) {
      Ctx cx{h->st, 0, false};
      RET(enq_step(h, cx, ext));
    } else {
      CK(cudaGraphLaunch(h->gexec[ext ? 1 : 0], h->st));
    }
    if (u_host) {
      sgk::k_gather_free<<<nblk(pr.n_free), 256, 0, h->st>>>(pr.n_free, pr.P, 0, h->free_owner, h->U, h->outbuf);
      CKL();
      CK(cudaMemcpyAsync(u_host + (size_t)s * pr.n_free, h->outbuf, sizeof(double) * pr.n_free, cudaMemcpyDeviceToHost,
                         h->st));
    }
    h->step += 1;
    // drain the per-step records before the ring buffer wraps
    if ((h->step - first) == REC_CAP || s == nsteps - 1) {
      const long long cnt = h->step - first;
      std::vector<int> it((size_t)cnt);
      std::vector<double> rl((size_t)cnt);
      const long long s0 = first % REC_CAP;
      for (long long i = 0; i < cnt; ++i) {
        CK(cudaMemcpyAsync(&it[i], h->rec_iters + (s0 + i) % REC_CAP, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(&rl[i], h->rec_rel + (s0 + i) % REC_CAP, sizeof(double), cudaMemcpyDeviceToHost, h->st));
      }
      CK(cudaStreamSynchronize(h->st));
      h->iters.insert(h->iters.end(), it.begin(), it.end());
      h->relres.insert(h->relres.end(), rl.begin(), rl.end());
      first = h->step;
    }
  }
  CK(cudaMemcpyAsync(h->hint, h->rec_flags, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->hint + 1, h->ctl.breakdown, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  *rc_out = SG_OK;
  if (h->hint[0] & 1) *rc_out = SG_ENOTCONV;
  if ((h->hint[0] & 2) || h->hint[1]) { h->err = "numerical breakdown in PCG"; *rc_out = SG_ENUMERIC; }
  if (h->hint[1] >= 16) {
    h->err = "a bounded wait of the tensor-core preconditioner expired (pipeline stage " +
             std::to_string(h->hint[1] - 16) + ")";
    *rc_out = SG_ETIMEOUT;
  }
  return SG_OK;
}

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
static void free_all(sg_handle h) {
  for (int w = 0; w < 2; ++w) {
    if (h->gexec[w]) cudaGraphExecDestroy(h->gexec[w]);
    if (h->graph[w]) cudaGraphDestroy(h->graph[w]);
  }
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  for (int i = 0; i < NSTREAMS; ++i)
    if (h->cs[i]) cudaStreamDestroy(h->cs[i]);
  if (h->hscal) cudaFreeHost(h->hscal);
  if (h->hint) cudaFreeHost(h->hint);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->kev0) cudaEventDestroy(h->kev0);
  if (h->kev1) cudaEventDestroy(h->kev1);
  if (h->own_st && h->st) cudaStreamDestroy(h->st);
}

// Autotuner: times the candidate tile shapes of the two hot kernels of the inner solve on this
// handle's own workspace (results discarded) and records the fastest per problem shape.  Candidates:
// fused apply with 1, 2, 4 or 8 grid lines per block (shared memory permitting); line solve with
// 1..gmax modes per block (warp-team kernel) or 1, 2, 4, 8 (block kernel).
template <typename T>
static int autotune_t(sg_handle h, int nb) {
  const auto& pr = h->pr;
  cudaStream_t st = h->st;
  auto& w = wsT<T>(h);
  const Op<T> op = h->op<T>();
  auto time_it = [&](auto&& launch, float* best_ms) -> int {
    for (int i = 0; i < 2; ++i) launch();
    CK(cudaEventRecord(h->kev0, st));
    for (int i = 0; i < 6; ++i) launch();
    CK(cudaEventRecord(h->kev1, st));
    CK(cudaEventSynchronize(h->kev1));
    CKL();
    CK(cudaEventElapsedTime(best_ms, h->kev0, h->kev1));
    return SG_OK;
  };
  // apply: lines per block
  {
    const TuneKey key{0, (int)sizeof(T), pr.L, pr.P, pr.PI, (int)pr.gk_v.size(), nb};
    if (!g_tune.count(key)) {
      int best_t = 0;
      float best = 1e30f;
      for (int t : {1, 2, 4, 8}) {
        if (t > pr.L) continue;
        g_tune[key] = t;
        int TL, NT, stage;
        size_t sm;
        apply_cfg<T>(pr, nb, &TL, &NT, &sm, &stage);
        if (TL != t || sm > SMEM_TILE) continue;
        float ms = 0.f;
        auto launch_ap = [&]() {
          launch_apply<T, T, true, true>(h, st, op, nb, 1, nullptr, nullptr, w.q, nullptr, h->am, h->bk, sgk::MASK_N,
                                         w.p0, w.p1, w.z);
        };
        RET(time_it(launch_ap, &ms));
        if (ms < best) { best = ms; best_t = t; }
      }
      if (best_t) g_tune[key] = best_t;
      else g_tune.erase(key);
    }
  }
  // line solve: modes per block
  {
    const TuneKey key{1, (int)sizeof(T), pr.L, pr.P, pr.PI, (int)pr.gk_v.size(), nb};
    if (!g_tune.count(key)) {
      const int L = pr.L;
      const long long pstride = (long long)L * L * L;
      const auto& lf = lfT<T>(h, 1);
      const long long pstride_pad = (long long)L * L * pad4(L);
      int best_g = 0;
      float best = 1e30f;
      std::vector<int> cands;
      g_tune.erase(key);
      if (line_cfg<T>(pr, nb).wide) {
        // register-tiled kernel: whole mode groups of 1 .. 4 blocks per problem
        for (int ng = 1; ng <= std::min(4, pr.P); ++ng) cands.push_back((pr.P + ng - 1) / ng);
      } else {
        for (int g = 1; g <= std::min(pr.P, 15); ++g) cands.push_back(g);
      }
      for (int g : cands) {
        g_tune[key] = g;
        const LineCfg lc = line_cfg<T>(pr, nb);
        if (!lc.wide && lc.G != g && !(lc.team && lc.G == (pr.P + lc.NG - 1) / lc.NG && lc.G <= g)) continue;
        int TL, NT, stage;
        size_t sm;
        apply_cfg<T>(pr, nb, &TL, &NT, &sm, &stage);
        const unsigned lg = (unsigned)nb * lc.NG;
        float ms = 0.f;
        auto launch_line = [&]() {
          if (lc.team) {
#define SG_TEAM_T(LSV)                                                                                           \
  case LSV:                                                                                                      \
    sgk::k_line_team<T, LSV><<<lg, lc.block, lc.smem, st>>>(L, pr.nl, pr.P, 1, lc.NG, NT, lc.G, pstride_pad,     \
                                                            lf.Spad, lf.Bd, lf.Bu, nb, w.x, w.r, w.z, w.p0, w.p1, \
                                                            w.q, h->ctl, 1, 1e-30, 1e300, 1, 0, 0);              \
    break;
            switch (pad4(L)) {
              SG_TEAM_T(4) SG_TEAM_T(8) SG_TEAM_T(12) SG_TEAM_T(16) SG_TEAM_T(20) SG_TEAM_T(24) SG_TEAM_T(28)
              SG_TEAM_T(32) SG_TEAM_T(36) SG_TEAM_T(40)
              default: break;
            }
#undef SG_TEAM_T
          } else if (lc.wide) {
            sgk::k_line_w<T><<<lg, lc.block, lc.smem, st>>>(L, pad4(L), pr.nl, pr.P, 1, lc.NG, NT, lc.G, lc.GS,
                                                            pstride_pad, lf.Spad, lf.Bd, lf.Bu, nb, w.x, w.r, w.z,
                                                            w.p0, w.p1, w.q, h->ctl, 1, 1e-30, 1e300, 1, 0, 0);
          } else if (lc.gs) {
            sgk::k_line<T, true><<<lg, lc.block, lc.smem, st>>>(L, pr.nl, pr.P, 1, lc.NG, NT, pstride, lf.Sinv, lf.Bd,
                                                                lf.Bu, nb, w.x, w.r, w.z, w.p0, w.p1, w.q, h->ctl, 1,
                                                                1e-30, 1e300, 1, 0, 0);
          } else {
            sgk::k_line<T><<<lg, lc.block, lc.smem, st>>>(L, pr.nl, pr.P, 1, lc.NG, NT, pstride, lf.Sinv, lf.Bd, lf.Bu,
                                                          nb, w.x, w.r, w.z, w.p0, w.p1, w.q, h->ctl, 1, 1e-30, 1e300,
                                                          1, 0, 0);
          }
        };
        RET(time_it(launch_line, &ms));
        if (ms < best) { best = ms; best_g = g; }
      }
      if (best_g) g_tune[key] = best_g;
      else g_tune.erase(key);
    }
  }
  return SG_OK;
}

static int autotune(sg_handle h) {
  RET(autotune_t<float>(h, h->pr.nsub));
  if (h->precision == SG_FP64) RET(autotune_t<double>(h, h->pr.nsub));
  return SG_OK;
}

// Compiled triple-product table matching the problem's PCE sizes, or -1 (SG_NO_GFIX forces -1).
static int select_gfix(const sgh::Problem& pr) {
  int id = -1;
  for (int i = 0; i < sgk::gfix::NCFG && id < 0; ++i)
    if (with_gfix(i, false, [&](auto c) { return gfix_matches<decltype(c)>(pr); })) id = i;
  return std::getenv("SG_NO_GFIX") ? -1 : id;
}

// Whether the per-step kernels of a precision fit their shared-memory limits at this subdomain size
// (the FP64 apply always runs; the line kernel and the FP32 apply of the precision in use).
static bool tiles_fit(const sgh::Problem& pr, int precision) {
  auto fits_apply = [&](auto tag) {
    using T = decltype(tag);
    int TL, NT, stage, nods;
    size_t sm;
    apply_cfg<T>(pr, pr.nsub, &TL, &NT, &sm, &stage, &nods);
    return sm <= (nods == 2 ? SMEM_MAX : SMEM_TILE);
  };
  auto fits_line = [&](auto tag) {
    using T = decltype(tag);
    const LineCfg lc = line_cfg<T>(pr, pr.nsub);
    return lc.smem <= (lc.team ? SMEM_MAX : SMEM_TILE);
  };
  return fits_apply(double{}) &&
         (precision != SG_FP64 ? (fits_apply(float{}) && fits_line(float{})) : fits_line(double{}));
}

// Problem construction and the size limits shared by sg_setup and sg_plan_query.
static int build_checked(sgh::Problem& pr, std::string& err, const sg_grid* grid, const sg_kl* kl,
                         const sg_pce* pce, const sg_params* prm, const sgh::SourceDesc& sd) {
  if (prm->precision < SG_FP64 || prm->precision > SG_BF16) { err = "precision"; return SG_EINVAL; }
  if (prm->precond < SG_PC_NN2 || prm->precond > SG_PC_LUMPED) { err = "precond"; return SG_EINVAL; }
  std::string msg = sgh::build_problem(pr, grid->N, grid->nsub_x, grid->nsub_y, kl->M, kl->sigma, kl->bx,
                                       kl->by, kl->g0, pce->p, pce->p_in, prm->dt, prm->alpha0, prm->alpha1, sd,
                                       kl->modes, kl->modes ? kl->lambdas : nullptr);
  if (!msg.empty()) { err = msg; return SG_EINVAL; }
  if (pr.L > 256 || pr.L * 2 > 1024) { err = "subdomains wider than 255 cells are not supported"; return SG_ENOTSUP; }
  if (pr.nsub < 2) { err = "at least 2 x 2 subdomains are required"; return SG_ENOTSUP; }
  pr.gfix = select_gfix(pr);
  if (prm->precision == SG_BF16 && !mma_applies(pr) && !line_tc_eligible(pr, SG_BF16)) {
    err = "SG_BF16: the BF16 tensor-core preconditioner needs subdomains of at most 40 x 40 nodes with P <= 32 "
          "(dense inverse) or 41 .. 65 nodes per side (line products)";
    return SG_ENOTSUP;
  }
  return SG_OK;
}

// Set-up pieces shared by the structured grid (sg_setup) and the general partitions (sg_setup_mesh).
static int check_source(sg_handle h, const sg_source* src, sgh::SourceDesc* out) {
  const sgh::SourceDesc sd{src ? src->kind : 0, src ? src->x0 : 0.5, src ? src->y0 : 0.5,
                     src ? src->width : 0.05, src ? src->freq : 10.0, src ? src->amp : 1.0};
  if (sd.kind < 0 || sd.kind > 2) { h->err = "source kind"; return SG_EINVAL; }
  if (sd.kind == 1 && !(sd.width > 0)) { h->err = "pulse width must be positive"; return SG_EINVAL; }
  if (sd.kind == 2 && (!(sd.freq > 0) || sd.x0 < 0 || sd.x0 > 1 || sd.y0 < 0 || sd.y0 > 1)) {
    h->err = "ricker source outside the unit square or non-positive frequency";
    return SG_EINVAL;
  }
  *out = sd;
  return SG_OK;
}

static int apply_params(sg_handle h, const sg_params* prm) {
  const auto& pr = h->pr;
  // the compute path: FP64, or FP32 subdomain solves inside the FP64 outer PCG (SG_MIXED, SG_FP32 and
  // SG_BF16 differ only in the mean-operator preconditioner, chosen in build_mma_precond)
  h->precision = prm->precision == SG_FP64 ? SG_FP64 : SG_MIXED;
  h->policy = prm->precision;
  h->pc = prm->precond;
  h->warm = prm->warm;
  h->tol = prm->tol > 0 ? prm->tol : 1e-8;
  h->max_iter = prm->max_iter > 0 ? prm->max_iter : 500;
  h->inner_tol = prm->inner_tol > 0 ? prm->inner_tol : 1e-14;
  // FP32 solves: a corrected Dirichlet solve is two FP32 solves (the second on the FP64 residual of
  // the first), so its accuracy is about the product of their tolerances; automatic choice: each
  // sqrt(0.1 tol), i.e. the product 10x below the outer tolerance, within [1e-6, 1e-4] (measured on
  // the 128^2 workload against 1e-2 tol and 1e-3 tol: 87.8 / 94.0 / 101.4 inner iterations per step,
  // the same 3 outer iterations)
  h->inner_tol32 = prm->inner_tol > 0 ? std::max(prm->inner_tol, 1e-7)
                                      : std::min(1e-4, std::max(1e-6, std::sqrt(0.1 * h->tol)));
  h->inner_max = prm->inner_max_iter > 0 ? prm->inner_max_iter : 400;
  h->eager = std::getenv("SG_EAGER") != nullptr;
  // measured on the 128^2 workload: 7.87 ms per step without, 7.96 with; opt-in only
  h->pdl = std::getenv("SG_PDL") != nullptr;
  if (prm->warm != SG_WARM_PREV && prm->warm != SG_WARM_LEARNED) { h->err = "warm"; return SG_EINVAL; }
  if (prm->warm_train_steps < 0 || prm->warm_lr < 0) { h->err = "warm-start training parameters"; return SG_EINVAL; }
  h->warm_train = prm->warm_train_steps > 0 ? prm->warm_train_steps : 20;
  h->warm_lr = prm->warm_lr > 0 ? (float)prm->warm_lr : 1e-3f;
  h->am = 1.0 / (ZETA * pr.dt * pr.dt) + pr.alpha0 * GAMMA / (ZETA * pr.dt);
  h->bk = 1.0 + pr.alpha1 * GAMMA / (ZETA * pr.dt);
  return SG_OK;
}

static int init_device(sg_handle h) {
  // first CUDA call: every argument check is above
  CK(cudaGetDevice(&h->dev));
  if (!h->st) {  // private stream when the caller passes none
    CK(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
    h->own_st = true;
  }
  for (int i = 0; i < NSTREAMS; ++i) CK(cudaStreamCreateWithFlags(&h->cs[i], cudaStreamNonBlocking));
  CK(cudaMallocHost(&h->hscal, sizeof(double) * 16));
  CK(cudaMallocHost(&h->hint, sizeof(int) * 16));
  CK(cudaEventCreate(&h->ev0));
  CK(cudaEventCreate(&h->ev1));
  CK(cudaEventCreate(&h->kev0));
  CK(cudaEventCreate(&h->kev1));
  // process-wide launch counter (device symbol read by every kernel)
  if (!g_nlaunch_dev) {
    CK(cudaMalloc(&g_nlaunch_dev, sizeof(unsigned long long)));
    CK(cudaMemset(g_nlaunch_dev, 0, sizeof(unsigned long long)));
    CK(cudaMemcpyToSymbol(sgk::g_nlaunch, &g_nlaunch_dev, sizeof(void*)));
  }
  h->nlaunch = g_nlaunch_dev;
  return SG_OK;
}

// triple products, interface / corner / output maps, point load, node weights and the step buffers
static int upload_common(sg_handle h) {
  const auto& pr = h->pr;
  RET(upload(h, &h->gk_ptr, pr.gk_ptr)); RET(upload(h, &h->gk_i, pr.gk_i)); RET(upload(h, &h->gk_j, pr.gk_j));
  {
    std::vector<unsigned> pk(pr.gk_i.size());
    for (size_t e = 0; e < pk.size(); ++e) pk[e] = (unsigned)pr.gk_i[e] | ((unsigned)pr.gk_j[e] << 16);
    RET(upload(h, &h->gk_pk, pk));
  }
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
  const long long n = h->nvec();
  for (double** p : {&h->U, &h->V, &h->A, &h->um, &h->uc, &h->xm, &h->ft, &h->Unew, &h->wa, &h->wb, &h->wc, &h->wd, &h->we})
    RET(dalloc(h, p, n));
  h->a6_rec = h->precision == SG_MIXED && std::getenv("SG_A6_SOLVE") == nullptr;
  if (h->a6_rec) RET(dalloc(h, &h->Wrec, n));
  RET(dalloc(h, &h->fa, n)); RET(dalloc(h, &h->fb, n));
  RET(dalloc(h, &h->fext, pr.n_free));
  RET(dalloc(h, &h->outbuf, 2LL * pr.n_free * pr.P));
  for (double** p : {&h->xG, &h->rG, &h->zG, &h->pG, &h->qG, &h->gG, &h->roG}) RET(dalloc(h, p, h->nGd()));
  RET(dalloc(h, &h->opart, NB_OUT)); RET(dalloc(h, &h->opart2, NB_OUT));
  RET(dalloc(h, &h->scal, 16));
  RET(dalloc(h, &h->octl, 1)); RET(dalloc(h, &h->omirror, 2));
  RET(dalloc(h, &h->stepctr, 1)); RET(dalloc(h, &h->rec_iters, REC_CAP)); RET(dalloc(h, &h->rec_rel, REC_CAP));
  RET(dalloc(h, &h->rec_flags, 1));
  RET(ensure_ws<double>(h, pr.nsub));
  RET(ensure_ws<float>(h, pr.nsub));
  CKL();
  return SG_OK;
}

// coarse space, warm start, initial state
static int finish_setup(sg_handle h) {
  if (h->pc == SG_PC_NN2) RET(build_coarse(h));  // the one-level preconditioners have no coarse space
  if (h->warm == SG_WARM_LEARNED) RET(warm_setup(h));
  RET(initial_state(h));
  RET(warm_reset_history(h));
  CK(cudaStreamSynchronize(h->st));
  return SG_OK;
}

static int setup_impl(sg_handle h, const sg_grid* grid, const sg_kl* kl, const sg_pce* pce,
                      const sg_params* prm, const sg_source* src) {
  sgh::SourceDesc sd;
  RET(check_source(h, src, &sd));
  RET(build_checked(h->pr, h->err, grid, kl, pce, prm, sd));
  auto& pr = h->pr;
  RET(apply_params(h, prm));
  RET(init_device(h));
  // shared-memory opt-in of the apply variants
  {
    const int lim = (int)SMEM_TILE;
    RET(smem_attr(h, sgk::k_apply<double, double, false, false>, lim));
    RET(smem_attr(h, sgk::k_apply<double, double, true, true>, lim));
    RET(smem_attr(h, sgk::k_apply<float, float, false, false>, lim));
    RET(smem_attr(h, sgk::k_apply<float, float, true, true>, lim));
    RET(smem_attr(h, sgk::k_apply<float, double, false, false>, lim));
    RET(smem_attr(h, sgk::k_line<double>, lim));
    RET(smem_attr(h, sgk::k_line<float>, lim));
    RET(smem_attr(h, sgk::k_line<double, true>, lim));
    RET(smem_attr(h, sgk::k_line<float, true>, lim));
    RET(smem_attr(h, sgk::k_line_w<double>, lim));
    RET(smem_attr(h, sgk::k_line_w<float>, lim));
    RET(smem_attr(h, sgk::k_apply<double, double, false, false, sgk::GDynNoDS>, lim));
    RET(smem_attr(h, sgk::k_apply<double, double, true, true, sgk::GDynNoDS>, lim));
    RET(smem_attr(h, sgk::k_apply<float, float, false, false, sgk::GDynNoDS>, lim));
    RET(smem_attr(h, sgk::k_apply<float, float, true, true, sgk::GDynNoDS>, lim));
    RET(smem_attr(h, sgk::k_apply<float, double, false, false, sgk::GDynNoDS>, lim));
    RET(smem_attr(h, sgk::k_apply<double, double, false, false, sgk::GDynNoDSG>, (int)SMEM_MAX));
    RET(smem_attr(h, sgk::k_apply<double, double, true, true, sgk::GDynNoDSG>, (int)SMEM_MAX));
    RET(smem_attr(h, sgk::k_apply<float, float, false, false, sgk::GDynNoDSG>, (int)SMEM_MAX));
    RET(smem_attr(h, sgk::k_apply<float, float, true, true, sgk::GDynNoDSG>, (int)SMEM_MAX));
    RET(smem_attr(h, sgk::k_apply<float, double, false, false, sgk::GDynNoDSG>, (int)SMEM_MAX));
#define SG_ATTR(LSV) \
  RET(smem_attr(h, sgk::k_line_team<float, LSV>, (int)SMEM_MAX));
    SG_ATTR(4) SG_ATTR(8) SG_ATTR(12) SG_ATTR(16) SG_ATTR(20) SG_ATTR(24) SG_ATTR(28) SG_ATTR(32) SG_ATTR(36) SG_ATTR(40)
#undef SG_ATTR
  }
  // compiled triple-product table for this PCE size (values into constant memory; the same
  // values for every handle of that size, so concurrent handles may share the slot)
  {
    if (pr.gfix >= 0) {
      const int rc = with_gfix(pr.gfix, (int)SG_EINVAL, [&](auto c) -> int {
        using C = decltype(c);
        std::vector<float> f(pr.gk_v.begin(), pr.gk_v.end());
        CK(cudaMemcpyToSymbol(sgk::c_gvf, f.data(), sizeof(float) * C::NNZ, sizeof(float) * C::OFF));
        CK(cudaMemcpyToSymbol(sgk::c_gvd, pr.gk_v.data(), sizeof(double) * C::NNZ, sizeof(double) * C::OFF));
        const int lim = (int)SMEM_TILE;
        RET(smem_attr(h, sgk::k_apply<float, float, false, false, C>, lim));
        RET(smem_attr(h, sgk::k_apply<float, float, true, true, C>, lim));
        RET(smem_attr(h, sgk::k_apply<float, double, false, false, C>, lim));
        if constexpr (gfix_fp64_ok<C>()) {
          RET(smem_attr(h, sgk::k_apply<double, double, false, false, C>, lim));
          RET(smem_attr(h, sgk::k_apply<double, double, true, true, C>, lim));
          RET(smem_attr(h, sgk::k_apply_f2<C>, lim));
        }
        // low parts of the float-float table: G - (double)(float)G
        std::vector<float> lo(C::NNZ);
        for (int e = 0; e < C::NNZ; ++e) lo[e] = (float)(pr.gk_v[e] - (double)f[e]);
        CK(cudaMemcpyToSymbol(sgk::c_gvf_lo, lo.data(), sizeof(float) * C::NNZ, sizeof(float) * C::OFF));
        return SG_OK;
      });
      RET(rc);
    }
  }
  // problem data (FP64 and FP32 copies of the operator coefficients)
  RET(upload(h, &h->cls, pr.cls)); RET(upload(h, &h->cells, pr.cells));
  RET(upload(h, &h->kapE, pr.kapE)); RET(upload(h, &h->kapN, pr.kapN));
  {
    std::vector<float> e32(pr.kapE.begin(), pr.kapE.end()), n32(pr.kapN.begin(), pr.kapN.end());
    std::vector<float> g32(pr.gk_v.begin(), pr.gk_v.end());
    RET(upload(h, &h->kapE32, e32)); RET(upload(h, &h->kapN32, n32)); RET(upload(h, &h->gk_v32, g32));
  }
  // The FP64 applies of the mixed-precision outer loop (effective load, residual corrections) in
  // float-float arithmetic: about 1e-13 relative, five orders below the smallest outer tolerance that
  // a mixed-precision solve reaches, at a fraction of the FP64 cost.  The FP64 path keeps FP64
  // arithmetic throughout; SG_APPLY_FP64 keeps it for the mixed path too.
  h->apply_f2 = h->precision == SG_MIXED && gfix_for<double>(pr) >= 0 && !std::getenv("SG_APPLY_FP64");
  if (h->apply_f2) {
    auto split = [](const std::vector<double>& v) {
      std::vector<float2> o(v.size());
      for (size_t i = 0; i < v.size(); ++i) {
        const float hi = (float)v[i];
        o[i] = make_float2(hi, (float)(v[i] - (double)hi));
      }
      return o;
    };
    RET(upload(h, &h->kapE2, split(pr.kapE))); RET(upload(h, &h->kapN2, split(pr.kapN)));
  }
  RET(upload_common(h));
  // shared-memory fit of the hot kernels at this subdomain size (per precision in use)
  if (!tiles_fit(pr, h->precision)) {
    h->err = "subdomain too large for the shared-memory tiles of this build (H = " + std::to_string(pr.H) + " cells)";
    return SG_ENOTSUP;
  }
  RET(build_line_factors(h));
  RET(build_mma_precond(h));
  RET(build_line_tc(h));
  if (prm->autotune) RET(autotune(h));
  return finish_setup(h);
}

// BF16 image of the mesh's mean-operator inverses (patterns 0 and 1, rows padded to Kp = nl rounded up to
// the 128-row tile) and its tensor map, as build_mma_precond lays out the grid's.
constexpr int MESH_MMA_NL_MAX = 1600;  // the grid's limit: 40 x 40 nodes
// Largest subdomain (free vertices) of the mesh path: its dense mean-operator inverse holds nl^2 values
// per pattern (128 MB in FP64 at 4096) and takes O(nl^3) host work at set-up.
constexpr int MESH_NL_MAX = 4096;
static int build_mesh_mma(sg_handle h, const std::vector<double>* inv) {
  const auto& pr = h->pr;
  const int nl = pr.nl;
  h->Kp = (nl + sgk::MMA_M - 1) / sgk::MMA_M * sgk::MMA_M;
  h->NC = h->Kp / sgk::MMA_KC;
  h->MT = h->Kp / sgk::MMA_M;
  h->mma_nb = pr.P <= 16 ? 16 : 32;
  const long long per = (long long)pr.nsub * h->Kp * h->Kp;
  {
    std::vector<__nv_bfloat16> img((size_t)(2 * per), __float2bfloat16_rn(0.f));
    for (int pat = 0; pat < 2; ++pat)
      for (int s = 0; s < pr.nsub; ++s)
        for (int a = 0; a < nl; ++a)
          for (int c = 0; c < nl; ++c)
            img[(size_t)pat * per + ((size_t)s * h->Kp + a) * h->Kp + c] =
                __float2bfloat16_rn((float)inv[pat][((size_t)s * nl + a) * nl + c]);
    RET(upload(h, &h->ainv, img));
  }
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  cudaDriverEntryPointQueryResult qr;
  CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&enc, 12000, cudaEnableDefault, &qr));
  if (!enc || qr != cudaDriverEntryPointSuccess) {
    h->err = "cuTensorMapEncodeTiled is not available from the driver";
    return SG_ECUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)h->Kp, (cuuint64_t)(2LL * pr.nsub * h->Kp)};
  const cuuint64_t strides[1] = {(cuuint64_t)h->Kp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)sgk::MMA_KC, (cuuint32_t)sgk::MMA_M};
  const cuuint32_t es[2] = {1, 1};
  const CUresult cr = enc(&h->tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, h->ainv, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    h->err = "tensor map encoding of the mean-operator inverse failed";
    return SG_ECUDA;
  }
  RET(smem_attr(h, sgk::k_pre_mma<32>, sgk::PreShape<32, 2>::SMEM));
  RET(smem_attr(h, sgk::k_pre_mma<16>, sgk::PreShape<16, 2>::SMEM));
  h->mma = true;
  RET(ensure_bimg(h, pr.nsub));
  return ensure_ws<float>(h, pr.nsub);
}

// General partition of a triangle mesh: host tables (vertex classes with the Sec. 3 corners, sparse
// rows, maps), the dense mean-operator inverses in the subdomain-solve precision, then the shared
// uploads, coarse space and initial state.
static int setup_mesh_impl(sg_handle h, const sg_mesh* m, const sg_kl* kl, const sg_pce* pce, const sg_params* prm,
                           const sg_source* src) {
  sgh::SourceDesc sd;
  RET(check_source(h, src, &sd));
  if (prm->precision < SG_FP64 || prm->precision > SG_BF16) { h->err = "precision"; return SG_EINVAL; }
  if (prm->precond < SG_PC_NN2 || prm->precond > SG_PC_LUMPED) { h->err = "precond"; return SG_EINVAL; }
  if (m->nv < 3 || m->ne < 1 || !m->xy || !m->dirichlet || !m->tri || !m->part) {
    h->err = "mesh: vertices, triangles and partition required";
    return SG_EINVAL;
  }
  sgh::MeshProblem mp;
  std::string msg = sgh::build_mesh_problem(mp, m->nv, m->xy, m->dirichlet, m->ne, m->tri, m->part, kl->M, kl->sigma,
                                            kl->bx, kl->by, kl->g0, pce->p, pce->p_in, kl->modes,
                                            kl->modes ? kl->lambdas : nullptr);
  if (!msg.empty()) { h->err = msg; return SG_EINVAL; }
  if (mp.nsub < 2 || mp.nG == 0) { h->err = "mesh: at least two subdomains with an interface are required"; return SG_ENOTSUP; }
  sgh::MeshRows mr;
  msg = sgh::mesh_to_problem(h->pr, mr, mp, m->xy, m->tri, prm->dt, prm->alpha0, prm->alpha1, sd);
  if (!msg.empty()) { h->err = msg; return SG_EINVAL; }
  auto& pr = h->pr;
  pr.sigma = kl->sigma; pr.bx = kl->bx; pr.by = kl->by; pr.g0 = kl->g0;
  if (pr.nl > MESH_NL_MAX) {
    h->err = "mesh: a subdomain has " + std::to_string(pr.nl) + " free vertices; the dense mean-operator "
             "inverse allows at most " + std::to_string(MESH_NL_MAX) + " (use more subdomains)";
    return SG_ENOTSUP;
  }
  if (prm->precision == SG_BF16 && (pr.P > 32 || pr.nl > MESH_MMA_NL_MAX)) {
    h->err = "SG_BF16: the BF16 tensor-core preconditioner needs P <= 32 and at most " +
             std::to_string(MESH_MMA_NL_MAX) + " free vertices per subdomain";
    return SG_ENOTSUP;
  }
  h->mesh = true;
  RET(apply_params(h, prm));
  // dense inverses of the mean operators (FP64 on the host): Dirichlet and Neumann patterns, and the
  // all-free pattern for the one-level Neumann-Neumann comparison
  const int npat = h->pc == SG_PC_NN1 ? 3 : 2;
  std::vector<double> inv[3];
  for (int pat = 0; pat < npat; ++pat)
    if (!sgh::mesh_mean_inverse(pr, mr, pat, h->am, h->bk, inv[pat])) {
      h->err = "mean operator of a subdomain not positive definite";
      return SG_ENUMERIC;
    }
  RET(init_device(h));
  RET(upload(h, &h->cls, pr.cls));
  RET(upload(h, &h->m_rp, mr.row_ptr)); RET(upload(h, &h->m_col, mr.col)); RET(upload(h, &h->m_npat, mr.npat));
  RET(upload(h, &h->m_kv, mr.kval)); RET(upload(h, &h->m_mv, mr.mval));
  {
    std::vector<float> k32(mr.kval.begin(), mr.kval.end()), m32(mr.mval.begin(), mr.mval.end());
    std::vector<float> g32(pr.gk_v.begin(), pr.gk_v.end());
    RET(upload(h, &h->m_kv32, k32)); RET(upload(h, &h->m_mv32, m32)); RET(upload(h, &h->gk_v32, g32));
  }
  // SG_BF16: the FP32 solves of patterns 0 and 1 take the inverse's BF16 image on the tensor cores
  if (h->policy == SG_BF16) RET(build_mesh_mma(h, inv));
  for (int pat = 0; pat < npat; ++pat) {
    if (h->precision == SG_FP64) {
      RET(upload(h, &h->m_ainv[pat], inv[pat]));
    } else {
      std::vector<float> f(inv[pat].begin(), inv[pat].end());
      RET(upload(h, &h->m_ainv32[pat], f));
    }
    std::vector<double>().swap(inv[pat]);
  }
  RET(upload_common(h));
  return finish_setup(h);
}

static int fill_stats(sg_handle h, int nsteps, long long inner0, sg_stats* stats) {
  if (!stats) return SG_OK;
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  long long inner = 0;
  CK(cudaMemcpy(&inner, h->ctl.it_total, sizeof(long long), cudaMemcpyDeviceToHost));
  stats->steps = nsteps;
  stats->step_index = (int)h->step;
  const size_t ni = h->iters.size();
  stats->iters_last = ni ? h->iters.back() : 0;
  long long tot = 0;
  for (size_t i = ni >= (size_t)nsteps ? ni - nsteps : 0; i < ni; ++i) tot += h->iters[i];
  stats->iters_total = tot;
  stats->inner_total = inner - inner0;
  stats->relres_last = h->relres.empty() ? 0.0 : h->relres.back();
  stats->ms = ms;
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

int sg_setup_mesh(const sg_mesh* mesh, const sg_kl* kl, const sg_pce* pce, const sg_params* params,
                  const sg_source* src, void* stream, sg_handle* out) {
  if (!out) return SG_EINVAL;
  *out = nullptr;
  if (!mesh || !kl || !pce || !params) { g_setup_err = "null argument"; return SG_EINVAL; }
  sg_handle h = new (std::nothrow) sg_handle_s();
  if (!h) return SG_ENOMEM;
  h->st = (cudaStream_t)stream;
  int rc = setup_mesh_impl(h, mesh, kl, pce, params, src);
  if (rc != SG_OK) {
    g_setup_err = h->err;
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return SG_OK;
}

static int step_common(sg_handle h, int nsteps, const double* f_host, double* u_host, sg_stats* stats) {
  if (!h || nsteps < 0) return SG_EINVAL;
  h->iters.clear();
  h->relres.clear();
  long long inner0 = 0;
  CK(cudaMemcpy(&inner0, h->ctl.it_total, sizeof(long long), cudaMemcpyDeviceToHost));
  CK(cudaEventRecord(h->ev0, h->st));
  int rc = SG_OK;
  RET(run_steps(h, nsteps, f_host, u_host, &rc));
  CK(cudaEventRecord(h->ev1, h->st));
  CK(cudaEventSynchronize(h->ev1));
  RET(fill_stats(h, nsteps, inner0, stats));
  return rc;
}

int sg_step(sg_handle h, int nsteps, sg_stats* stats) { return step_common(h, nsteps, nullptr, nullptr, stats); }

int sg_step_host(sg_handle h, int nsteps, const double* f_host, double* u_host, sg_stats* stats) {
  return step_common(h, nsteps, f_host, u_host, stats);
}

// Batched run: one CUDA graph holds one time step of EVERY handle as concurrent branches (fork from
// a private stream to each handle's own capture stream, join back); the graph is launched once per
// time step, so a step of the whole batch is a single launch.  Each handle's step keeps its own
// conditional WHILE/IF loops (same nesting depth as the single-handle graph).
static int batch_impl(sg_handle* hs, int n, int nsteps, sg_stats* out_n) {
  sg_handle h = hs[0];  // errors are reported on the first handle
  for (int i = 1; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (hs[i] == hs[j]) { h->err = "sg_solve_batch: duplicate handle"; return SG_EINVAL; }
  std::vector<cudaEvent_t> ev(n + 1, nullptr);
  for (auto& e : ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaStream_t root;
  CK(cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking));
  for (int i = 0; i < n; ++i) CK(cudaStreamSynchronize(hs[i]->st));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  int rc = SG_OK;
  std::string why;
  if (cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    h->err = "batch: begin capture failed";
    rc = SG_ECUDA;
  } else {
    cudaEventRecord(ev[n], root);  // fork point
    int joined = 0;
    for (int i = 0; i < n; ++i) {
      sg_handle hi = hs[i];
      if (cudaStreamWaitEvent(hi->cs[0], ev[n], 0) != cudaSuccess) { why = "fork"; rc = SG_ECUDA; break; }
      ++joined;
      Ctx ci{hi->cs[0], 0, true};
      const int r = enq_step(hi, ci, false);
      cudaEventRecord(ev[i], hi->cs[0]);
      cudaStreamWaitEvent(root, ev[i], 0);  // join (also after a failure, so the capture can end)
      if (r != SG_OK) {
        why = hi->err;
        rc = r;
        break;
      }
    }
    (void)joined;
    const cudaError_t e = cudaStreamEndCapture(root, &g);
    if (rc == SG_OK && e != cudaSuccess) { why = std::string("end capture: ") + cudaGetErrorString(e); rc = SG_ECUDA; }
    if (rc != SG_OK) h->err = "sg_solve_batch: " + why;
  }
  if (rc == SG_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    h->err = "sg_solve_batch: graph instantiation failed";
    rc = SG_ECUDA;
  }
  std::vector<long long> first(n);
  float ms = 0.f;
  if (rc == SG_OK) {
    for (int i = 0; i < n; ++i) {
      first[i] = hs[i]->step;
      hs[i]->iters.clear();
      hs[i]->relres.clear();
      CK(cudaMemsetAsync(hs[i]->rec_flags, 0, sizeof(int), root));
    }
    CK(cudaEventRecord(h->ev0, root));
    for (int s = 0; s < nsteps && rc == SG_OK; ++s)
      if (cudaGraphLaunch(ex, root) != cudaSuccess) { h->err = "sg_solve_batch: graph launch failed"; rc = SG_ECUDA; }
    CK(cudaEventRecord(h->ev1, root));
    if (cudaStreamSynchronize(root) != cudaSuccess) { h->err = "sg_solve_batch: run failed"; rc = SG_ECUDA; }
    if (rc == SG_OK) cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  }
  if (ex) cudaGraphExecDestroy(ex);
  if (g) cudaGraphDestroy(g);
  for (auto& e : ev) cudaEventDestroy(e);
  cudaStreamDestroy(root);
  if (rc != SG_OK) return rc;
  int worst = SG_OK;
  for (int i = 0; i < n; ++i) {
    sg_handle hi = hs[i];
    const long long cnt = std::min<long long>(nsteps, REC_CAP);
    std::vector<int> it((size_t)cnt);
    std::vector<double> rl((size_t)cnt);
    const long long s0 = (first[i] + nsteps - cnt) % REC_CAP;
    for (long long k = 0; k < cnt; ++k) {
      CK(cudaMemcpy(&it[k], hi->rec_iters + (s0 + k) % REC_CAP, sizeof(int), cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(&rl[k], hi->rec_rel + (s0 + k) % REC_CAP, sizeof(double), cudaMemcpyDeviceToHost));
    }
    hi->iters = it;
    hi->relres = rl;
    hi->step += nsteps;
    int flags = 0, brk = 0;
    CK(cudaMemcpy(&flags, hi->rec_flags, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&brk, hi->ctl.breakdown, sizeof(int), cudaMemcpyDeviceToHost));
    if (brk >= 16) worst = SG_ETIMEOUT;
    else if ((flags & 2) || brk) worst = SG_ENUMERIC;
    else if ((flags & 1) && worst == SG_OK) worst = SG_ENOTCONV;
    if (out_n) {
      sg_stats& st = out_n[i];
      st.steps = nsteps;
      st.step_index = (int)hi->step;
      st.iters_last = cnt ? it.back() : 0;
      long long tot = 0;
      for (int v : it) tot += v;
      st.iters_total = tot;
      long long inner = 0;
      CK(cudaMemcpy(&inner, hi->ctl.it_total, sizeof(long long), cudaMemcpyDeviceToHost));
      st.inner_total = inner;  // cumulative for the handle
      st.relres_last = cnt ? rl.back() : 0.0;
      st.ms = ms;              // wall time of the whole batched run
    }
  }
  return worst;
}

int sg_solve_batch(sg_handle* hs, int n, int nsteps, sg_stats* out_n) {
  if (!hs || n <= 0 || nsteps < 0) return SG_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!hs[i]) return SG_EINVAL;
  return batch_impl(hs, n, nsteps, out_n);
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

// ---- PCE surrogate sampling ----
int sg_sample_field(sg_handle h, int nsamp, const double* xi, int npts, const int* nodes, double* out, int on_device) {
  if (!h || nsamp < 1 || npts < 1 || !xi || !nodes || !out) return SG_EINVAL;
  const auto& pr = h->pr;
  if (pr.M > sgk::SURR_MAXM || pr.p > sgk::SURR_MAXA) {
    h->err = "sg_sample_field: more random variables or a higher order than the sampler supports";
    return SG_ENOTSUP;
  }
  if (!h->alpha_d) {
    std::vector<signed char> a((size_t)pr.P * std::max(pr.M, 1), 0);
    for (int k = 0; k < pr.P; ++k)
      for (int n = 0; n < pr.M; ++n) a[(size_t)k * pr.M + n] = (signed char)pr.alpha_out[k][n];
    RET(upload(h, &h->alpha_d, a));
  }
  if (!on_device)
    for (int j = 0; j < npts; ++j)
      if (nodes[j] < 0 || nodes[j] >= pr.n_free) { h->err = "sg_sample_field: node index out of range"; return SG_EINVAL; }
  const long long ns = nsamp, np = npts;
  if (h->samp_cap_s < ns) {
    dfree(h, &h->samp_psi);
    dfree(h, &h->samp_xi);
    RET(dalloc(h, &h->samp_psi, ns * pr.P));
    RET(dalloc(h, &h->samp_xi, ns * std::max(pr.M, 1)));
    h->samp_cap_s = ns;
  }
  const double* dxi = xi;
  const int* dnodes = nodes;
  double* dout = out;
  if (!on_device) {
    if (h->samp_cap_p < np) {
      dfree(h, &h->samp_nodes);
      RET(dalloc(h, &h->samp_nodes, np));
      h->samp_cap_p = np;
    }
    if (h->samp_cap_out < ns * np) {
      dfree(h, &h->samp_out);
      RET(dalloc(h, &h->samp_out, ns * np));
      h->samp_cap_out = ns * np;
    }
    if (pr.M > 0)
      CK(cudaMemcpyAsync(h->samp_xi, xi, sizeof(double) * ns * pr.M, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->samp_nodes, nodes, sizeof(int) * np, cudaMemcpyHostToDevice, h->st));
    dxi = h->samp_xi;
    dnodes = h->samp_nodes;
    dout = h->samp_out;
  }
  const int pmax = pr.p;
  sgk::k_psi<<<nblk(ns, 128), 128, 0, h->st>>>(nsamp, pr.M, pr.P, pmax, h->alpha_d, dxi, h->samp_psi);
  sgk::k_surrogate<<<nblk(ns * np), 256, 0, h->st>>>(nsamp, npts, pr.P, pr.n_free, dnodes, h->free_owner, h->U,
                                                     h->samp_psi, dout);
  CKL();
  if (!on_device) CK(cudaMemcpyAsync(out, dout, sizeof(double) * ns * np, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return SG_OK;
}

// ---- moments without allocation: static device staging array ----
// Capacity: SG_NOALLOC_MAX_FREE (include/sg.h) free nodes, mean and variance: 2 x 2^20 doubles =
// 16 MiB.  The array is a file-scope device variable, so every GPU that loads this library holds it
// until the process exits.
static __device__ __align__(256) double g_noalloc_stage[2 * (size_t)SG_NOALLOC_MAX_FREE];
constexpr int SG_NOALLOC_MAX_DEV = 64;
// Device address of the array per device.  Threads that race on the first look-up on a device all
// store the same address, so a relaxed atomic is enough.
static std::atomic<double*> g_noalloc_ptr[SG_NOALLOC_MAX_DEV];

int sg_get_moments_noalloc(sg_handle h, double* mean, double* var) {
  if (!h) return SG_EINVAL;
  if (!mean && !var) {
    h->err = "sg_get_moments_noalloc: mean and var are both NULL";
    return SG_EINVAL;
  }
  const auto& pr = h->pr;
  if (pr.n_free > SG_NOALLOC_MAX_FREE) {
    h->err = "sg_get_moments_noalloc: more free nodes than the static staging array holds (2^20)";
    return SG_EINVAL;
  }
  // the kernel runs on the handle's stream, which belongs to the device of sg_setup: the array's
  // address must be that device's
  int cur = -1;
  CK(cudaGetDevice(&cur));
  if (cur != h->dev) {
    h->err = "sg_get_moments_noalloc: the current device is not the one the handle was set up on";
    return SG_EINVAL;
  }
  if (h->dev < 0 || h->dev >= SG_NOALLOC_MAX_DEV) {
    h->err = "sg_get_moments_noalloc: device index out of range";
    return SG_EINVAL;
  }
  double* dm = g_noalloc_ptr[h->dev].load(std::memory_order_relaxed);
  if (!dm) {
    // one-time set-up on this device, with it current: in host code the array's name is only a
    // stand-in, the kernel needs the device address
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_stage));
    dm = static_cast<double*>(p);
    g_noalloc_ptr[h->dev].store(dm, std::memory_order_relaxed);
  }
  double* dv = dm + SG_NOALLOC_MAX_FREE;
  // every entry that is copied out is written first, so nothing needs clearing between calls
  sgk::k_moments<<<nblk(pr.n_free), 256, 0, h->st>>>(pr.n_free, pr.P, h->free_owner, h->U, mean ? dm : nullptr,
                                                      var ? dv : nullptr);
  CKL();
  if (mean) CK(cudaMemcpyAsync(mean, dm, sizeof(double) * pr.n_free, cudaMemcpyDeviceToHost, h->st));
  if (var) CK(cudaMemcpyAsync(var, dv, sizeof(double) * pr.n_free, cudaMemcpyDeviceToHost, h->st));
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
  double stepd = 0.0;
  CK(cudaMemcpy(&stepd, src + 3 * cnt, sizeof(double), on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  if (!(stepd >= 0) || stepd != std::floor(stepd)) return SG_EINVAL;
  double* dst[3] = {h->U, h->V, h->A};
  for (int q = 0; q < 3; ++q) {
    CK(cudaMemcpyAsync(h->outbuf, src + q * cnt, sizeof(double) * cnt,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    sgk::k_scatter_free<<<nblk(h->nvec()), 256, 0, h->st>>>(h->nloc(), pr.P, h->free_of_local, h->outbuf, dst[q]);
    CKL();
  }
  h->step = (long long)stepd;
  CK(cudaMemcpyAsync(h->stepctr, &h->step, sizeof(long long), cudaMemcpyHostToDevice, h->st));
  sgk::k_scatter<double><<<nblk(h->nGd()), 256, 0, h->st>>>(pr.nG, pr.P, h->owners, pr.mo, h->Dw, h->U, h->xG, 1);
  CKL();
  RET(warm_reset_history(h));
  CK(cudaStreamSynchronize(h->st));
  return SG_OK;
}

int sg_get_sizes(sg_handle h, sg_sizes* out) {
  if (!h || !out) return SG_EINVAL;
  const auto& pr = h->pr;
  out->N = pr.N; out->nsub = pr.nsub; out->P = pr.P; out->P_in = pr.PI; out->n_free = pr.n_free;
  out->n_gamma = pr.nG; out->n_corner = pr.nC; out->n_sub_nodes = pr.nl; out->device_bytes = h->bytes;
  out->fp32_precond = h->mma ? 1 : 0;
  out->compiled_apply = gfix_for<float>(pr) >= 0 ? 1 : 0;
  return SG_OK;
}

int sg_partition_rcb(int nv, const double* xy, int ne, const int* tri, int nparts, int* part) {
  const std::string msg = sgh::partition_rcb(nv, xy, ne, tri, nparts, part);
  if (!msg.empty()) { g_setup_err = msg; return SG_EINVAL; }
  return SG_OK;
}

int sg_mesh_plan_query(const sg_mesh* mesh, const sg_kl* kl, const sg_pce* pce, const sg_params* params,
                       sg_mesh_plan* out) {
  if (!mesh || !kl || !pce || !params || !out) { g_setup_err = "null argument"; return SG_EINVAL; }
  if (params->precision < SG_FP64 || params->precision > SG_BF16) { g_setup_err = "precision"; return SG_EINVAL; }
  if (params->precond < SG_PC_NN2 || params->precond > SG_PC_LUMPED) { g_setup_err = "precond"; return SG_EINVAL; }
  if (mesh->nv < 3 || mesh->ne < 1 || !mesh->xy || !mesh->dirichlet || !mesh->tri || !mesh->part) {
    g_setup_err = "mesh: vertices, triangles and partition required";
    return SG_EINVAL;
  }
  sgh::MeshProblem mp;
  std::string msg = sgh::build_mesh_problem(mp, mesh->nv, mesh->xy, mesh->dirichlet, mesh->ne, mesh->tri, mesh->part,
                                            kl->M, kl->sigma, kl->bx, kl->by, kl->g0, pce->p, pce->p_in, kl->modes,
                                            kl->modes ? kl->lambdas : nullptr);
  if (!msg.empty()) { g_setup_err = msg; return SG_EINVAL; }
  sgh::Problem pr;
  sgh::MeshRows mr;
  const sgh::SourceDesc sd{0, 0.5, 0.5, 0.05, 10.0, 1.0};
  msg = sgh::mesh_to_problem(pr, mr, mp, mesh->xy, mesh->tri, params->dt, params->alpha0, params->alpha1, sd);
  if (!msg.empty()) { g_setup_err = msg; return SG_EINVAL; }
  sg_mesh_plan p{};
  p.nsub = pr.nsub; p.n_free = pr.n_free; p.n_gamma = pr.nG; p.n_corner = pr.nC;
  p.P = pr.P; p.P_in = pr.PI; p.nnz_G = (int)pr.gk_v.size();
  p.n_sub_nodes = pr.nl; p.max_owners = pr.mo; p.max_corners = pr.max_corner; p.max_gamma = pr.nGam;
  p.row_entries = (long long)mr.col.size();
  p.coarse_dim = (long long)pr.nC * pr.P;
  const bool fp64 = params->precision == SG_FP64;
  const long long nloc = (long long)pr.nsub * pr.nl, nvec = nloc * pr.P;
  // sparse rows: columns, FP64 and FP32 values (mass and every input-mode stiffness), row pointers
  p.bytes_rows = p.row_entries * (4 + 12LL * (pr.PI + 1)) + 4 * (nloc + 1);
  // dense mean-operator inverses in the subdomain-solve type, plus the BF16 image for SG_BF16
  const int npat = params->precond == SG_PC_NN1 ? 3 : 2;
  p.bytes_inverses = (long long)npat * pr.nsub * pr.nl * pr.nl * (fp64 ? 8 : 4);
  p.mma = params->precision == SG_BF16 && pr.P <= 32 && pr.nl <= MESH_MMA_NL_MAX ? 1 : 0;
  if (p.mma) {
    const long long kp = (pr.nl + sgk::MMA_M - 1) / sgk::MMA_M * sgk::MMA_M;
    p.bytes_inverses += 2LL * pr.nsub * kp * kp * 2;
  }
  // coarse space of the two-level preconditioner: local bases Phi and the dense inverse of F_cc
  if (params->precond == SG_PC_NN2) {
    p.bytes_coarse_basis = (long long)pr.nsub * std::max(pr.max_corner * pr.P, 1) * pr.nGam * pr.P * 8;
    p.bytes_coarse_matrix = p.coarse_dim * p.coarse_dim * 8;
  }
  // state and step vectors of the local layout (FP64: U, V, A, the Newmark and work vectors, the
  // interior accumulator of the mixed path; FP32: two work vectors) and the inner-CG workspaces of
  // both types (six vectors each, one problem per subdomain)
  p.bytes_vectors = nvec * (14 * 8 + 2 * 4) + 6 * nvec * (8 + 4);
  p.fits = pr.nl <= MESH_NL_MAX && (params->precision != SG_BF16 || p.mma) ? 1 : 0;
  *out = p;
  return SG_OK;
}

int sg_plan_query(const sg_grid* grid, const sg_kl* kl, const sg_pce* pce, const sg_params* params, sg_plan* out) {
  if (!grid || !kl || !pce || !params || !out) { g_setup_err = "null argument"; return SG_EINVAL; }
  sgh::Problem pr;
  const sgh::SourceDesc sd{0, 0.5, 0.5, 0.05, 10.0, 1.0};
  const int rc = build_checked(pr, g_setup_err, grid, kl, pce, params, sd);
  if (rc != SG_OK) return rc;
  sg_plan p{};
  p.L = pr.L; p.P = pr.P; p.P_in = pr.PI; p.nsub = pr.nsub; p.nnz_G = (int)pr.gk_v.size();
  auto fill = [&](auto tag, int i) {
    using T = decltype(tag);
    int TL, NT, stage, nods;
    size_t sm;
    apply_cfg<T>(pr, pr.nsub, &TL, &NT, &sm, &stage, &nods);
    p.apply_variant[i] = gfix_for<T>(pr) >= 0 ? 3 : nods;
    p.apply_lines[i] = TL;
    p.apply_tiles[i] = NT;
    p.apply_smem[i] = (long long)sm;
    const LineCfg lc = line_cfg<T>(pr, pr.nsub);
    p.line_kind[i] = lc.team ? 1 : lc.gs ? 2 : lc.wide ? 3 : 0;
    p.line_modes[i] = lc.G;
    p.line_groups[i] = lc.NG;
    p.line_block[i][0] = (int)lc.block.x; p.line_block[i][1] = (int)lc.block.y; p.line_block[i][2] = (int)lc.block.z;
    p.line_smem[i] = (long long)lc.smem;
    if (sizeof(T) == 4 && line_tc_eligible(pr, params->precision)) {
      p.line_kind[i] = 4;
      p.line_block[i][0] = ltc_threads(pr.L, lc.G); p.line_block[i][1] = 1; p.line_block[i][2] = 1;
      p.line_smem[i] = (long long)sgk::ltc_smem(pr.L, lc.G, ltc_nb(lc.G));
    }
  };
  fill(double{}, 0);
  fill(float{}, 1);
  if (mma_eligible(pr, params->precision)) {
    p.mma = 1;
    p.mma_kp = (pr.L * pr.L + sgk::MMA_M - 1) / sgk::MMA_M * sgk::MMA_M;
    p.mma_nc = p.mma_kp / sgk::MMA_KC;
    p.mma_mt = p.mma_kp / sgk::MMA_M;
    p.mma_nb = pr.P <= 16 ? 16 : 32;
    p.mma_smem = p.mma_nb == 16 ? sgk::PreShape<16, 2>::SMEM : sgk::PreShape<32, 2>::SMEM;
  }
  p.fits = tiles_fit(pr, params->precision) ? 1 : 0;
  *out = p;
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

long long sg_launch_count(sg_handle h) {
  if (!h) return SG_EINVAL;
  unsigned long long v = 0;
  if (cudaMemcpy(&v, h->nlaunch, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return SG_ECUDA;
  return (long long)v;
}

int sg_warm_weights(sg_handle h, float* get_host, const float* set_host, int n) {
  if (!h || h->warm != SG_WARM_LEARNED || n != sgk::NN_NP) return SG_EINVAL;
  if (get_host) {
    CK(cudaMemcpyAsync(get_host, h->wctl.theta, sizeof(float) * n, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  if (set_host) {
    CK(cudaMemcpyAsync(h->wctl.theta, set_host, sizeof(float) * n, cudaMemcpyHostToDevice, h->st));
    sgk::k_to_bf16<<<nblk(n), 256, 0, h->st>>>(n, h->wctl.theta, h->wctl.wb);
    CKL();
    const int one = 1;
    CK(cudaMemcpyAsync(h->wctl.trained, &one, sizeof(int), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(h->wctl.train_left, 0, sizeof(int), h->st));  // a given network is not retrained
    CK(cudaMemsetAsync(h->wctl.m, 0, sizeof(float) * n, h->st));
    CK(cudaMemsetAsync(h->wctl.v, 0, sizeof(float) * n, h->st));
    CK(cudaMemsetAsync(h->wctl.adam_it, 0, sizeof(int), h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  return SG_OK;
}

int sg_warm_status(sg_handle h, int* trained, int* train_left, float* loss) {
  if (!h || h->warm != SG_WARM_LEARNED) return SG_EINVAL;
  int a = 0, b = 0;
  float l = 0.f;
  CK(cudaMemcpy(&a, h->wctl.trained, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&b, h->wctl.train_left, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&l, h->wctl.loss, sizeof(float), cudaMemcpyDeviceToHost));
  if (trained) *trained = a;
  if (train_left) *train_left = b;
  if (loss) *loss = l;
  return SG_OK;
}

int sg_mlp_eval(int rows, const float* X, const float* t, const float* theta, float* y, float* grad, double* loss) {
  if (rows <= 0 || !X || !theta) return SG_EINVAL;
  const int nb = (rows + sgk::NN_ROWS - 1) / sgk::NN_ROWS;
  __nv_bfloat16* wb = nullptr;
  float* part = nullptr;
  double *lp = nullptr, *ld = nullptr;
  int rc = SG_OK;
  if (cudaMalloc(&wb, sizeof(__nv_bfloat16) * sgk::NN_NP) != cudaSuccess ||
      cudaMalloc(&part, sizeof(float) * (size_t)nb * sgk::NN_NP) != cudaSuccess ||
      cudaMalloc(&lp, sizeof(double) * nb) != cudaSuccess || cudaMalloc(&ld, sizeof(double)) != cudaSuccess)
    rc = SG_ENOMEM;
  if (rc == SG_OK) {
    sgk::k_to_bf16<<<nblk(sgk::NN_NP), 256>>>(sgk::NN_NP, theta, wb);
    if (y) sgk::k_mlp<false><<<nb, sgk::NN_ROWS>>>(rows, X, nullptr, wb, y, nullptr, nullptr, nullptr);
    if (grad && t) {
      sgk::k_mlp<true><<<nb, sgk::NN_ROWS>>>(rows, X, t, wb, nullptr, part, lp, nullptr);
      sgk::k_mlp_reduce<<<1, 256>>>(nb, rows, part, lp, grad, ld);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) rc = SG_ECUDA;
    if (rc == SG_OK && loss && grad && t && cudaMemcpy(loss, ld, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = SG_ECUDA;
  }
  cudaFree(wb);
  cudaFree(part);
  cudaFree(lp);
  cudaFree(ld);
  return rc;
}

int sg_set_enqueue_mode(sg_handle h, int eager) {
  if (!h || (eager != 0 && eager != 1)) return SG_EINVAL;
  h->eager = eager != 0;
  return SG_OK;
}

int sg_kernel_timing(sg_handle h, int which, double* total_ms, long long* launches) {
  if (!h || which < 0 || which > 4) return SG_EINVAL;
  if (total_ms) *total_ms = h->kprof_ms;
  if (launches) *launches = h->kprof_n;
  h->kprof = which;
  h->kprof_ms = 0.0;
  h->kprof_n = 0;
  return SG_OK;
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
