// Device kernels of the SG-DD wave solver (sm_103a).
//
// Vectors of subdomain problems use the local layout [problem b][local node ln][PCE mode k],
// ln = lj * L + li on the (H+1) x (H+1) node grid of a subdomain; problem b belongs to subdomain
// b / R (R right-hand sides per subdomain).  Interface vectors use [global interface node][k].
// Nodes outside a problem's free set always hold 0, so operators never need input masks.
// Every kernel bumps a device launch counter from its first thread (for launch accounting).
#pragma once
#include <cmath>
#include <cstdint>
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include "sg_gfix.cuh"
#include "sg_mma.cuh"

namespace sgk {

enum : int { DIR = 0, INT = 1, REM = 2, COR = 3 };
constexpr int MASK_I = 1 << INT, MASK_R = 1 << REM, MASK_C = 1 << COR;
constexpr int MASK_G = MASK_R | MASK_C, MASK_FREE = MASK_I | MASK_R | MASK_C, MASK_N = MASK_I | MASK_R;

__device__ unsigned long long* g_nlaunch;  // set once per context by the host (may stay null)

// Optional per-phase cycle marks of block 0 (only when a profiling build defines SG_PHASE_TIMING).
#ifdef SG_PHASE_TIMING
__device__ long long g_phase[16];
#define SG_MARK(i)                                                          \
  do {                                                                      \
    if (blockIdx.x == 0 && threadIdx.x == 0) g_phase[i] = clock64();        \
  } while (0)
#else
#define SG_MARK(i) \
  do {             \
  } while (0)
#endif

__device__ __forceinline__ void count_launch() {
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0 && g_nlaunch)
    atomicAdd(g_nlaunch, 1ULL);
}

// FP32 partial sums at any magnitude: a thread's operands are scaled by powers of two (exactly) so
// that the largest lies in [1, 2), the scaled products are summed in FP32 and the partial joins the
// FP64 total with one multiplication by the inverse scale.  Scaled products can neither overflow nor
// lose to underflow anything that the FP32 sum would keep, so subdomain problems whose values are
// far from 1 (the far field of the wave reaches 1e-30 and below) are summed like any other; FP64
// arithmetic, which runs at a small fraction of the FP32 rate on this part, stays out of the loop.
// f32_exp: binary exponent of amax >= 0, clamped so that 2^-e is a normal FP32 value (0 for 0).
__device__ __forceinline__ int f32_exp(float amax) {
  const int f = (int)((__float_as_uint(amax) >> 23) & 0xffu);
  if (f == 0) return amax == 0.f ? 0 : -126;
  return min(f - 127, 126);
}
__device__ __forceinline__ float f32_pow2(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }  // |e| <= 126
__device__ __forceinline__ double f64_pow2(int e) { return __hiloint2double((e + 1023) << 20, 0); }      // |e| <= 1022
// Running total (h + l) 2^e of such partials across the steps of a launch in FP32 arithmetic (TwoSum
// keeps the rounding error of each addition in l), converted to FP64 once at the end.
struct XAcc {
  float h = 0.f, l = 0.f;
  int e = -1000;  // exponent of an empty total
  __device__ __forceinline__ void add(float v, int ev) {  // += v 2^ev, 0 <= |v| < 2^24
    if (v == 0.f) return;
    if (ev > e) {  // rescale the total to the new exponent (parts far below it vanish)
      const int d = e - ev;
      const float f = d >= -126 ? f32_pow2(d) : 0.f;
      h *= f;
      l *= f;
      e = ev;
    } else {
      const int d = ev - e;
      v = d >= -126 ? v * f32_pow2(d) : 0.f;
    }
    const float s = __fadd_rn(h, v);
    const float bb = __fsub_rn(s, h);
    l = __fadd_rn(l, __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(v, bb)));
    h = s;
  }
  __device__ __forceinline__ double value() const {
    return e == -1000 ? 0.0 : ((double)h + (double)l) * f64_pow2(max(min(e, 1022), -1022));
  }
};

// Division by a runtime constant d >= 1 for 0 <= x < 2^31 without a divide instruction:
// q = floor(x * m / 2^(31+s)) with s = ceil(log2 d) and m = ceil(2^(31+s) / d) < 2^32, which is
// exact for every x < 2^31 (round-up multiplier method for 31-bit dividends).
struct FD {
  unsigned m;
  int s;
  unsigned d;
};
__host__ __device__ inline FD make_fd(unsigned d) {
  FD f;
  int s = 0;
  while ((1u << s) < d) ++s;
  f.s = s;
  f.d = d;
  f.m = (unsigned)((((unsigned long long)1 << (31 + s)) + d - 1) / d);
  return f;
}
__device__ __forceinline__ int fdiv(int x, const FD& f) {
  return (int)(((unsigned long long)(unsigned)x * f.m) >> (31 + f.s));
}

// Geometry and Galerkin data of one problem family (shared by every right-hand side).
template <typename T>
struct Op {
  const uint8_t* cls;    // [sub][ln] node class
  const uint8_t* cells;  // [sub][ln] presence bits of the four cells around the node
  const T* kapE;         // [sub][ln][PI] stiffness weight of the edge to (li+1, lj)
  const T* kapN;         // [sub][ln][PI] stiffness weight of the edge to (li, lj+1)
  const int* gk_ptr;     // [P+1] triple products grouped by output mode k
  const int* gk_i;
  const int* gk_j;
  const T* gk_v;
  const unsigned* gk_pk;  // gk_i | gk_j << 16
  int L, nl, P, PI;
  T mass_h;              // h^2 / 24: unit entry of the consistent P1 mass on a right triangle
  FD fP, fPI, fL, fLm1, fLP;  // fast division by P, PI, L, L-1, L*P
};

// Inner-CG control block (device memory), one per batched solve.
struct CgCtl {
  double* rz;        // [nb] r . z of the current iterate
  double* bb;        // [nb] ||b||^2
  double* beta;      // [nb]
  int* active;       // [nb]
  double* part_pq;   // [nb][NT]
  double* part_rz;   // [nb][NG]
  double* part_rr;   // [nb][NG]
  unsigned* counter; // last-block counter of the line kernel
  int* parity;       // which p buffer holds the current direction
  int* it;           // iterations of the current solve
  long long* it_total;
  int* cond;         // mirror of the while condition (eager mode)
  int* breakdown;    // set when p.q <= 0 or non-finite values appear
};

// BF16 terms of an FP32 value, f = t0 + t1 (+ t2) up to the last term's rounding: each remainder
// is exact in FP32.  Two terms keep about 17 significant bits, three about 25.
template <int TERMS>
__device__ __forceinline__ void bf16_split(float f, __nv_bfloat16 (&t)[TERMS]) {
  float rem = f;
#pragma unroll
  for (int i = 0; i < TERMS; ++i) {
    t[i] = __float2bfloat16_rn(rem);
    rem -= __bfloat162float(t[i]);
  }
}

// ------------------------------------------------------------------------------------------
// SG operator apply, tile form.
//   y = add + cm (M (x) I) xm + ck (sum_i K_i (x) G_i) xk      on nodes with class in out_mask
// Stiffness: graph-Laplacian form of P1 on right triangles (each leg carries half the element
// coefficient, the hypotenuse none).  Every edge (a, b) inside a tile computes the flux
//   z_e[k] = sum_{(i,j,k) in G} kappa_i(e) G_ijk (x_a[j] - x_b[j])          (Sec. 4, Eq. stoksub)
// once into shared memory; node a then adds +z for edges where it is the left/bottom end and
// -z otherwise.  Mass: consistent P1 mass h^2/24 [2 1 1; 1 2 1; 1 1 2] per element, block
// diagonal over the modes (deterministic mass, Sec. 4).
// A block handles TL consecutive grid lines of one problem; shared memory holds the input
// lines (TL + 2 with halos), the differences d_e and the fluxes z_e of the block's edges.
// FUSEDP: the input is the CG direction p_new = z + beta p_old, formed on the fly (halo
// included) and written back for the owned lines; DOT: per-block partial of p_new . y.
// ------------------------------------------------------------------------------------------
// C = GDyn: runtime triple-product table staged in shared memory (any PCE size).  C = gfix::Cfg<...>:
// the table is a compile-time constant (sg_gfix.cuh); each work item (edge, output-mode group) keeps
// kappa_e and d_e in registers and the values come from constant memory, so the flux phase issues two
// instructions per triple product and needs neither the difference nor the staging buffers.
template <typename T, typename TO, bool FUSEDP, bool DOT, class C = GDyn>
__global__ void __launch_bounds__(256) k_apply(Op<T> op, int nb, int R, int TL, int NT, int nnz, int stage_kap,
                                               const T* __restrict__ xm, const T* __restrict__ xk, TO* y,
                                               const TO* add, T cm, T ck, int out_mask,
                                               // fused-CG inputs
                                               T* pbuf0, T* pbuf1, const T* __restrict__ zin, const int* parity,
                                               const double* beta, const int* active, double* part_pq) {
  count_launch();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = op.P, L = op.L, nl = op.nl, PI = op.PI;
  const int PS = P | 1, PIS = PI | 1;               // odd row strides: conflict-free per-edge rows
  const int b = blockIdx.x / NT, tile = blockIdx.x % NT;
  const int lj0 = tile * TL;
  const int nlin = min(TL, L - lj0);  // owned lines
  pdl_trigger();
  pdl_wait();
  // the fused-CG scalars in one round trip
  int act_b = 1, par = 0;
  double bet_d = 0.0;
  if (FUSEDP) {
    act_b = active[b];
    par = *parity;
    bet_d = beta[b];
  }
  if (FUSEDP && !act_b) return;
  const int sub = b / R;
  const int nE = nlin * (L - 1), nNr = nlin + 1;
  const int nEd = nE + nNr * L;                     // edges of the block: horizontal then vertical
  T* xs = reinterpret_cast<T*>(smem_raw);           // [(TL+2)][L][P]
  T* ds = xs + (size_t)(TL + 2) * L * P;            // [edges][PS] differences (runtime table only)
  T* zs = (C::fixed || C::nods) ? ds : ds + (size_t)(TL * (L - 1) + (TL + 1) * L) * PS;   // [edges][PS] fluxes
  T* gv_s = zs + (size_t)(TL * (L - 1) + (TL + 1) * L) * PS; // [nnz] (staged table only)
  T* ks = gv_s + (C::gglob ? 0 : nnz);              // [edges][PIS] edge weights (when staged)
  unsigned* gpk_s = reinterpret_cast<unsigned*>(stage_kap ? ks + (size_t)(TL * (L - 1) + (TL + 1) * L) * PIS : ks);
  int* gptr_s = reinterpret_cast<int*>(gpk_s + (C::gglob ? 0 : nnz));  // [P+1]
  const long long pb = (long long)b * nl * P;
  const long long so0 = (long long)sub * nl;
  const int nt = blockDim.x;
  const T* pold = nullptr;
  T* pnew = nullptr;
  T bet = T(0);
  if (FUSEDP) {
    pold = par ? pbuf1 : pbuf0;
    pnew = par ? pbuf0 : pbuf1;
    bet = (T)bet_d;
  }
  SG_MARK(0);
  // phase 0: triple products (values, packed (i, j), per-k ranges) and the block's edge weights
  if constexpr (!C::fixed) {
  if constexpr (!C::gglob) {
    for (int e = threadIdx.x; e < nnz; e += nt) {
      gv_s[e] = op.gk_v[e];
      gpk_s[e] = op.gk_pk[e];
    }
    for (int e = threadIdx.x; e <= P; e += nt) gptr_s[e] = op.gk_ptr[e];
  }
  if (stage_kap) {
    for (int e = threadIdx.x; e < nE * PI; e += nt) {
      const int ed = fdiv(e, op.fPI), i = e - ed * PI;
      const int t = fdiv(ed, op.fLm1), c = ed - t * (L - 1);
      ks[(size_t)ed * PIS + i] = op.kapE[(so0 + (long long)(lj0 + t) * L + c) * PI + i];
    }
    for (int e = threadIdx.x; e < nNr * L * PI; e += nt) {
      const int ed = fdiv(e, op.fPI), i = e - ed * PI;
      const int t = fdiv(ed, op.fL), c = ed - t * L;
      const int jb = lj0 - 1 + t;
      ks[(size_t)(nE + ed) * PIS + i] = (jb >= 0 && jb + 1 < L) ? op.kapN[(so0 + (long long)jb * L + c) * PI + i] : T(0);
    }
  }
  }
  // phase 1: input lines lj0-1 .. lj0+nlin (zeros outside the grid)
  const int nin = (nlin + 2) * L * P;
  const bool vec16 = sizeof(T) == 4 && ((L * P) & 3) == 0 &&
                     ((FUSEDP ? ((reinterpret_cast<uintptr_t>(zin) | reinterpret_cast<uintptr_t>(pold) |
                                  reinterpret_cast<uintptr_t>(pnew)) & 15)
                              : (reinterpret_cast<uintptr_t>(xk) & 15)) == 0);
  // Loads are issued in batches of UB per thread before any store: the output buffers may alias the
  // inputs as far as the compiler knows, so a load-then-store loop would wait a full memory round
  // trip per element.
  constexpr int UB = 8;
  constexpr bool DOT32 = DOT && sizeof(T) == 4;  // p.q partial in scaled FP32 (see f32_exp)
  float axm = 0.f;                                 // largest |p| this thread stages
  if (vec16) {
    // 16-byte vectors: a line of L x P values starts on a 16-byte boundary and holds whole vectors
    const int LP4 = (L * P) >> 2;
    const FD fLP4 = make_fd((unsigned)LP4);
    const int nin4 = nin >> 2;
    for (int e0 = threadIdx.x; e0 < nin4; e0 += nt * UB) {
      float4 va[UB], vb[UB];
      long long gg[UB];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int e4 = e0 + u * nt;
        va[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        vb[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        gg[u] = -1;
        if (e4 < nin4) {
          const int t = fdiv(e4, fLP4);
          const int jl = lj0 - 1 + t;
          if (jl >= 0 && jl < L) {
            gg[u] = pb + (long long)jl * L * P + 4LL * (e4 - t * LP4);
            if (FUSEDP) {
              va[u] = *reinterpret_cast<const float4*>(zin + gg[u]);
              if (bet != T(0)) vb[u] = *reinterpret_cast<const float4*>(pold + gg[u]);
            } else {
              va[u] = *reinterpret_cast<const float4*>(xk + gg[u]);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int e4 = e0 + u * nt;
        if (e4 < nin4) {
          float4 v = va[u];
          if (FUSEDP && gg[u] >= 0) {
            if (bet != T(0)) {
              v.x += (float)bet * vb[u].x;
              v.y += (float)bet * vb[u].y;
              v.z += (float)bet * vb[u].z;
              v.w += (float)bet * vb[u].w;
            }
            const int t = fdiv(e4, fLP4);
            if (t >= 1 && t <= nlin) *reinterpret_cast<float4*>(pnew + gg[u]) = v;
          }
          *reinterpret_cast<float4*>(xs + 4 * e4) = v;
          if constexpr (DOT32) axm = fmaxf(axm, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
      }
    }
  } else {
    for (int e0 = threadIdx.x; e0 < nin; e0 += nt * UB) {
      T va[UB], vb[UB];
      long long gg[UB];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int e = e0 + u * nt;
        va[u] = T(0);
        vb[u] = T(0);
        gg[u] = -1;
        if (e < nin) {
          const int t = fdiv(e, op.fLP);
          const int jl = lj0 - 1 + t;
          if (jl >= 0 && jl < L) {
            gg[u] = pb + (long long)jl * L * P + (e - t * L * P);
            if (FUSEDP) {
              va[u] = zin[gg[u]];
              if (bet != T(0)) vb[u] = pold[gg[u]];
            } else {
              va[u] = xk[gg[u]];
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int e = e0 + u * nt;
        if (e < nin) {
          T v = va[u];
          if (FUSEDP && gg[u] >= 0) {
            if (bet != T(0)) v += bet * vb[u];
            const int t = fdiv(e, op.fLP);
            if (t >= 1 && t <= nlin) pnew[gg[u]] = v;
          }
          xs[e] = v;
          if constexpr (DOT32) axm = fmaxf(axm, fabsf((float)v));
        }
      }
    }
  }
  __shared__ unsigned red_ax[32];
  if constexpr (DOT32) {
    const unsigned w = __reduce_max_sync(0xffffffffu, __float_as_uint(axm));  // order-preserving for x >= 0
    if ((threadIdx.x & 31) == 0) red_ax[threadIdx.x >> 5] = w;
  }
  __syncthreads();
  SG_MARK(1);
  int dex = 0;  // binary exponent of the block's largest |p|
  if constexpr (DOT32) {
    unsigned w = 0u;
    for (int i = 0; i < (nt >> 5); ++i) w = max(w, red_ax[i]);
    dex = f32_exp(__uint_as_float(w));
  }
  const float dsc = DOT32 ? f32_pow2(-dex) : 1.f;
  float dsf = 0.f;
  if constexpr (C::fixed) {
    // phase 2 (compile-time table): one work item per (edge, output-mode group); the group is
    // uniform across a warp (32 consecutive edges), so the unrolled group code never diverges
    if (ck != T(0)) {
      const int nEd32 = (nEd + 31) & ~31;
      for (int it = threadIdx.x; it < nEd32 * C::KG; it += nt) {
        const int wi = it >> 5, g = wi % C::KG;
        const int ed = ((wi / C::KG) << 5) + (it & 31);
        if (ed >= nEd) continue;
        const T* xa;
        const T* xb;
        const T* kp;
        bool live = true;
        if (ed < nE) {
          const int t = fdiv(ed, op.fLm1), c = ed - t * (L - 1);
          xa = xs + ((size_t)(t + 1) * L + c) * P;
          xb = xa + P;
          kp = op.kapE + (so0 + (long long)(lj0 + t) * L + c) * PI;
        } else {
          const int v = ed - nE, t = fdiv(v, op.fL), c = v - t * L;
          const int jb = lj0 - 1 + t;
          live = jb >= 0 && jb + 1 < L;
          xa = xs + ((size_t)t * L + c) * P;
          xb = xa + (size_t)L * P;
          kp = op.kapN + (so0 + (long long)max(jb, 0) * L + c) * PI;
        }
        gflux<C, T>(g, kp, xa, xb, zs + (size_t)ed * PS, live);
      }
    }
  } else {
  // phase 2a: differences d_e = x_a - x_b of every edge (a = left / bottom end); the no-staging
  // variant (nods, for the widest subdomains) forms them on the fly in phase 2b
  if constexpr (!C::nods)
  for (int e = threadIdx.x; e < nEd * P; e += nt) {
    const int ed = fdiv(e, op.fP), j = e - ed * P;
    T dv;
    if (ed < nE) {
      const int t = fdiv(ed, op.fLm1), i = ed - t * (L - 1);
      const T* xr = xs + ((size_t)(t + 1) * L + i) * P;
      dv = xr[j] - xr[P + j];
    } else {
      const int v = ed - nE, t = fdiv(v, op.fL), i = v - t * L;
      const T* xb = xs + ((size_t)t * L + i) * P;
      dv = xb[j] - xb[(size_t)L * P + j];
    }
    ds[(size_t)ed * PS + j] = dv;
  }
  __syncthreads();
  SG_MARK(2);
  // phase 2b: fluxes.  A work item is (pair of edges, range of output modes); the G entries are
  // warp-uniform (broadcast) and each is applied to both edges of the pair.
  if (ck != T(0)) {
    const T* gv_t = C::gglob ? op.gk_v : gv_s;
    const unsigned* gpk_t = C::gglob ? op.gk_pk : gpk_s;
    const int* gptr_t = C::gglob ? op.gk_ptr : gptr_s;
    const int npair = (nEd + 1) >> 1;
    const int KS = max(1, min(P, (2 * nt + npair - 1) / npair));   // mode ranges per pair
    const int kchunk = (P + KS - 1) / KS;
    const FD fpair = make_fd((unsigned)npair);
    for (int it = threadIdx.x; it < npair * KS; it += nt) {
      const int krg = fdiv(it, fpair), pr = it - krg * npair;
      const int e0 = pr, e1 = pr + npair;
      const bool has1 = e1 < nEd;
      const T* kap0;
      const T* kap1;
      bool live0 = true, live1 = has1;
      auto kap_of = [&](int ed, bool& live) -> const T* {
        if (stage_kap) {
          if (ed >= nE) {
            const int v = ed - nE, t = fdiv(v, op.fL);
            const int jb = lj0 - 1 + t;
            live = live && jb >= 0 && jb + 1 < L;
          }
          return (const T*)(ks + (size_t)ed * PIS);
        }
        if (ed < nE) {
          const int t = fdiv(ed, op.fLm1), c = ed - t * (L - 1);
          return op.kapE + (so0 + (long long)(lj0 + t) * L + c) * PI;
        }
        const int v = ed - nE, t = fdiv(v, op.fL), c = v - t * L;
        const int jb = lj0 - 1 + t;
        live = live && jb >= 0 && jb + 1 < L;
        return op.kapN + (so0 + (long long)max(jb, 0) * L + c) * PI;
      };
      kap0 = kap_of(e0, live0);
      kap1 = has1 ? kap_of(e1, live1) : kap0;
      auto ends = [&](int ed, const T*& xa, const T*& xb) {
        if (ed < nE) {
          const int t = fdiv(ed, op.fLm1), c = ed - t * (L - 1);
          xa = xs + ((size_t)(t + 1) * L + c) * P;
          xb = xa + P;
        } else {
          const int v = ed - nE, t = fdiv(v, op.fL), c = v - t * L;
          xa = xs + ((size_t)t * L + c) * P;
          xb = xa + (size_t)L * P;
        }
      };
      const T *xa0 = nullptr, *xb0 = nullptr, *xa1 = nullptr, *xb1 = nullptr;
      if constexpr (C::nods) {
        ends(e0, xa0, xb0);
        ends(has1 ? e1 : e0, xa1, xb1);
      }
      const T* d0 = ds + (size_t)e0 * PS;
      const T* d1 = ds + (size_t)(has1 ? e1 : e0) * PS;
      auto D0 = [&](unsigned j) -> T {
        if constexpr (C::nods) return xa0[j] - xb0[j];
        else return d0[j];
      };
      auto D1 = [&](unsigned j) -> T {
        if constexpr (C::nods) return xa1[j] - xb1[j];
        else return d1[j];
      };
      T* z0 = zs + (size_t)e0 * PS;
      T* z1 = zs + (size_t)(has1 ? e1 : e0) * PS;
      const int k0 = krg * kchunk, k1 = min(P, k0 + kchunk);
      for (int kk = k0; kk < k1; ++kk) {
        T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0);
        const int q1 = gptr_t[kk + 1];
        int q = gptr_t[kk];
        for (; q + 3 < q1; q += 4) {  // four entries per round: loads issue together
          const unsigned p0 = gpk_t[q], p1 = gpk_t[q + 1], p2 = gpk_t[q + 2], p3 = gpk_t[q + 3];
          const T g0 = gv_t[q], g1 = gv_t[q + 1], g2 = gv_t[q + 2], g3 = gv_t[q + 3];
          const unsigned i0 = p0 & 0xffffu, i1 = p1 & 0xffffu, i2 = p2 & 0xffffu, i3 = p3 & 0xffffu;
          const unsigned j0 = p0 >> 16, j1 = p1 >> 16, j2 = p2 >> 16, j3 = p3 >> 16;
          a0 += (kap0[i0] * g0) * D0(j0);
          a1 += (kap1[i0] * g0) * D1(j0);
          b0 += (kap0[i1] * g1) * D0(j1);
          b1 += (kap1[i1] * g1) * D1(j1);
          a0 += (kap0[i2] * g2) * D0(j2);
          a1 += (kap1[i2] * g2) * D1(j2);
          b0 += (kap0[i3] * g3) * D0(j3);
          b1 += (kap1[i3] * g3) * D1(j3);
        }
        for (; q < q1; ++q) {
          const unsigned pk = gpk_t[q];
          const T g = gv_t[q];
          const unsigned i = pk & 0xffffu, j = pk >> 16;
          a0 += (kap0[i] * g) * D0(j);
          a1 += (kap1[i] * g) * D1(j);
        }
        a0 += b0;
        a1 += b1;
        z0[kk] = live0 ? a0 : T(0);
        if (has1) z1[kk] = live1 ? a1 : T(0);
      }
    }
  }
  }
  __syncthreads();
  SG_MARK(3);
  // phase 3: outputs of the owned lines (p.q partial in FP64: the FP32 products of a correction
  // solve can be far below the FP32 normal range)
  double dsum = 0.0;
  constexpr int UB3 = 4;  // batched loads, as in phase 1
  const int nout = nlin * L * P;
  for (int e0 = threadIdx.x; e0 < nout; e0 += nt * UB3) {
    int cl[UB3], cbs[UB3];
    TO ad[UB3];
#pragma unroll
    for (int u = 0; u < UB3; ++u) {
      const int e = e0 + u * nt;
      cl[u] = 0;
      cbs[u] = 0;
      ad[u] = TO(0);
      if (e < nout) {
        const int nd = fdiv(e, op.fP), k = e - nd * P;
        const int t = fdiv(nd, op.fL), i = nd - t * L;
        const long long so = so0 + (long long)(lj0 + t) * L + i;
        cl[u] = op.cls[so];
        if (cm != T(0)) cbs[u] = op.cells[so];
        if (add) ad[u] = add[pb + ((long long)(lj0 + t) * L + i) * P + k];
      }
    }
#pragma unroll
    for (int u = 0; u < UB3; ++u) {
      const int e = e0 + u * nt;
      if (e >= nout) continue;
      const int nd = fdiv(e, op.fP), k = e - nd * P;
      const int t = fdiv(nd, op.fL), i = nd - t * L;
      const int lj = lj0 + t;
      const long long g = pb + ((long long)lj * L + i) * P + k;
      const int c = cl[u];
      TO out = TO(0);
      if ((out_mask >> c) & 1) {
        T acc = T(0);
        if (ck != T(0)) {
          T sz = T(0);
          if (i < L - 1) sz += zs[((size_t)t * (L - 1) + i) * PS + k];
          if (i > 0) sz -= zs[((size_t)t * (L - 1) + i - 1) * PS + k];
          sz += zs[((size_t)nE + (size_t)(t + 1) * L + i) * PS + k];
          sz -= zs[((size_t)nE + (size_t)t * L + i) * PS + k];
          acc += ck * sz;
        }
        if (cm != T(0)) {
          const int cb = cbs[u];
          T self = T(0), nbs = T(0);
          const long long dN_ = (long long)L * P;
          const T* xa = (FUSEDP || xm == xk) ? xs + ((size_t)(t + 1) * L + i) * P + k : xm + g;
          if (cb & 1) { self += T(4); nbs += T(2) * xa[-dN_ - P] + xa[-dN_] + xa[-P]; }
          if (cb & 2) { self += T(2); nbs += xa[-dN_] + xa[P]; }
          if (cb & 4) { self += T(2); nbs += xa[-P] + xa[dN_]; }
          if (cb & 8) { self += T(4); nbs += xa[P] + T(2) * xa[dN_ + P] + xa[dN_]; }
          acc += cm * op.mass_h * (self * xa[0] + nbs);
        }
        out = (TO)acc;
        if (add) out += ad[u];
        if constexpr (DOT32) dsf = fmaf(xs[((size_t)(t + 1) * L + i) * P + k] * dsc, (float)out * dsc, dsf);
        else if (DOT) dsum += (double)xs[((size_t)(t + 1) * L + i) * P + k] * (double)out;
      }
      y[g] = out;
    }
  }
  SG_MARK(4);
  if constexpr (DOT32) dsum = (double)dsf * f64_pow2(2 * dex);
  if (DOT) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = dsum;
    __syncthreads();
    if (w == 0) {
      dsum = l < (nt >> 5) ? red[l] : 0.0;
      for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
      if (l == 0) part_pq[(long long)b * NT + tile] = dsum;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Operator apply in float-float arithmetic (compiled triple-product table only):
//   y = add + cm (M (x) I) xm + ck (sum_i K_i (x) G_i) xk       on nodes with class in out_mask
// the operator of k_apply<double, double, false, false, C> with FP64 inputs and outputs.  The block's
// input lines are scaled by a power of two (its largest |xk| maps into [1/2, 1), so the FP32 exponent
// range of the pairs cannot flush small vectors) and staged as float-float pairs; each edge's
// differences, weights (float-float copies of the FP64 edge weights) and triple products combine by
// error-free transformations (about 2^-44 relative per operation, gflux_f2), and every output is formed
// in float-float, unscaled exactly and summed in FP64.  FP64 instructions issue at about 1/64 of the
// FP32 rate on this part: a float-float triple product costs about 16 FP32 operations, and the
// staging and output conversions work on the bit patterns with integer operations (f2_split_scaled,
// f32_to_f64_scaled).  A mass input xm other than xk is applied in FP64 from global memory.  Shared memory as the FP64 compiled variant:
// xs [(TL+2)][L][P] pairs, zs [edges][PS] pairs.
// ------------------------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(256, 2) k_apply_f2(Op<double> op, int nb, int R, int TL, int NT,
                                                  const double* __restrict__ xm, const double* __restrict__ xk,
                                                  double* y, const double* add, double cm, double ck, int out_mask,
                                                  const float2* __restrict__ kapE2, const float2* __restrict__ kapN2) {
  count_launch();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned red[32];
  const int P = op.P, L = op.L, nl = op.nl, PI = op.PI;
  const int PS = P | 1;
  const int b = blockIdx.x / NT, tile = blockIdx.x % NT;
  const int lj0 = tile * TL;
  const int nlin = min(TL, L - lj0);
  const int sub = b / R;
  const int nE = nlin * (L - 1), nNr = nlin + 1;
  const int nEd = nE + nNr * L;
  f2* xs = reinterpret_cast<f2*>(smem_raw);      // [(TL+2)][L][P] (FP64 values until the scale is known)
  double* xd = reinterpret_cast<double*>(smem_raw);
  f2* zs = xs + (size_t)(TL + 2) * L * P;        // [edges][PS]
  const long long pb = (long long)b * nl * P;
  const long long so0 = (long long)sub * nl;
  const int nt = blockDim.x;
  const bool same = xm == xk;
  // phase 1: input lines lj0-1 .. lj0+nlin (zeros outside the grid), loads in batches; the block's
  // largest binary exponent (integer maximum of the high words of |x|)
  constexpr int UB = 8;
  const int nin = (nlin + 2) * L * P;
  unsigned amax = 0u;
  for (int e0 = threadIdx.x; e0 < nin; e0 += nt * UB) {
    double v[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int e = e0 + u * nt;
      v[u] = 0.0;
      if (e < nin) {
        const int t = fdiv(e, op.fLP);
        const int jl = lj0 - 1 + t;
        if (jl >= 0 && jl < L) v[u] = xk[pb + (long long)jl * L * P + (e - t * L * P)];
      }
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int e = e0 + u * nt;
      if (e < nin) {
        xd[e] = v[u];
        amax = max(amax, (unsigned)__double2hiint(v[u]) & 0x7fffffffu);
      }
    }
  }
  amax = __reduce_max_sync(0xffffffffu, amax);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  amax = 0u;
  for (int w = 0; w < (nt >> 5); ++w) amax = max(amax, red[w]);
  // scale 2^-ex maps the largest |x| into [1/2, 1) (no scaling for an all-zero or subnormal block)
  const int ex = (amax >> 20) ? (int)(amax >> 20) - 1022 : 0;
  for (int e = threadIdx.x; e < nin; e += nt) xs[e] = f2_split_scaled(xd[e], ex);   // own elements
  __syncthreads();
  // phase 2: fluxes, one work item per (edge, output-mode group), the group uniform across a warp
  if (ck != 0.0) {
    const int nEd32 = (nEd + 31) & ~31;
    for (int it = threadIdx.x; it < nEd32 * C::KG; it += nt) {
      const int wi = it >> 5, g = wi % C::KG;
      const int ed = ((wi / C::KG) << 5) + (it & 31);
      if (ed >= nEd) continue;
      const f2* xa;
      const f2* xb;
      const float2* kp;
      bool live = true;
      if (ed < nE) {
        const int t = fdiv(ed, op.fLm1), c = ed - t * (L - 1);
        xa = xs + ((size_t)(t + 1) * L + c) * P;
        xb = xa + P;
        kp = kapE2 + (so0 + (long long)(lj0 + t) * L + c) * PI;
      } else {
        const int v = ed - nE, t = fdiv(v, op.fL), c = v - t * L;
        const int jb = lj0 - 1 + t;
        live = jb >= 0 && jb + 1 < L;
        xa = xs + ((size_t)t * L + c) * P;
        xb = xa + (size_t)L * P;
        kp = kapN2 + (so0 + (long long)max(jb, 0) * L + c) * PI;
      }
      gflux_f2<C>(g, kp, xa, xb, zs + (size_t)ed * PS, live);
    }
  }
  __syncthreads();
  // phase 3: outputs of the owned lines (the FP64 tests on the coefficients are made once)
  const f2 ckf = f2_from(ck), cmf = f2_from(cm * op.mass_h);
  const double cmd = cm * op.mass_h;
  const bool has_k = ck != 0.0, has_m = cm != 0.0, mass_f2 = has_m && same, mass_64 = has_m && !same;
  constexpr int UB3 = 4;
  const int nout = nlin * L * P;
  const long long dN_ = (long long)L * P;
  for (int e0 = threadIdx.x; e0 < nout; e0 += nt * UB3) {
    int cl[UB3], cbs[UB3];
    double ad[UB3];
#pragma unroll
    for (int u = 0; u < UB3; ++u) {
      const int e = e0 + u * nt;
      cl[u] = 0;
      cbs[u] = 0;
      ad[u] = 0.0;
      if (e < nout) {
        const int nd = fdiv(e, op.fP), k = e - nd * P;
        const int t = fdiv(nd, op.fL), i = nd - t * L;
        const long long so = so0 + (long long)(lj0 + t) * L + i;
        cl[u] = op.cls[so];
        if (has_m) cbs[u] = op.cells[so];
        if (add) ad[u] = add[pb + ((long long)(lj0 + t) * L + i) * P + k];
      }
    }
#pragma unroll
    for (int u = 0; u < UB3; ++u) {
      const int e = e0 + u * nt;
      if (e >= nout) continue;
      const int nd = fdiv(e, op.fP), k = e - nd * P;
      const int t = fdiv(nd, op.fL), i = nd - t * L;
      const long long g = pb + ((long long)(lj0 + t) * L + i) * P + k;
      double out = 0.0;
      if ((out_mask >> cl[u]) & 1) {
        f2 acc = {0.f, 0.f};
        if (has_k) {
          f2 sz = zs[((size_t)nE + (size_t)(t + 1) * L + i) * PS + k];
          sz = f2_sub(sz, zs[((size_t)nE + (size_t)t * L + i) * PS + k]);
          if (i < L - 1) sz = f2_add(sz, zs[((size_t)t * (L - 1) + i) * PS + k]);
          if (i > 0) sz = f2_sub(sz, zs[((size_t)t * (L - 1) + i - 1) * PS + k]);
          acc = f2_mul(ckf, sz);
        }
        const int cb = cbs[u];
        double md = 0.0;
        if (mass_f2) {
          const f2* xa = xs + ((size_t)(t + 1) * L + i) * P + k;
          auto twice = [](f2 a) -> f2 { return {2.f * a.h, 2.f * a.l}; };  // exact
          float self = 0.f;
          f2 nbs = {0.f, 0.f};
          if (cb & 1) { self += 4.f; nbs = f2_add(f2_add(f2_add(nbs, twice(xa[-dN_ - P])), xa[-dN_]), xa[-P]); }
          if (cb & 2) { self += 2.f; nbs = f2_add(f2_add(nbs, xa[-dN_]), xa[P]); }
          if (cb & 4) { self += 2.f; nbs = f2_add(f2_add(nbs, xa[-P]), xa[dN_]); }
          if (cb & 8) { self += 4.f; nbs = f2_add(f2_add(f2_add(nbs, xa[P]), twice(xa[dN_ + P])), xa[dN_]); }
          acc = f2_add(acc, f2_mul(cmf, f2_add(f2_mul({self, 0.f}, xa[0]), nbs)));
        } else if (mass_64) {
          const double* xa = xm + g;
          double self = 0.0, nbs = 0.0;
          if (cb & 1) { self += 4.0; nbs += 2.0 * xa[-dN_ - P] + xa[-dN_] + xa[-P]; }
          if (cb & 2) { self += 2.0; nbs += xa[-dN_] + xa[P]; }
          if (cb & 4) { self += 2.0; nbs += xa[-P] + xa[dN_]; }
          if (cb & 8) { self += 4.0; nbs += xa[P] + 2.0 * xa[dN_ + P] + xa[dN_]; }
          md = cmd * (self * xa[0] + nbs);
        }
        out = f32_to_f64_scaled(acc.h, ex) + f32_to_f64_scaled(acc.l, ex);
        if (mass_64) out += md;
        if (add) out += ad[u];
      }
      y[g] = out;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Mean-operator preconditioner fused with the inner CG update and control.
// A0 = cm M + ck K_0 on a pattern's free set is block tridiagonal over grid lines; the set-up
// stores S_j^{-1} (dense L x L) with S_0 = D_0, S_j = D_j - B_{j-1}^T S_{j-1}^{-1} B_{j-1};
// B_j couples (a, j) to (a, j+1) (Bd) and (a+1, j+1) (Bu).  Non-free nodes carry identity rows.
// Grid: nb * NG blocks (problem, group of G modes); block (L, G) threads.
//   init  : z = A0^{-1} r; partials r.z, r.r
//   iterate: alpha = rz / sum(pq partials); x += alpha p; r -= alpha q; z = A0^{-1} r;
//            partials r.z, r.r
// The last block to finish reduces the partials of every problem (fixed order), updates the
// per-problem scalars and convergence flags and sets the loop condition.
// ------------------------------------------------------------------------------------------
// async copy of one element (4 or 8 bytes) global -> shared (cp.async, Ampere and later)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (sizeof(T) == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc));
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc));
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Partials of r.z and r.r for block (b, grp), then the last block to finish reduces the
// partials of every problem (fixed order), updates the per-problem scalars and convergence flags
// and sets the loop condition.  Every block of the launch must call this exactly once.
__device__ __forceinline__ void line_control(double s_rz, double s_rr, int b, int grp, int NG, int NT, int nb,
                                             const CgCtl& ctl, int init, double tol2, double bb_min, int max_it,
                                             cudaGraphConditionalHandle cond_handle, int use_handle) {
  __shared__ double red_rz[32], red_rr[32];
  __shared__ int am_last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  for (int o = 16; o > 0; o >>= 1) {
    s_rz += __shfl_down_sync(0xffffffffu, s_rz, o);
    s_rr += __shfl_down_sync(0xffffffffu, s_rr, o);
  }
  if ((tid & 31) == 0) { red_rz[tid >> 5] = s_rz; red_rr[tid >> 5] = s_rr; }
  __syncthreads();
  if (tid == 0) {
    double a1 = 0.0, a2 = 0.0;
    for (int wdx = 0; wdx < (nthr + 31) / 32; ++wdx) { a1 += red_rz[wdx]; a2 += red_rr[wdx]; }
    ctl.part_rz[(long long)b * NG + grp] = a1;
    ctl.part_rr[(long long)b * NG + grp] = a2;
    __threadfence();
    const unsigned prev = atomicAdd(ctl.counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // control (last block): per-problem scalars, convergence, loop condition
  __shared__ int n_act;
  if (tid == 0) n_act = 0;
  __syncthreads();
  for (int bb = tid; bb < nb; bb += nthr) {
    double rz = 0.0, rr = 0.0;
    for (int g = 0; g < NG; ++g) {
      rz += ctl.part_rz[(long long)bb * NG + g];
      rr += ctl.part_rr[(long long)bb * NG + g];
    }
    if (init) {
      ctl.bb[bb] = rr;
      ctl.rz[bb] = rz;
      ctl.beta[bb] = 0.0;
      if (!isfinite(rr) || !isfinite(rz)) ctl.breakdown[0] = 1;
      const int ac = rr > bb_min && isfinite(rr) && rz > 0.0;
      ctl.active[bb] = ac;
      if (ac) atomicAdd(&n_act, 1);
    } else if (ctl.active[bb]) {
      double pq = 0.0;
      for (int t = 0; t < NT; ++t) pq += ctl.part_pq[(long long)bb * NT + t];
      if (!isfinite(rr) || !isfinite(rz)) ctl.breakdown[0] = 1;
      const bool stop = !(pq > 0.0) || !isfinite(pq) || !isfinite(rr) || !(rz > 0.0);
      const bool conv = stop || !(rr > tol2 * ctl.bb[bb]);
      if (conv) {
        ctl.active[bb] = 0;
      } else {
        ctl.beta[bb] = rz / ctl.rz[bb];
        ctl.rz[bb] = rz;
        atomicAdd(&n_act, 1);
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    int itn = init ? 0 : (*ctl.it + 1);
    *ctl.it = itn;
    if (!init) {
      *ctl.it_total += 1;
      *ctl.parity ^= 1;
    } else {
      *ctl.parity = 0;
    }
    const int cond = (n_act > 0) && (itn < max_it);
    *ctl.cond = cond;
    *ctl.counter = 0u;
    if (use_handle) cudaGraphSetConditional(cond_handle, cond ? 1u : 0u);
  }
}

// GS: the factor is read from global memory instead of being staged, and so is the residual
// (subdomains too wide for the factor buffers and both slices); only the solution slice stays in
// shared memory.  S_j^{-1} is symmetric, so row a is read as column a, which makes the accesses of
// consecutive threads (consecutive a) contiguous.
template <typename T, bool GS = false>
__global__ void k_line(int L, int nl, int P, int R, int NG, int NT, long long pat_stride,
                       const T* __restrict__ Sinv, const T* __restrict__ Bd, const T* __restrict__ Bu, int nb,
                       T* __restrict__ x, T* __restrict__ r, T* __restrict__ z, T* pbuf0, T* pbuf1,
                       const T* __restrict__ q, CgCtl ctl, int init, double tol2, double bb_min, int max_it,
                       cudaGraphConditionalHandle cond_handle, int use_handle) {
  count_launch();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = blockDim.x;                      // modes of the block (fast index)
  const int LL = L * L;
  T* Sb = reinterpret_cast<T*>(smem_raw);        // [2][L][L] double-buffered S_j^{-1} (not with GS)
  T* rs = GS ? Sb : Sb + 2 * LL;                 // [L lines][L][G] residual slice (not with GS)
  T* ys = GS ? rs : rs + (size_t)LL * G;         // [L lines][L][G] solution slice
  T* w = ys + (size_t)LL * G;                    // [L][G]
  const int b = blockIdx.x / NG, grp = blockIdx.x % NG;
  const int m = threadIdx.x, a = threadIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  const int k = grp * G + m;
  const bool ok = (a < L) && (k < P);
  const bool act = init ? true : (ctl.active[b] != 0);
  double s_rz = 0.0, s_rr = 0.0;
  if (act) {
    const int sub = b / R;
    const T* S = Sinv + (long long)sub * pat_stride;
    const T* bd = Bd + (long long)sub * LL;
    const T* bu = Bu + (long long)sub * LL;
    const long long base = (long long)b * nl * P;
    const int kb = grp * G;
    const int gl = min(G, P - kb);  // modes of this block
    // prefetch S_0^{-1} while the CG update runs
    if (!GS) {
      for (int e = tid; e < LL; e += nthr) cp_async_elem(Sb + e, S + e);
      cp_async_commit();
    }
    // phase A (parallel over the block's slice): x += alpha p, r -= alpha q, stage r
    T alpha = T(0);
    const T* pc = nullptr;
    if (!init) {
      double pq = 0.0;
      for (int t = 0; t < NT; ++t) pq += ctl.part_pq[(long long)b * NT + t];
      // a vanishing or non-finite p.q (right-hand side at the underflow level of T) freezes the
      // problem at its current iterate; the control step below then retires it
      const double al = (pq > 0.0 && isfinite(pq)) ? ctl.rz[b] / pq : 0.0;
      alpha = isfinite(al) ? (T)al : T(0);
      pc = (*ctl.parity) ? pbuf0 : pbuf1;  // p_new written by the apply kernel
    }
    const FD fgl = make_fd((unsigned)gl);
    for (int e = tid; e < LL * gl; e += nthr) {
      const int node = fdiv(e, fgl), mm = e - node * gl;
      const long long o = base + (long long)node * P + kb + mm;
      T rv = r[o];
      if (!init) {
        x[o] += alpha * pc[o];
        rv -= alpha * q[o];
        r[o] = rv;
      }
      if (!GS) rs[(size_t)node * G + mm] = rv;
    }
    __syncthreads();
    // residual of line j, position a, mode m of the block (shared slice, or global with GS)
    auto rval = [&](int node, int mm) -> T {
      if (GS) return r[base + (long long)node * P + kb + mm];
      return rs[(size_t)node * G + mm];
    };
    // phase B: forward sweep y_j = S_j^{-1} (r_j - B_{j-1}^T y_{j-1}) in shared memory
    for (int j = 0; j < L; ++j) {
      if (!GS) {
        if (j + 1 < L) {
          const T* src = S + (long long)(j + 1) * LL;
          T* dst = Sb + ((j + 1) & 1) * LL;
          for (int e = tid; e < LL; e += nthr) cp_async_elem(dst + e, src + e);
        }
        cp_async_commit();
      }
      if (ok) {
        T rhs = rval(j * L + a, m);
        if (j > 0) {
          const T* yp = ys + (size_t)(j - 1) * L * G;
          rhs -= bd[(j - 1) * L + a] * yp[a * G + m];
          if (a > 0) rhs -= bu[(j - 1) * L + a - 1] * yp[(a - 1) * G + m];
        }
        w[a * G + m] = rhs;
      }
      if (!GS) cp_async_wait1();   // S_j^{-1} has landed (the newest group may still be in flight)
      __syncthreads();
      if (ok) {
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        if (GS) {
          const T* Sj = S + (long long)j * LL + a;  // column a of the symmetric S_j^{-1}
          int c = 0;
          for (; c + 3 < L; c += 4) {
            s0 += Sj[(size_t)c * L] * w[c * G + m];
            s1 += Sj[(size_t)(c + 1) * L] * w[(c + 1) * G + m];
            s2 += Sj[(size_t)(c + 2) * L] * w[(c + 2) * G + m];
            s3 += Sj[(size_t)(c + 3) * L] * w[(c + 3) * G + m];
          }
          for (; c < L; ++c) s0 += Sj[(size_t)c * L] * w[c * G + m];
        } else {
          const T* Sj = Sb + (j & 1) * LL + a * L;
          int c = 0;
          for (; c + 3 < L; c += 4) {
            s0 += Sj[c] * w[c * G + m];
            s1 += Sj[c + 1] * w[(c + 1) * G + m];
            s2 += Sj[c + 2] * w[(c + 2) * G + m];
            s3 += Sj[c + 3] * w[(c + 3) * G + m];
          }
          for (; c < L; ++c) s0 += Sj[c] * w[c * G + m];
        }
        ys[((size_t)j * L + a) * G + m] = (s0 + s1) + (s2 + s3);
      }
      __syncthreads();
    }
    if (!GS) cp_async_wait0();
    __syncthreads();
    // phase C: backward sweep x_j = y_j - S_j^{-1} B_j x_{j+1} in place in ys
    if (!GS) {
      if (L >= 2) {
        const T* src = S + (long long)(L - 2) * LL;
        for (int e = tid; e < LL; e += nthr) cp_async_elem(Sb + ((L - 2) & 1) * LL + e, src + e);
      }
      cp_async_commit();
    }
    for (int j = L - 2; j >= 0; --j) {
      if (!GS) {
        if (j - 1 >= 0) {
          const T* src = S + (long long)(j - 1) * LL;
          T* dst = Sb + ((j - 1) & 1) * LL;
          for (int e = tid; e < LL; e += nthr) cp_async_elem(dst + e, src + e);
        }
        cp_async_commit();
      }
      if (ok) {
        const T* xn = ys + (size_t)(j + 1) * L * G;
        T tv = bd[j * L + a] * xn[a * G + m];
        if (a + 1 < L) tv += bu[j * L + a] * xn[(a + 1) * G + m];
        w[a * G + m] = tv;
      }
      if (!GS) cp_async_wait1();
      __syncthreads();
      if (ok) {
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        if (GS) {
          const T* Sj = S + (long long)j * LL + a;
          int c = 0;
          for (; c + 3 < L; c += 4) {
            s0 += Sj[(size_t)c * L] * w[c * G + m];
            s1 += Sj[(size_t)(c + 1) * L] * w[(c + 1) * G + m];
            s2 += Sj[(size_t)(c + 2) * L] * w[(c + 2) * G + m];
            s3 += Sj[(size_t)(c + 3) * L] * w[(c + 3) * G + m];
          }
          for (; c < L; ++c) s0 += Sj[(size_t)c * L] * w[c * G + m];
        } else {
          const T* Sj = Sb + (j & 1) * LL + a * L;
          int c = 0;
          for (; c + 3 < L; c += 4) {
            s0 += Sj[c] * w[c * G + m];
            s1 += Sj[c + 1] * w[(c + 1) * G + m];
            s2 += Sj[c + 2] * w[(c + 2) * G + m];
            s3 += Sj[c + 3] * w[(c + 3) * G + m];
          }
          for (; c < L; ++c) s0 += Sj[c] * w[c * G + m];
        }
        ys[((size_t)j * L + a) * G + m] -= (s0 + s1) + (s2 + s3);
      }
      __syncthreads();
    }
    if (!GS) cp_async_wait0();
    // phase D (parallel): write z, partial r.z and r.r
    for (int e = tid; e < LL * gl; e += nthr) {
      const int node = fdiv(e, fgl), mm = e - node * gl;
      const T zv = ys[(size_t)node * G + mm];
      const double rv = (double)rval(node, mm);
      z[base + (long long)node * P + kb + mm] = zv;
      s_rz += rv * (double)zv;
      s_rr += rv * rv;
    }
  }
  line_control(s_rz, s_rr, b, grp, NG, NT, nb, ctl, init, tol2, bb_min, max_it, cond_handle, use_handle);
}

// Mean-operator line solve fused with the inner CG update, warp-team form (FP32, small L):
// the whole factor {S_j^{-1}} of the subdomain (L^3 values) and the coupling coefficients are
// staged in shared memory once; each PCE mode is swept by its own team of ceil(L/32) warps that
// synchronises with a named barrier (or __syncwarp), so the 2L sequential line steps of
// different modes never wait on one another.
// 16-byte async copy global -> shared (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc));
}

// Fully unrolled dot of a zero-padded row (length LS, 16-byte aligned) with a broadcast vector.
template <typename T, int LS>
__device__ __forceinline__ T row_dot(const T* __restrict__ row, const T* __restrict__ w) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  if constexpr (sizeof(T) == 4) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    const float4* w4 = reinterpret_cast<const float4*>(w);
#pragma unroll
    for (int c = 0; c < LS / 4; ++c) {
      const float4 a = r4[c], b = w4[c];
      s0 += a.x * b.x;
      s1 += a.y * b.y;
      s2 += a.z * b.z;
      s3 += a.w * b.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < LS; c += 4) {
      s0 += row[c] * w[c];
      s1 += row[c + 1] * w[c + 1];
      s2 += row[c + 2] * w[c + 2];
      s3 += row[c + 3] * w[c + 3];
    }
  }
  return (s0 + s1) + (s2 + s3);
}

template <typename T, int LS>
__global__ void k_line_team(int L, int nl, int P, int R, int NG, int NT, int G, long long pat_stride,
                            const T* __restrict__ Sinv, const T* __restrict__ Bd, const T* __restrict__ Bu, int nb,
                            T* __restrict__ x, T* __restrict__ r, T* __restrict__ z, T* pbuf0, T* pbuf1,
                            const T* __restrict__ q, CgCtl ctl, int init, double tol2, double bb_min, int max_it,
                            cudaGraphConditionalHandle cond_handle, int use_handle) {
  count_launch();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LL = L * L;
  const int W = (L + 31) >> 5;                   // warps per team
  T* Ss = reinterpret_cast<T*>(smem_raw);        // [L][L][LS] rows zero-padded to LS
  T* bds = Ss + (size_t)LL * LS;                 // [L][L]
  T* bus = bds + LL;                             // [L][L]
  T* team_base = Ss + (size_t)LL * LS + ((2 * LL + 3) & ~3);  // per team: w [LS], rs [LL], ys [LL]
  const int tstride = LS + 2 * LL + ((4 - ((2 * LL) & 3)) & 3);  // keeps every w 16-byte aligned
  const int b = blockIdx.x / NG, grp = blockIdx.x % NG;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int team = warp / W;
  const int a = (warp % W) * 32 + lane;          // row (node along the line)
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  const int kb = grp * G;
  const int gl = min(G, P - kb);
  const bool tok = team < gl;
  const bool act = init ? true : (ctl.active[b] != 0);
  double s_rz = 0.0, s_rr = 0.0;
  if (act) {
    const int sub = b / R;
    const T* S = Sinv + (long long)sub * pat_stride;  // padded layout [L][L][LS]
    const T* bd = Bd + (long long)sub * LL;
    const T* bu = Bu + (long long)sub * LL;
    const long long base = (long long)b * nl * P;
    for (int e = tid; e < LL * LS / 4; e += nthr) cp_async16(Ss + 4 * e, S + 4 * e);
    for (int e = tid; e < LL; e += nthr) {
      cp_async_elem(bds + e, bd + e);
      cp_async_elem(bus + e, bu + e);
    }
    cp_async_commit();
    // phase A: CG update of the block's modes, residual staged per team
    T alpha = T(0);
    const T* pc = nullptr;
    if (!init) {
      double pq = 0.0;
      for (int t = 0; t < NT; ++t) pq += ctl.part_pq[(long long)b * NT + t];
      const double al = (pq > 0.0 && isfinite(pq)) ? ctl.rz[b] / pq : 0.0;
      alpha = isfinite(al) ? (T)al : T(0);
      pc = (*ctl.parity) ? pbuf0 : pbuf1;
    }
    const FD fgl = make_fd((unsigned)gl);
    for (int e = tid; e < LL * gl; e += nthr) {
      const int node = fdiv(e, fgl), mm = e - node * gl;
      const long long o = base + (long long)node * P + kb + mm;
      T rv = r[o];
      if (!init) {
        x[o] += alpha * pc[o];
        rv -= alpha * q[o];
        r[o] = rv;
      }
      team_base[(size_t)mm * tstride + LS + node] = rv;
    }
    cp_async_wait0();
    __syncthreads();
    if (tok) {
      T* w = team_base + (size_t)team * tstride;
      T* rs = w + LS;
      T* ys = rs + LL;
      if (a < LS && a >= L) w[a] = T(0);
      auto tsync = [&]() {
        if (W == 1) __syncwarp();
        else asm volatile("bar.sync %0, %1;\n" ::"r"(team + 1), "r"(W * 32) : "memory");
      };
      const bool ok = a < L;
      for (int j = 0; j < L; ++j) {
        if (ok) {
          T rhs = rs[j * L + a];
          if (j > 0) {
            rhs -= bds[(j - 1) * L + a] * ys[(j - 1) * L + a];
            if (a > 0) rhs -= bus[(j - 1) * L + a - 1] * ys[(j - 1) * L + a - 1];
          }
          w[a] = rhs;
        }
        tsync();
        if (ok) ys[j * L + a] = row_dot<T, LS>(Ss + ((size_t)j * L + a) * LS, w);
        tsync();
      }
      for (int j = L - 2; j >= 0; --j) {
        if (ok) {
          T tv = bds[j * L + a] * ys[(j + 1) * L + a];
          if (a + 1 < L) tv += bus[j * L + a] * ys[(j + 1) * L + a + 1];
          w[a] = tv;
        }
        tsync();
        if (ok) ys[j * L + a] -= row_dot<T, LS>(Ss + ((size_t)j * L + a) * LS, w);
        tsync();
      }
    }
    __syncthreads();
    // phase D: write z, partial r.z and r.r
    for (int e = tid; e < LL * gl; e += nthr) {
      const int node = fdiv(e, fgl), mm = e - node * gl;
      const T* rs = team_base + (size_t)mm * tstride + LS;
      const T zv = rs[LL + node];
      const double rv = (double)rs[node];
      z[base + (long long)node * P + kb + mm] = zv;
      s_rz += rv * (double)zv;
      s_rr += rv * rv;
    }
  }
  line_control(s_rz, s_rr, b, grp, NG, NT, nb, ctl, init, tol2, bb_min, max_it, cond_handle, use_handle);
}

// Mean-operator line solve fused with the inner CG update, register-tiled form for wide subdomains
// (one block per (problem, group of G modes); with G = P the factor of a subdomain is streamed once
// per sweep).  Per line step the block forms Y = S_j^{-1} W for all L rows and its G modes; thread
// (rt, mt) accumulates the 2 x 4 tile rows 2 rt, 2 rt + 1, modes 4 mt .. 4 mt + 3 in registers (two
// accumulator sets, even and odd c, so consecutive multiply-adds never wait on one another).
// Because S_j^{-1} is symmetric, row c of the stored factor holds column c, so the two factor
// values of a tile for one c are one vector load, as are the four modes of W.  The factor is
// stored with rows padded to LSP = 4 ceil(L / 4) values (zeros beyond L) and double-buffered by
// 16-byte cp.async together with the coupling rows B_j.  Global vectors move in row order: thread t
// keeps mode t mod G and visits rows t / G, t / G + RPI, ... (RPI = threads / G rows per pass), so a
// line is read and written contiguously; the next line is prefetched into registers while the
// current one is multiplied.  The forward sweep keeps y_j in shared memory for one step and parks
// it in z; the backward sweep reads it back.  r . z = r^T A0^{-1} r is formed in the forward sweep as
// sum_j w_j . y_j (block LDL^T: A0^{-1} = L^{-T} D^{-1} L^{-1}, w = L^{-1} r, y = D^{-1} w), so the
// backward sweep needs no residual.  Shared memory: Sb [2][L][LSP], Ws [L][GS], Ys [L][GS],
// Yp [LSP][GS], Bs [3][2][L] (GS = G rounded up to a multiple of 4).  The factor of line j is copied
// one step ahead (double buffer) and the coupling row j two steps ahead (three slots): the step that
// uses either reads it only after a cp.async wait and a barrier that cover its copy.
// One line product acc = S_j-tile x W over c = 0 .. L-1 (rows r0, r0 + 1 of the tile from row c of the
// stored symmetric factor, four modes of W); even and odd c accumulate separately.
template <typename T>
__device__ __forceinline__ void tile_product(T (&acc)[2][4], const T* __restrict__ Sj, const T* __restrict__ Wc,
                                             int L, int LSP, int GS) {
  using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  T acc2[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc2[i][k] = T(0);
  auto ld4 = [](const T* p, T (&w)[4]) {
    if constexpr (sizeof(T) == 4) {
      const float4 v = *reinterpret_cast<const float4*>(p);
      w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else {
      const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 2);
      w[0] = v0.x; w[1] = v0.y; w[2] = v1.x; w[3] = v1.y;
    }
  };
  int c = 0;
#pragma unroll 2
  for (; c + 1 < L; c += 2) {
    const V2 s0 = *reinterpret_cast<const V2*>(Sj + c * LSP);
    const V2 s1 = *reinterpret_cast<const V2*>(Sj + (c + 1) * LSP);
    T w0[4], w1[4];
    ld4(Wc + c * GS, w0);
    ld4(Wc + (c + 1) * GS, w1);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[0][k] = fma(s0.x, w0[k], acc[0][k]);
      acc[1][k] = fma(s0.y, w0[k], acc[1][k]);
      acc2[0][k] = fma(s1.x, w1[k], acc2[0][k]);
      acc2[1][k] = fma(s1.y, w1[k], acc2[1][k]);
    }
  }
  if (c < L) {
    const V2 s0 = *reinterpret_cast<const V2*>(Sj + c * LSP);
    T w0[4];
    ld4(Wc + c * GS, w0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[0][k] = fma(s0.x, w0[k], acc[0][k]);
      acc[1][k] = fma(s0.y, w0[k], acc[1][k]);
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[i][k] += acc2[i][k];
}


// rows per thread and line of the row-ordered line I/O: four arrays of them stay in registers
template <typename T>
__host__ __device__ constexpr int lw_npf() { return 8; }
constexpr int LW_MAXT = 256;  // threads per block of k_line_w
template <typename T>
__host__ __device__ constexpr int lw_minb() { return sizeof(T) == 4 ? 2 : 1; }  // blocks per SM (register budget)

template <typename T>
__global__ void __launch_bounds__(LW_MAXT, lw_minb<T>()) k_line_w(int L, int LSP, int nl, int P, int R, int NG, int NT, int G, int GS,
                                                    long long pat_stride, const T* __restrict__ Spad,
                                                    const T* __restrict__ Bd, const T* __restrict__ Bu, int nb,
                                                    T* __restrict__ x, T* __restrict__ r, T* __restrict__ z, T* pbuf0,
                                                    T* pbuf1, const T* __restrict__ q, CgCtl ctl, int init, double tol2,
                                                    double bb_min, int max_it, cudaGraphConditionalHandle cond_handle,
                                                    int use_handle) {
  count_launch();
  constexpr int NPF = lw_npf<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T alpha_s;
  const int LLS = L * LSP;
  T* Sb = reinterpret_cast<T*>(smem_raw);  // [2][L][LSP]
  T* Ws = Sb + 2 * LLS;                    // [L][GS]
  T* Ys = Ws + L * GS;                     // [L][GS]
  T* Yp = Ys + L * GS;                     // [LSP][GS]
  T* Bs = Yp + LSP * GS;                   // [3][2][L]: coupling row r in slot r % 3 (Bd, then Bu)
  const int b = blockIdx.x / NG, grp = blockIdx.x % NG;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int NMT = GS >> 2, NRT = LSP >> 1;
  const int mt = tid % NMT, rt = tid / NMT;
  const bool worker = rt < NRT;
  const int a0 = rt * 2, m0 = mt * 4;
  const int kb = grp * G;
  const int gl = min(G, P - kb);
  // row-ordered I/O: fixed mode io_m, rows io_a + kk * RPI
  const int RPI = nthr / gl;
  const int io_m = tid % gl, io_a = tid / gl;
  const bool io_on = io_a < RPI;
  const int LP = L * P;
  const int rstep = RPI * P, sstep = RPI * GS;
  const bool act = init ? true : (ctl.active[b] != 0);
  double s_rz = 0.0, s_rr = 0.0;
  XAcc x_rz, x_rr;  // FP32 per-thread totals over the launch's steps
  if (act) {
    const int sub = b / R;
    const T* S = Spad + (long long)sub * pat_stride;
    const T* bd = Bd + (long long)sub * L * L;
    const T* bu = Bu + (long long)sub * L * L;
    const long long base = (long long)b * nl * P + kb + io_m;  // + (j L + a) P for element (j, a)
    T* rb = r + base;
    T* xb = x + base;
    T* zb = z + base;
    const T* qb = q + base;
    auto copy_line = [&](int j) {  // S_j^{-1} -> Sb[j & 1] (16-byte pieces)
      const int4* src = reinterpret_cast<const int4*>(S + (long long)j * LLS);
      int4* dst = reinterpret_cast<int4*>(Sb + (j & 1) * LLS);
      const int n16 = LLS * (int)sizeof(T) / 16;
      for (int e = tid; e < n16; e += nthr) cp_async16(dst + e, src + e);
    };
    auto copy_coupling = [&](int row) {  // Bd, Bu of line `row` -> slot row % 3
      T* dst = Bs + (row % 3) * 2 * L;
      for (int e = tid; e < 2 * L; e += nthr)
        cp_async_elem(dst + e, e < L ? bd + (long long)row * L + e : bu + (long long)row * L + (e - L));
    };
    copy_line(0);
    if (L >= 2) copy_coupling(0);
    cp_async_commit();
    for (int e = tid; e < L * GS; e += nthr) Ws[e] = T(0);
    for (int e = tid; e < LSP * GS; e += nthr) Yp[e] = T(0);
    const T* pb = nullptr;
    if (!init) {
      pb = ((*ctl.parity) ? pbuf0 : pbuf1) + base;  // p_new written by the apply kernel
      if (tid < 32) {
        double pq = 0.0;
        for (int t = tid; t < NT; t += 32) pq += ctl.part_pq[(long long)b * NT + t];
        for (int o = 16; o > 0; o >>= 1) pq += __shfl_down_sync(0xffffffffu, pq, o);
        if (tid == 0) {
          // a vanishing or non-finite p.q freezes the problem at its current iterate; the control
          // step below then retires it
          const double al = (pq > 0.0 && isfinite(pq)) ? ctl.rz[b] / pq : 0.0;
          alpha_s = isfinite(al) ? (T)al : T(0);
        }
      }
    }
    T pr_r[NPF], pr_q[NPF], pr_p[NPF], pr_x[NPF];
    auto fetch = [&](int j) {
      if (!io_on) return;
      const int o0 = j * LP + io_a * P;
#pragma unroll
      for (int kk = 0; kk < NPF; ++kk) {
        if (io_a + kk * RPI < L) {
          const int o = o0 + kk * rstep;
          pr_r[kk] = rb[o];
          if (!init) { pr_q[kk] = qb[o]; pr_p[kk] = pb[o]; pr_x[kk] = xb[o]; }
        }
      }
    };
    fetch(0);
    __syncthreads();
    const T alpha = init ? T(0) : alpha_s;
    // ---- forward sweep: y_j = S_j^{-1} (r_j - B_{j-1}^T y_{j-1}) ----
    for (int j = 0; j < L; ++j) {
      if (io_on) {
        const T* cb = Bs + ((j + 2) % 3) * 2 * L;  // coupling row j - 1
        const int o0 = j * LP + io_a * P;
        const int s0 = io_a * GS + io_m;
        T amax = T(0);
        T rr = T(0);
#pragma unroll
        for (int kk = 0; kk < NPF; ++kk) {
          const int a = io_a + kk * RPI;
          if (a < L) {
            const int o = o0 + kk * rstep, si = s0 + kk * sstep;
            T rv = pr_r[kk];
            if (!init) {
              rv -= alpha * pr_q[kk];
              rb[o] = rv;
              xb[o] = pr_x[kk] + alpha * pr_p[kk];
            }
            amax = max(amax, abs(rv));
            if constexpr (sizeof(T) == 8) rr = fma(rv, rv, rr);
            pr_r[kk] = rv;  // for the scaled FP32 partial below
            T wv = rv;
            if (j > 0) {
              const T yp = Yp[si];
              wv -= cb[a] * yp;
              if (a > 0) wv -= cb[L + a - 1] * Yp[si - GS];
              zb[o - LP] = yp;  // y_{j-1} parked in z
            }
            Ws[si] = wv;
          }
        }
        if constexpr (sizeof(T) == 8) {
          s_rr += (double)rr;
        } else {
          const int e = f32_exp((float)amax);
          const float sc = f32_pow2(-e);
          float rs = 0.f;
#pragma unroll
          for (int kk = 0; kk < NPF; ++kk)
            if (io_a + kk * RPI < L) {
              const float v = (float)pr_r[kk] * sc;
              rs = fmaf(v, v, rs);
            }
          x_rr.add(rs, 2 * e);
        }
      }
      // line j + 1 (used by this sweep's next step) and coupling row j + 1 (used by the input
      // phase two steps on, after the next step's wait and barrier)
      if (j + 1 < L) copy_line(j + 1);
      if (j + 1 <= L - 2) copy_coupling(j + 1);
      cp_async_commit();
      if (j + 1 < L) fetch(j + 1);
      cp_async_wait1();
      __syncthreads();
      if (worker) {
        T acc[2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[i][k] = T(0);
        const T* Sj = Sb + (j & 1) * LLS + a0;
        const T* Wc = Ws + m0;
        tile_product(acc, Sj, Wc, L, LSP, GS);
        T rz = T(0), awm = T(0), aym = T(0), wt[2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int a = a0 + i;
            Yp[a * GS + m0 + k] = acc[i][k];
            wt[i][k] = a < L ? Ws[a * GS + m0 + k] : T(0);  // zero for modes beyond the block's
            if constexpr (sizeof(T) == 8) rz = fma(wt[i][k], acc[i][k], rz);
            awm = max(awm, abs(wt[i][k]));
            aym = max(aym, a < L ? abs(acc[i][k]) : T(0));
          }
        if constexpr (sizeof(T) == 8) {
          s_rz += (double)rz;
        } else {
          const int ew = f32_exp((float)awm), ey = f32_exp((float)aym);
          const float sw = f32_pow2(-ew), sy = f32_pow2(-ey);
          float rs = 0.f;
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) rs = fmaf((float)wt[i][k] * sw, (float)acc[i][k] * sy, rs);
          x_rz.add(rs, ew + ey);
        }
      }
      __syncthreads();
    }
    // ---- backward sweep: x_j = y_j - S_j^{-1} B_j x_{j+1} (x_{L-1} = y_{L-1} is in Yp) ----
    // y_j is read back by the thread that parked it (same row order); S_{L-2} and coupling rows
    // L - 2 and L - 3 are still in their buffers (the forward sweep loaded nothing after them)
    T pr_y[NPF];
    auto fetch_y = [&](int j) {
      if (!io_on) return;
      const int o0 = j * LP + io_a * P;
#pragma unroll
      for (int kk = 0; kk < NPF; ++kk)
        if (io_a + kk * RPI < L) pr_y[kk] = zb[o0 + kk * rstep];
    };
    if (L >= 2) fetch_y(L - 2);
    for (int j = L - 2; j >= 0; --j) {
      if (io_on) {
        const T* cb = Bs + (j % 3) * 2 * L;  // coupling row j
        const int o0 = j * LP + io_a * P;
        const int s0 = io_a * GS + io_m;
#pragma unroll
        for (int kk = 0; kk < NPF; ++kk) {
          const int a = io_a + kk * RPI;
          if (a < L) {
            const int o = o0 + kk * rstep, si = s0 + kk * sstep;
            const T xn = Yp[si];
            T tv = cb[a] * xn;
            if (a + 1 < L) tv += cb[L + a] * Yp[si + GS];
            zb[o + LP] = xn;  // x_{j+1} final
            Ws[si] = tv;
            Ys[si] = pr_y[kk];
          }
        }
      }
      if (j >= 1) copy_line(j - 1);
      if (j >= 2) copy_coupling(j - 2);
      cp_async_commit();
      if (j >= 1) fetch_y(j - 1);
      cp_async_wait1();
      __syncthreads();
      if (worker) {
        T acc[2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[i][k] = T(0);
        const T* Sj = Sb + (j & 1) * LLS + a0;
        const T* Wc = Ws + m0;
        tile_product(acc, Sj, Wc, L, LSP, GS);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int a = a0 + i;
            Yp[a * GS + m0 + k] = a < L ? Ys[a * GS + m0 + k] - acc[i][k] : T(0);
          }
      }
      __syncthreads();
    }
    cp_async_wait0();
    // x_0
    if (io_on) {
      const int s0 = io_a * GS + io_m;
      const int o0 = io_a * P;
#pragma unroll
      for (int kk = 0; kk < NPF; ++kk)
        if (io_a + kk * RPI < L) zb[o0 + kk * rstep] = Yp[s0 + kk * sstep];
    }
  }
  if constexpr (sizeof(T) == 4) {
    s_rz += x_rz.value();
    s_rr += x_rr.value();
  }
  line_control(s_rz, s_rr, b, grp, NG, NT, nb, ctl, init, tol2, bb_min, max_it, cond_handle, use_handle);
}

// ------------------------------------------------------------------------------------------
// Line sweeps of the mean-operator preconditioner with the per-line products on the tensor cores
// (FP32 subdomain CG; subdomains of 41 .. 65 nodes per side; at most 32 modes per block).  The same
// sweeps, fused CG update and control as k_line_w; the product y = S_j^{-1} w of each line step is one
// tcgen05.mma chain (M = 128, N = 2 NB, K = 4 x 16):
//   A = S_j^{-1} in BF16, rows a < L and columns c < 64, K-major with the 128-byte swizzle (image of
//       the symmetrised FP64 factor, fetched by TMA into one of two stages);
//   B = [w_hi; w_lo]: w split into two BF16 terms (about 17 significant bits), written by the input
//       phase in the same swizzled layout (modes beyond the block's and rows c >= L stay zero);
//   D = 128 TMEM lanes x 2 NB FP32 columns; the epilogue adds the two column blocks.
// For L = 65 the column c = 64 enters as an FP32 rank-one update with the BF16-rounded values of the
// same symmetric image (col).  Rounding S_j^{-1} to BF16 is a fixed, symmetric perturbation of the
// preconditioner; w keeps about 17 bits per application (the precision design of k_pre_mma).
// Per step: input phase (all threads) -> proxy fence, barrier -> thread 0 waits for the stage's TMA,
// issues the four MMAs and commits -> warps 0-3 (row a = 32 warp + lane) wait for the commit, read
// the accumulator and finish the step -> barrier.  Thread 0 issues the next step's TMA at the start of
// each step.  Every wait is bounded (1 s); on a timeout the block records 20 + where in
// ctl.breakdown, stops its sweep, waits (bounded) for its copies in flight and frees its TMEM.
// Shared memory (1024-aligned): A [2][128][64] BF16, B [2 NB][64] BF16, col [2][68], Ws, Ys, Yp
// [L][WS] FP32 (WS = odd row stride >= G), the subdomain's coupling rows Bd, Bu [L][L] FP32.
// ------------------------------------------------------------------------------------------
constexpr int LTC_ABYTES = 128 * 128;  // one A stage: 128 rows x 64 BF16
constexpr int LTC_COLN = 68;           // FP32 values of one column stage (65 used; 272 bytes)
__host__ __device__ constexpr int ltc_ws(int G) { return G | 1; }
__host__ __device__ constexpr size_t ltc_smem(int L, int G, int NB) {
  return 1024 + 2 * (size_t)LTC_ABYTES + (size_t)2 * NB * 128 + 2 * LTC_COLN * 4 + 3 * (size_t)L * ltc_ws(G) * 4 +
         2 * (size_t)L * L * 4;
}

template <int NB>
__global__ void __maxnreg__(168) k_line_tc(const __grid_constant__ CUtensorMap tmS, int L, int nl, int P,
                                                    int R, int NG, int NT, int G, long long img_row0,
                                                    const float* __restrict__ col, const float* __restrict__ Bd,
                                                    const float* __restrict__ Bu, int nb, float* __restrict__ x,
                                                    float* __restrict__ r, float* __restrict__ z, float* pbuf0,
                                                    float* pbuf1, const float* __restrict__ q, CgCtl ctl, int init,
                                                    double tol2, double bb_min, int max_it,
                                                    cudaGraphConditionalHandle cond_handle, int use_handle) {
  count_launch();
  constexpr int NPF = 8;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[3];  // full[0], full[1], mma done
  __shared__ unsigned tmem_slot;
  __shared__ float alpha_s;
  __shared__ int s_abort;
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* As = sm;                                        // [2][128 x 128 B]
  unsigned char* Bt = sm + 2 * LTC_ABYTES;                       // [2 NB x 128 B]
  float* cols = reinterpret_cast<float*>(Bt + 2 * NB * 128);     // [2][LTC_COLN]
  const int WS = ltc_ws(G);
  float* Ws = cols + 2 * LTC_COLN;                               // [L][WS]
  float* Ys = Ws + L * WS;
  float* Yp = Ys + L * WS;
  float* Bds = Yp + L * WS;  // [L][L] coupling rows of the subdomain
  float* Bus = Bds + L * L;
  const int b = blockIdx.x / NG, grp = blockIdx.x % NG;
  const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int kb = grp * G;
  const int gl = min(G, P - kb);
  const int RPI = nthr / gl;
  const int io_m = tid % gl, io_a = tid / gl;
  const bool io_on = io_a < RPI;
  const int LP = L * P;
  const int rstep = RPI * P, sstep = RPI * WS;
  const bool act = init ? true : (ctl.active[b] != 0);
  double s_rz = 0.0, s_rr = 0.0;
  XAcc x_rz, x_rr;  // FP32 per-thread totals over the launch's steps
  if (act) {
    const int sub = b / R;
    const long long base = (long long)b * nl * P + kb + io_m;
    float* rb = r + base;
    float* xb = x + base;
    float* zb = z + base;
    const float* qb = q + base;
    const float* bd = Bd + (long long)sub * L * L;
    const float* bu = Bu + (long long)sub * L * L;
    const long long irow = img_row0 + (long long)sub * L * L;    // image row of (line 0, a = 0)
    const float* colp = col + (long long)sub * L * LTC_COLN;     // [line][LTC_COLN]
    const unsigned full0 = smem_u32(&bars[0]), mdone = smem_u32(&bars[2]);
    const bool wide_col = L == 65;
    const unsigned tx = (unsigned)L * 128 + (wide_col ? LTC_COLN * 4 : 0);
    auto issue = [&](int t) {  // TMA of step t's line into stage t & 1 (thread 0)
      const int line = t < L ? t : 2 * L - 2 - t;
      const int s = t & 1;
      mbar_expect_tx(full0 + 8 * s, tx);
      tma_load_2d(smem_u32(As + s * LTC_ABYTES), &tmS, full0 + 8 * s, 0, (int)(irow + (long long)line * L));
      if (wide_col) bulk_load(smem_u32(cols + s * LTC_COLN), colp + (long long)line * LTC_COLN, LTC_COLN * 4,
                              full0 + 8 * s);
    };
    // set-up: barriers, TMEM accumulator, zero B tile
    if (tid == 0) {
      mbar_init(full0, 1);
      mbar_init(full0 + 8, 1);
      mbar_init(mdone, 1);
      s_abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                   "r"(2 * NB)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int e = tid; e < NB * 2 * 128 / 16; e += nthr) reinterpret_cast<uint4*>(Bt)[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < L * L; e += nthr) {
      Bds[e] = bd[e];
      Bus[e] = bu[e];
    }
    const float* pb = nullptr;
    if (!init) {
      pb = ((*ctl.parity) ? pbuf0 : pbuf1) + base;  // p_new written by the apply kernel
      if (tid < 32) {
        double pq = 0.0;
        for (int t = tid; t < NT; t += 32) pq += ctl.part_pq[(long long)b * NT + t];
        for (int o = 16; o > 0; o >>= 1) pq += __shfl_down_sync(0xffffffffu, pq, o);
        if (tid == 0) {
          const double al = (pq > 0.0 && isfinite(pq)) ? ctl.rz[b] / pq : 0.0;
          alpha_s = isfinite(al) ? (float)al : 0.f;
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;
    if (tid == 0) issue(0);
    const float alpha = init ? 0.f : alpha_s;
    // prefetched registers: forward r, q, p, x of line j; backward y_j (in pr_r)
    float pr_r[NPF], pr_q[NPF], pr_p[NPF], pr_x[NPF];
    auto fetch = [&](int j) {
      if (!io_on) return;
      const int o0 = j * LP + io_a * P;
#pragma unroll
      for (int kk = 0; kk < NPF; ++kk) {
        const int a = io_a + kk * RPI;
        if (a < L) {
          const int o = o0 + kk * rstep;
          pr_r[kk] = rb[o];
          if (!init) { pr_q[kk] = qb[o]; pr_p[kk] = pb[o]; pr_x[kk] = xb[o]; }
        }
      }
    };
    auto fetch_y = [&](int j) {
      if (!io_on) return;
      const int o0 = j * LP + io_a * P;
#pragma unroll
      for (int kk = 0; kk < NPF; ++kk) {
        const int a = io_a + kk * RPI;
        if (a < L) pr_r[kk] = zb[o0 + kk * rstep];
      }
    };
    // B tile entry (row n = mode, column c = a) of both terms
    auto put_b = [&](int a, int m, float w) {
      if (a < 64) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(w);
        const __nv_bfloat16 lo = __float2bfloat16_rn(w - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16*>(Bt + sw128_offset(m, a)) = hi;
        *reinterpret_cast<__nv_bfloat16*>(Bt + sw128_offset(NB + m, a)) = lo;
      }
    };
    fetch(0);
    __syncthreads();
    const int T_END = 2 * L - 1;  // steps: forward t = j = 0 .. L-1, backward t = L .. 2L-2 (j = 2L-2-t)
    int t = 0;
    for (; t < T_END; ++t) {
      const bool fwd = t < L;
      const int j = fwd ? t : 2 * L - 2 - t;
      const int s = t & 1;
      if (tid == 0 && t + 1 < T_END) issue(t + 1);
      // ---- input phase: w = r_j - B_{j-1}^T y_{j-1} (forward), w = B_j x_{j+1} (backward) ----
      if (io_on) {
        const int o0 = j * LP + io_a * P;
        const int s0 = io_a * WS + io_m;
        if (fwd) {
          float amax = 0.f;
#pragma unroll
          for (int kk = 0; kk < NPF; ++kk) {
            const int a = io_a + kk * RPI;
            if (a < L) {
              const int o = o0 + kk * rstep, si = s0 + kk * sstep;
              float rv = pr_r[kk];
              if (!init) {
                rv -= alpha * pr_q[kk];
                rb[o] = rv;
                xb[o] = pr_x[kk] + alpha * pr_p[kk];
              }
              amax = fmaxf(amax, fabsf(rv));
              pr_r[kk] = rv;  // for the scaled partial below
              float wv = rv;
              if (j > 0) {
                const float yp = Yp[si];
                wv -= Bds[(j - 1) * L + a] * yp;
                if (a > 0) wv -= Bus[(j - 1) * L + a - 1] * Yp[si - WS];
                zb[o - LP] = yp;  // y_{j-1} parked in z
              }
              Ws[si] = wv;
              put_b(a, io_m, wv);
            }
          }
          const int e = f32_exp(amax);
          const float sc = f32_pow2(-e);
          float rs = 0.f;
#pragma unroll
          for (int kk = 0; kk < NPF; ++kk)
            if (io_a + kk * RPI < L) {
              const float v = pr_r[kk] * sc;
              rs = fmaf(v, v, rs);
            }
          x_rr.add(rs, 2 * e);
        } else {
#pragma unroll
          for (int kk = 0; kk < NPF; ++kk) {
            const int a = io_a + kk * RPI;
            if (a < L) {
              const int o = o0 + kk * rstep, si = s0 + kk * sstep;
              const float xn = Yp[si];
              float tv = Bds[j * L + a] * xn;
              if (a + 1 < L) tv += Bus[j * L + a] * Yp[si + WS];
              zb[o + LP] = xn;  // x_{j+1} final
              Ws[si] = tv;
              Ys[si] = pr_r[kk];  // y_j
              put_b(a, io_m, tv);
            }
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B tile -> tensor-core reads
      if (fwd) {
        if (j + 1 < L) fetch(j + 1);
        else fetch_y(L - 2);  // first backward step (y_{L-2} was parked by this thread above)
      } else if (j >= 1) {
        fetch_y(j - 1);
      }
      __syncthreads();
      // ---- product on the tensor cores ----
      if (tid == 0) {
        if (!mbar_wait(full0 + 8 * s, (unsigned)((t >> 1) & 1))) {
          atomicExch(ctl.breakdown, 20);
          s_abort = 1;
        } else {
          tc_fence_after();
          const unsigned a0 = smem_u32(As + s * LTC_ABYTES), b0 = smem_u32(Bt);
          constexpr unsigned idesc = idesc_bf16(128, 2 * NB);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            umma_bf16(tmem, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), idesc, k > 0 ? 1u : 0u);
          umma_commit(mdone);
        }
      }
      // ---- epilogue: row a of y (warps 0-3 own TMEM lanes 32 warp ..) ----
      if (warp < 4) {
        const int a = 32 * warp + lane;
        bool ok = mbar_wait(mdone, (unsigned)(t & 1));
        if (ok && wide_col) ok = mbar_wait(full0 + 8 * s, (unsigned)((t >> 1) & 1));  // column stage landed
        if (!ok) {
          atomicExch(ctl.breakdown, 21);
          s_abort = 1;
        }
        __syncwarp();
        tc_fence_after();
        const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
        const float ca = (ok && wide_col && a < L) ? cols[s * LTC_COLN + a] : 0.f;
        const float* w64 = Ws + 64 * WS;  // row c = 64 of w (read only when L = 65)
        float* yrow = Yp + min(a, L - 1) * WS;
        const float* wrow = Ws + min(a, L - 1) * WS;
        const float* ysrc = Ys + min(a, L - 1) * WS;
        float awm = 0.f, aym = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += 16) {
          float hi[16], lo[16];
          tmem_ld<16>(trow + c0, hi);        // warp-collective: every lane of warps 0-3
          tmem_ld<16>(trow + NB + c0, lo);
          if (ok && a < L) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int m = c0 + i;
              if (m < gl) {
                float y = hi[i] + lo[i];
                if (wide_col) y = fmaf(ca, w64[m], y);
                if (fwd) {
                  yrow[m] = y;
                  awm = fmaxf(awm, fabsf(wrow[m]));
                  aym = fmaxf(aym, fabsf(y));
                } else {
                  yrow[m] = ysrc[m] - y;
                }
              }
            }
          }
        }
        if (fwd && ok && a < L) {  // r.z partial of row a: sum_m w y, scaled
          const int ew = f32_exp(awm), ey = f32_exp(aym);
          const float sw = f32_pow2(-ew), sy = f32_pow2(-ey);
          float rs = 0.f;
          for (int m = 0; m < gl; ++m) rs = fmaf(wrow[m] * sw, yrow[m] * sy, rs);
          x_rz.add(rs, ew + ey);
        }
      }
      tc_fence_before();
      __syncthreads();
      if (s_abort) break;
    }
    if (!s_abort) {
      // x_0
      if (io_on) {
        const int s0 = io_a * WS + io_m;
        const int o0 = io_a * P;
#pragma unroll
        for (int kk = 0; kk < NPF; ++kk)
          if (io_a + kk * RPI < L) zb[o0 + kk * rstep] = Yp[s0 + kk * sstep];
      }
    } else if (tid == 0) {
      // timed out: let the copy and the products this block issued finish (bounded) before TMEM is freed
      if (t + 1 < T_END) (void)mbar_wait(full0 + 8 * ((t + 1) & 1), (unsigned)(((t + 1) >> 1) & 1));
      (void)mbar_wait(mdone, (unsigned)(t & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
      tc_fence_after();
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * NB) : "memory");
    }
  }
  s_rz += x_rz.value();
  s_rr += x_rr.value();
  line_control(s_rz, s_rr, b, grp, NG, NT, nb, ctl, init, tol2, bb_min, max_it, cond_handle, use_handle);
}

// BF16 image of the line factors for k_line_tc: img[m][a][c] = S_m(a, c) for c < min(L, 64), zero
// for L <= c < 64, with S_m = (S_m^{-1} + S_m^{-T}) / 2 of the FP64 factor (an exactly symmetric
// BF16 matrix); col[m][a] = the BF16-rounded S_m(a, 64) as FP32 (L = 65), m = (subdomain, line).
__global__ void k_line_img(long long nmat, int L, const double* __restrict__ Sinv, __nv_bfloat16* __restrict__ img,
                           float* __restrict__ col) {
  count_launch();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nmat * L * 64) return;
  const long long mat = i / ((long long)L * 64);
  const int rem = (int)(i - mat * L * 64), a = rem >> 6, c = rem & 63;
  const double* S = Sinv + mat * L * L;
  const double v = c < L ? 0.5 * (S[(long long)a * L + c] + S[(long long)c * L + a]) : 0.0;
  img[i] = __float2bfloat16_rn((float)v);
  if (L == 65 && c == 0) {
    const double u = 0.5 * (S[(long long)a * L + 64] + S[64LL * L + a]);
    col[mat * LTC_COLN + a] = __bfloat162float(__float2bfloat16_rn((float)u));
  }
}

// Line factorisation, FP64: one block per (subdomain, pattern).  D (within-line tridiagonal)
// diag Dd[j][a], upper Du[j][a]; coupling Bd, Bu as above.  Writes Sinv[j] (L x L).
// status[blk] = 1 when a pivot is not positive (the matrix is not SPD).
__global__ void k_line_factor(int L, const double* __restrict__ Dd, const double* __restrict__ Du,
                              const double* __restrict__ Bd, const double* __restrict__ Bu,
                              double* __restrict__ Sinv, int* status) {
  count_launch();
  extern __shared__ double sm[];
  double* S = sm;            // [L][L]
  double* col = S + L * L;   // [L] pivot column
  double* prow = col + L;    // [L] pivot row
  const int blk = blockIdx.x;
  const double* dd = Dd + (long long)blk * L * L;
  const double* du = Du + (long long)blk * L * L;
  const double* bd = Bd + (long long)blk * L * L;
  const double* bu = Bu + (long long)blk * L * L;
  double* out = Sinv + (long long)blk * L * L * L;
  const int nt = blockDim.x;
  for (int j = 0; j < L; ++j) {
    const double* Xp = out + (long long)(j - 1) * L * L;  // S_{j-1}^{-1}
    for (int e = threadIdx.x; e < L * L; e += nt) {
      const int a = e / L, c = e % L;
      double v = 0.0;
      if (a == c) v = dd[j * L + a];
      else if (c == a + 1) v = du[j * L + a];
      else if (a == c + 1) v = du[j * L + c];
      if (j > 0) {
        // (B^T X B)[a][c] = sum_{p in {a, a-1}} sum_{q in {c, c-1}} B[p][a] X[p][q] B[q][c]
        const double* bdp = bd + (j - 1) * L;
        const double* bup = bu + (j - 1) * L;
        double acc = 0.0;
        for (int pi = 0; pi < 2; ++pi) {
          const int pr = a - pi;
          if (pr < 0) continue;
          const double Bpa = pi == 0 ? bdp[a] : bup[a - 1];
          if (Bpa == 0.0) continue;
          for (int qi = 0; qi < 2; ++qi) {
            const int qr = c - qi;
            if (qr < 0) continue;
            const double Bqc = qi == 0 ? bdp[c] : bup[c - 1];
            if (Bqc == 0.0) continue;
            acc += Bpa * Xp[(long long)pr * L + qr] * Bqc;
          }
        }
        v -= acc;
      }
      S[e] = v;
    }
    __syncthreads();
    // in-place Gauss-Jordan inversion of the SPD block (no pivoting needed); the pivot row and
    // column are saved first so every update of a pass reads values of the previous pass
    for (int piv = 0; piv < L; ++piv) {
      const double d = S[piv * L + piv];
      if (!(d > 0.0) && threadIdx.x == 0) status[blk] = 1;
      for (int rr = threadIdx.x; rr < L; rr += nt) {
        col[rr] = S[rr * L + piv];
        prow[rr] = S[piv * L + rr];
      }
      __syncthreads();
      const double inv = 1.0 / d;
      for (int e = threadIdx.x; e < L * L; e += nt) {
        const int rr = e / L, c = e % L;
        double val;
        if (rr == piv && c == piv) val = inv;
        else if (rr == piv) val = prow[c] * inv;
        else if (c == piv) val = -col[rr] * inv;
        else val = S[e] - col[rr] * prow[c] * inv;
        S[e] = val;
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < L * L; e += nt) out[(long long)j * L * L + e] = S[e];
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// Outer (interface) PCG: device scalars and fused vector kernels, FP64.
// ------------------------------------------------------------------------------------------
struct OuterCtl {
  double gn;       // ||G||
  double rz;       // r . z
  double alpha, beta;
  double rel;      // ||r|| / ||G||
  int it;          // iterations of this step
  int done;
  int notconv;
  int breakdown;
};

enum : int { OP_INIT_G = 0, OP_RES0 = 1, OP_RZ0 = 2, OP_ALPHA = 3, OP_CHECK = 4, OP_BETA = 5, OP_BETA_FLEX = 6 };

// Interior accumulator of the mixed-precision step: on interior nodes (class INT),
//   W = v + e          (init, the interior solution K_II^{-1} f~_I of the condensed right-hand side)
//   W += a (v + e)     (otherwise; a = c->alpha of the outer PCG, or 1 when c is null),
// where v holds the FP32 solve widened to FP64 (plus interface values, ignored) and e the FP32
// correction.  By linearity u_I = K_II^{-1} (f~_I - K_IG u_G) is then W_I once u_G = x0 + sum a p.
__global__ void k_wacc(long long n, int P, const uint8_t* __restrict__ cls, const OuterCtl* c, int init,
                       const double* __restrict__ v, const float* __restrict__ e, double* __restrict__ W) {
  count_launch();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool interior = cls[i / P] == INT;
  if (init) {
    W[i] = interior ? v[i] + (double)e[i] : 0.0;
    return;
  }
  if (!interior) return;
  const double a = c ? c->alpha : 1.0;
  W[i] += a * (v[i] + (double)e[i]);
}

// partial sums of up to two dot products: part[blk] = x.y, part2[blk] = u.v
__global__ void k_odot(long long n, const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ u, const double* __restrict__ v, double* part, double* part2) {
  count_launch();
  double s = 0.0, s2 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    s += x[i] * y[i];
    if (u) s2 += u[i] * v[i];
  }
  __shared__ double sh[32], sh2[32];
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[w] = s; sh2[w] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, a2 = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += sh[q]; a2 += sh2[q]; }
    part[blockIdx.x] = a;
    if (part2) part2[blockIdx.x] = a2;
  }
}

// Scalar program of the outer PCG on reduced partials (single thread, fixed order).
__global__ void k_octl(int op, int npart, const double* part, const double* part2, OuterCtl* c, double tol,
                       int max_iter, cudaGraphConditionalHandle hwhile, cudaGraphConditionalHandle hif,
                       int use_handle, int* cond_mirror) {
  count_launch();
  if (threadIdx.x != 0) return;
  double s = 0.0, s2 = 0.0;
  for (int i = 0; i < npart; ++i) s += part[i];
  if (part2)
    for (int i = 0; i < npart; ++i) s2 += part2[i];
  switch (op) {
    case OP_INIT_G:
      c->gn = sqrt(s);
      c->it = 0;
      c->done = 0;
      c->notconv = 0;
      c->breakdown = !isfinite(s);
      c->rz = 0.0;
      break;
    case OP_RES0: {
      const double rel = c->gn > 0.0 ? sqrt(s) / c->gn : 0.0;
      c->rel = rel;
      c->done = !(rel > tol) || c->gn == 0.0 || c->breakdown;
      if (!isfinite(rel)) { c->breakdown = 1; c->done = 1; }
      const int cond = !c->done;
      cond_mirror[0] = cond;
      cond_mirror[1] = cond;
      if (use_handle) {
        cudaGraphSetConditional(hwhile, cond);
        cudaGraphSetConditional(hif, cond);
      }
      break;
    }
    case OP_RZ0:
      c->rz = s;
      break;
    case OP_ALPHA:
      if (!(s > 0.0) || !isfinite(s)) { c->breakdown = 1; c->alpha = 0.0; }
      else c->alpha = c->rz / s;
      break;
    case OP_CHECK: {
      c->it += 1;
      const double rel = sqrt(s) / c->gn;
      c->rel = rel;
      if (!isfinite(rel)) c->breakdown = 1;
      int done = !(rel > tol) || c->breakdown;
      if (!done && c->it >= max_iter) { done = 1; c->notconv = 1; }
      c->done = done;
      cond_mirror[0] = !done;
      cond_mirror[1] = !done;
      if (use_handle) {
        cudaGraphSetConditional(hwhile, done ? 0u : 1u);
        cudaGraphSetConditional(hif, done ? 0u : 1u);
      }
      break;
    }
    case OP_BETA:  // standard: beta = (r.z)_new / (r.z)_old
      c->beta = c->rz != 0.0 ? s / c->rz : 0.0;
      c->rz = s;
      break;
    case OP_BETA_FLEX:  // flexible (Polak-Ribiere): beta = z.(r - r_old) / (r.z)_old; s = r.z, s2 = z.r_old
      c->beta = c->rz != 0.0 ? (s - s2) / c->rz : 0.0;
      c->rz = s;
      break;
  }
}

// x += alpha p; r -= alpha q; partial ||r||^2
__global__ void k_oupd(long long n, const OuterCtl* c, const double* __restrict__ p, const double* __restrict__ q,
                       double* __restrict__ x, double* __restrict__ r, double* part) {
  count_launch();
  const double a = c->alpha;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    const double rv = r[i] - a * q[i];
    r[i] = rv;
    s += rv * rv;
  }
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int qq = 0; qq < (int)(blockDim.x >> 5); ++qq) acc += sh[qq];
    part[blockIdx.x] = acc;
  }
}

// r = g - q (initial residual) with partial ||r||^2
__global__ void k_ores0(long long n, const double* __restrict__ g, const double* __restrict__ q, double* __restrict__ r,
                        double* part) {
  count_launch();
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double rv = g[i] - q[i];
    r[i] = rv;
    s += rv * rv;
  }
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int qq = 0; qq < (int)(blockDim.x >> 5); ++qq) acc += sh[qq];
    part[blockIdx.x] = acc;
  }
}

// p = z + beta p (beta from the control block; first == 1: p = z)
__global__ void k_op(long long n, const OuterCtl* c, const double* __restrict__ z, double* __restrict__ p, int first) {
  count_launch();
  const double bt = first ? 0.0 : c->beta;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = first ? z[i] : z[i] + bt * p[i];
}

// zero x when the right-hand side vanishes (||G|| = 0)
__global__ void k_ozero_if(long long n, const OuterCtl* c, double* x) {
  count_launch();
  if (c->gn != 0.0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = 0.0;
}

// per-step record of the outer iteration count and relative residual
__global__ void k_record(OuterCtl* c, long long* stepctr, int cap, int* iters, double* relres, int* flags) {
  count_launch();
  if (threadIdx.x != 0) return;
  const long long s = *stepctr;
  iters[s % cap] = c->it;
  relres[s % cap] = c->rel;
  if (c->notconv) atomicOr(&flags[0], 1);
  if (c->breakdown) atomicOr(&flags[0], 2);
  *stepctr = s + 1;
}

// ------------------------------------------------------------------------------------------
// Interface gathers / scatters.
// ------------------------------------------------------------------------------------------
// x_loc[b][ln][k] = (class in mask) ? src[gidx][k] * (useD ? D[g] : 1) : 0
template <typename T>
__global__ void k_gather(int nb, int R, int nl, int P, const uint8_t* cls, const int* gidx, const double* D,
                         const double* __restrict__ src, T* __restrict__ dst, int mask, int useD) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nb * nl * P) return;
  const int k = (int)(idx % P);
  const long long t = idx / P;
  const int ln = (int)(t % nl), b = (int)(t / nl);
  const long long so = (long long)(b / R) * nl + ln;
  T v = T(0);
  if ((mask >> cls[so]) & 1) {
    const int g = gidx[so];
    double s = src[(long long)g * P + k];
    if (useD) s *= D[g];
    v = (T)s;
  }
  dst[idx] = v;
}

// dst[g][k] = sum over owners o of src[o][k] (* D[g] when useD); owners are (sub * nl + ln), mo per
// interface node (-1 padded), R = 1
template <typename T>
__global__ void k_scatter(int nG, int P, const int* owners, int mo, const double* D, const T* __restrict__ src,
                          double* __restrict__ dst, int useD) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nG * P) return;
  const int k = (int)(idx % P), g = (int)(idx / P);
  double s = 0.0;
  for (int q = 0; q < mo; ++q) {
    const int o = owners[g * mo + q];
    if (o >= 0) s += (double)src[(long long)o * P + k];
  }
  if (useD) s *= D[g];
  dst[idx] = s;
}

// Sum the interface values of all owners and write the sum back to every owner (global
// assembly of a local-layout vector on the interface).
__global__ void k_assemble_gamma(int nG, int P, const int* owners, int mo, double* __restrict__ v) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nG * P) return;
  const int k = (int)(idx % P), g = (int)(idx / P);
  double s = 0.0;
  for (int q = 0; q < mo; ++q) {
    const int o = owners[g * mo + q];
    if (o >= 0) s += v[(long long)o * P + k];
  }
  for (int q = 0; q < mo; ++q) {
    const int o = owners[g * mo + q];
    if (o >= 0) v[(long long)o * P + k] = s;
  }
}

// weight for counting each global dof once in local-layout dots: 1 on interior, D on interface
__global__ void k_node_weight(int n, const uint8_t* cls, const int* gidx, const double* D, double* w) {
  count_launch();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = cls[i];
  w[i] = c == DIR ? 0.0 : (c == INT ? 1.0 : D[gidx[i]]);
}

// res = sum_i w[node(i)] x_i y_i over a local-layout vector (single block, fixed order)
__global__ void k_dot_w(long long nnodes, int P, const double* w, const double* x, const double* y,
                        double* res) {
  count_launch();
  double s = 0.0;
  for (long long i = threadIdx.x; i < nnodes * P; i += blockDim.x) s += w[i / P] * x[i] * y[i];
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[wi] = s;
  __syncthreads();
  if (wi == 0) {
    s = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (l == 0) *res = s;
  }
}

// ------------------------------------------------------------------------------------------
// Coarse space.
// ------------------------------------------------------------------------------------------
// z_loc on the local interface of each subdomain (R = 1):
//   corner node: u_c[cidx][k];  remaining node: v + sum_{lc,m} Phi[sub][lc*P+m][gam][k] u_c[corner(lc)][m]
template <typename TV>
__global__ void k_coarse_extend(int nsub, int nl, int P, int nGam, int maxc, const uint8_t* cls,
                                const int* cidx, const int* gam_ln, const int* n_gam, const int* loc_corner,
                                int mc, const int* n_loc_corner, const double* __restrict__ Phi,
                                const double* __restrict__ uc, const TV* __restrict__ v,
                                double* __restrict__ zloc) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nsub * nGam * P) return;
  const int k = (int)(idx % P);
  const long long t = idx / P;
  const int q = (int)(t % nGam), sub = (int)(t / nGam);
  if (q >= n_gam[sub]) return;
  const int ln = gam_ln[(long long)sub * nGam + q];
  const long long so = (long long)sub * nl + ln;
  double val;
  if (cls[so] == COR) {
    val = uc[(long long)cidx[so] * P + k];
  } else {
    val = (double)v[so * P + k];
    const int nc = n_loc_corner[sub];
    const int ncolmax = maxc * P;
    for (int lc = 0; lc < nc; ++lc) {
      const int cg = cidx[(long long)sub * nl + loc_corner[sub * mc + lc]];
      for (int m = 0; m < P; ++m) {
        const int col = lc * P + m;
        val += Phi[(((long long)sub * ncolmax + col) * nGam + q) * P + k] * uc[(long long)cg * P + m];
      }
    }
  }
  zloc[so * P + k] = val;
}

// d[c][k] = sum over owners o of (wc - y)[o][k]
template <typename TY>
__global__ void k_corner_rhs(int nC, int P, const int* cowners, int mo, const double* __restrict__ wc,
                             const TY* __restrict__ y, double* __restrict__ d) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nC * P) return;
  const int k = (int)(idx % P), c = (int)(idx / P);
  double s = 0.0;
  for (int q = 0; q < mo; ++q) {
    const int o = cowners[c * mo + q];
    if (o >= 0) s += wc[(long long)o * P + k] - (double)y[(long long)o * P + k];
  }
  d[idx] = s;
}

// y = A x for a dense n x n row-major matrix (one warp per row)
__global__ void k_gemv(int n, const double* __restrict__ A, const double* __restrict__ x,
                       double* __restrict__ y) {
  count_launch();
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int l = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = A + (long long)row * n;
  double s = 0.0;
  for (int c = l; c < n; c += 32) s += a[c] * x[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (l == 0) y[row] = s;
}

// unit vectors of the coarse basis problems: problem b = sub * R + (lc * P + m)
__global__ void k_coarse_units(int nsub, int R, int nl, int P, int sub0, const int* loc_corner, int mc,
                               const int* n_loc_corner, double* e) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nsub * R) return;
  const int col = (int)(idx % R), sl = (int)(idx / R);
  const int sub = sub0 + sl;
  const int lc = col / P, m = col % P;
  if (lc >= n_loc_corner[sub]) return;
  const int ln = loc_corner[sub * mc + lc];
  e[(((long long)sl * R + col) * nl + ln) * P + m] = 1.0;
}

// Phi[sub][col][q][k] = v[b][gam_ln[q]][k] on remaining nodes (0 on corners)
template <typename TV>
__global__ void k_coarse_phi(int nsub_chunk, int sub0, int R, int nl, int P, int nGam, const uint8_t* cls,
                             const int* gam_ln, const int* n_gam, const TV* __restrict__ v,
                             double* __restrict__ Phi) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nsub_chunk * R * nGam * P) return;
  const int k = (int)(idx % P);
  long long t = idx / P;
  const int q = (int)(t % nGam);
  t /= nGam;
  const int col = (int)(t % R), sl = (int)(t / R);
  const int sub = sub0 + sl;
  double val = 0.0;
  if (q < n_gam[sub]) {
    const int ln = gam_ln[(long long)sub * nGam + q];
    if (cls[(long long)sub * nl + ln] == REM) val = (double)v[(((long long)sl * R + col) * nl + ln) * P + k];
  }
  Phi[(((long long)sub * R + col) * nGam + q) * P + k] = val;
}

// local coarse matrix entries: Fs[sub][row = lc'*P+m'][col] = y[b(col)][loc_corner[lc']][m']
__global__ void k_coarse_fs(int nsub_chunk, int sub0, int R, int nl, int P, const int* loc_corner, int mc,
                            const int* n_loc_corner, const double* __restrict__ y, double* __restrict__ Fs) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nsub_chunk * R * R) return;
  const int col = (int)(idx % R);
  long long t = idx / R;
  const int row = (int)(t % R), sl = (int)(t / R);
  const int sub = sub0 + sl;
  const int lr = row / P, mr = row % P;
  double val = 0.0;
  if (lr < n_loc_corner[sub] && col / P < n_loc_corner[sub]) {
    const int ln = loc_corner[sub * mc + lr];
    val = y[(((long long)sl * R + col) * nl + ln) * P + mr];
  }
  Fs[((long long)sub * R + row) * R + col] = val;
}

// ------------------------------------------------------------------------------------------
// Newmark and loads.
// ------------------------------------------------------------------------------------------
// um = (U + dt V)/(zeta dt^2) + (1 - 2 zeta) A/(2 zeta); uc = gamma dt um - V - (1-gamma) dt A
// xm = um + alpha0 uc (mass input of the effective load), on every node (Eqs. UmCm)
__global__ void k_newmark_pre(long long n, double dt, double alpha0, const double* __restrict__ U,
                              const double* __restrict__ V, const double* __restrict__ A,
                              double* __restrict__ um, double* __restrict__ uc, double* __restrict__ xm) {
  count_launch();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double zeta = 0.25, gamma = 0.5;
  const double m = (U[i] + dt * V[i]) / (zeta * dt * dt) + (1.0 - 2.0 * zeta) * A[i] / (2.0 * zeta);
  const double c = gamma * dt * m - V[i] - (1.0 - gamma) * A[i] * dt;
  um[i] = m;
  uc[i] = c;
  xm[i] = m + alpha0 * c;
}

// A_{n+1} = U_{n+1}/(zeta dt^2) - um; V_{n+1} = V + dt((1-gamma) A + gamma A_{n+1}); U = U_{n+1}
__global__ void k_newmark_post(long long n, double dt, const double* __restrict__ Un,
                               const double* __restrict__ um, double* __restrict__ U,
                               double* __restrict__ V, double* __restrict__ A) {
  count_launch();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double zeta = 0.25, gamma = 0.5;
  const double an = Un[i] / (zeta * dt * dt) - um[i];
  V[i] = V[i] + dt * ((1.0 - gamma) * A[i] + gamma * an);
  A[i] = an;
  U[i] = Un[i];
}

// point source: f[node][0] += w * ricker(t), t = (step + 1 + toff) dt read from the device step
// counter (amp folded into w)
__global__ void k_point_load(int n, const int* node, const double* w, const long long* stepctr, double dt,
                             double toff, double freq, int P, double* f) {
  count_launch();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double t = stepctr ? ((double)(*stepctr) + toff) * dt : toff * dt;
  const double pi = 3.14159265358979323846;
  const double tau = t - 1.0 / freq;
  const double a = (pi * freq * tau) * (pi * freq * tau);
  f[(long long)node[i] * P] += w[i] * (1.0 - 2.0 * a) * exp(-a);
}

// external nodal load (mode 0) split over the owners with D_s
__global__ void k_ext_load(long long nloc, int P, const int* free_of_local, const uint8_t* cls,
                           const int* gidx, const double* D, const double* __restrict__ fext,
                           double* __restrict__ f) {
  count_launch();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nloc) return;
  const int fi = free_of_local[i];
  if (fi < 0) return;
  double w = cls[i] == INT ? 1.0 : D[gidx[i]];
  f[i * P] += w * fext[fi];
}

// out[f][k] = src[owner(f)][k] (mode < 0: all modes; else one mode into out[f])
__global__ void k_gather_free(int nfree, int P, int mode, const int* owner, const double* __restrict__ src,
                              double* __restrict__ out) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (mode < 0) {
    if (idx >= (long long)nfree * P) return;
    const int k = (int)(idx % P), f = (int)(idx / P);
    out[idx] = src[(long long)owner[f] * P + k];
  } else {
    if (idx >= nfree) return;
    out[idx] = src[(long long)owner[idx] * P + mode];
  }
}

__global__ void k_moments(int nfree, int P, const int* owner, const double* __restrict__ src,
                          double* mean, double* var) {
  count_launch();
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfree) return;
  const double* u = src + (long long)owner[f] * P;
  if (mean) mean[f] = u[0];
  if (var) {
    double s = 0.0;
    for (int k = 1; k < P; ++k) s += u[k] * u[k];
    var[f] = s;
  }
}

// local[sub][ln][k] = src[free_of_local][k] for free nodes (checkpoint restore)
// PCE surrogate sampling (statistics of the SG solution, Sec. 6.2): psi[s][k] = Psi_k(xi_s), the
// orthonormal multivariate Hermite polynomial of multi-index alpha_k (P x M exponents, row-major),
// from the three-term recurrence He_{a+1} = x He_a - a He_{a-1} and the factor 1 / sqrt(a!).
constexpr int SURR_MAXM = 12, SURR_MAXA = 10;
__global__ void k_psi(int nsamp, int M, int P, int pmax, const signed char* __restrict__ alpha,
                      const double* __restrict__ xi, double* __restrict__ psi) {
  count_launch();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsamp) return;
  double he[SURR_MAXM][SURR_MAXA + 1];
  for (int n = 0; n < M; ++n) {
    const double x = xi[(long long)s * M + n];
    he[n][0] = 1.0;
    if (pmax >= 1) he[n][1] = x;
    for (int a = 1; a < pmax; ++a) he[n][a + 1] = x * he[n][a] - a * he[n][a - 1];
    double f = 1.0;  // a!
    for (int a = 1; a <= pmax; ++a) {
      f *= a;
      he[n][a] /= sqrt(f);
    }
  }
  for (int k = 0; k < P; ++k) {
    double v = 1.0;
    for (int n = 0; n < M; ++n) v *= he[n][alpha[k * M + n]];
    psi[(long long)s * P + k] = v;
  }
}

// out[s][j] = sum_k U[node_j][k] psi[s][k] (nodes are free-node indices; out of range -> NaN)
__global__ void k_surrogate(int nsamp, int npts, int P, int nfree, const int* __restrict__ nodes,
                            const int* __restrict__ free_owner, const double* __restrict__ U,
                            const double* __restrict__ psi, double* __restrict__ out) {
  count_launch();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nsamp * npts) return;
  const int j = (int)(i % npts);
  const long long s = i / npts;
  const int f = nodes[j];
  if (f < 0 || f >= nfree) { out[i] = nan(""); return; }
  const double* u = U + (long long)free_owner[f] * P;
  const double* ps = psi + s * P;
  double acc = 0.0;
  for (int k = 0; k < P; ++k) acc = fma(u[k], ps[k], acc);
  out[i] = acc;
}

__global__ void k_scatter_free(long long nloc, int P, const int* free_of_local, const double* __restrict__ src,
                               double* __restrict__ dst) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nloc * P) return;
  const int k = (int)(idx % P);
  const long long i = idx / P;
  const int f = free_of_local[i];
  dst[idx] = f >= 0 ? src[(long long)f * P + k] : 0.0;
}

// ------------------------------------------------------------------------------------------
// Small vector kernels
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_axpby(long long n, T a, const T* __restrict__ x, T b, const T* __restrict__ y,
                        T* __restrict__ out) {
  count_launch();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

// FP64 line factor [sub][j][a][c] -> FP32 copy with rows zero-padded to LS columns
template <typename TO>
__global__ void k_pad_factor(long long nrows, int L, int LS, const double* __restrict__ src, TO* __restrict__ dst) {
  count_launch();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows * LS) return;
  const long long row = i / LS;
  const int c = (int)(i - row * LS);
  dst[i] = c < L ? (TO)src[row * L + c] : TO(0);
}

// plain type conversion y = (TO) x
template <typename TI, typename TO>
__global__ void k_cvt(long long n, const TI* __restrict__ x, TO* __restrict__ y) {
  count_launch();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (TO)x[i];
}

// out = (double) xa + ya  (mixed-type sum of a converted vector and an FP64 vector)
template <typename TA>
__global__ void k_add_conv(long long n, const TA* __restrict__ xa, const double* __restrict__ ya,
                           double* __restrict__ out) {
  count_launch();
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)xa[i] + ya[i];
}

// out = convert(s * x) on nodes whose class is in mask (else 0)
template <typename TI, typename TO>
__global__ void k_conv_mask(int nb, int R, int nl, int P, const uint8_t* cls, const TI* __restrict__ x,
                            TO* __restrict__ y, int mask, double s) {
  count_launch();
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nb * nl * P) return;
  const long long t = idx / P;
  const int ln = (int)(t % nl), b = (int)(t / nl);
  y[idx] = ((mask >> cls[(long long)(b / R) * nl + ln]) & 1) ? (TO)(s * (double)x[idx]) : TO(0);
}


// ------------------------------------------------------------------------------------------
// Learned PCG warm start (an extension of the method): per interface (dof, mode) row a small
// MLP maps normalised features [u^n, u^{n-1}, u^{n-2}, predictor] / s to a correction c of the
// Newmark predictor, guess = predictor + s c.  BF16 weights, FP32 arithmetic and accumulation;
// FP32 master weights with Adam.  Parameter order: W1 (H x F), b1, W2 (H x H), b2, W3 (H), b3.
// ------------------------------------------------------------------------------------------
constexpr int NN_F = 4, NN_H = 32;
constexpr int NN_OW1 = 0, NN_OB1 = NN_OW1 + NN_H * NN_F, NN_OW2 = NN_OB1 + NN_H, NN_OB2 = NN_OW2 + NN_H * NN_H;
constexpr int NN_OW3 = NN_OB2 + NN_H, NN_OB3 = NN_OW3 + NN_H, NN_NP = NN_OB3 + 1;
constexpr int NN_ROWS = 64;   // rows per block of the network kernels (static shared memory < 48 KB)

struct WarmCtl {
  float* theta;           // [NP] FP32 master weights
  float* m;               // [NP] Adam first moment
  float* v;               // [NP] Adam second moment
  __nv_bfloat16* wb;      // [NP] BF16 weights used by the network kernels
  float* part;            // [blocks][NP] gradient partials
  double* loss_part;      // [blocks] loss partials
  float* loss;            // last training loss (mean squared error)
  int* train_left;        // online training steps still to do
  int* trained;           // training steps done (the guess is used once > 0)
  int* adam_it;           // Adam iteration counter
  double* arw;            // [4] autoregressive weights of the predictor-error model
  int* use_net;           // 1: the network's correction beat the AR model on the last step
  double* spart;          // [blocks][WS_NSTAT] statistics partials of k_wstats
};
constexpr int WS_NSTAT = 16;  // normal equations (10 + 4), squared errors without and with the network

// Predictor and features per row (interface dof, mode).  pred = u + dt v + dt^2/2 a, the Taylor
// predictor of u^{n+1} from the Newmark state (its error is O(dt^3), against O(dt) for the previous
// step's solution).  Features: the predictor's errors e_k = u^k - pred^k at the last four steps,
// divided by their RMS s; the network predicts the next error in units of s, so its BF16 weights set
// the accuracy of a correction of size |e|, not of size |u|.  s = 0 (no history yet) leaves the guess
// at the predictor.
__global__ void k_wfeat(int nrows, double dt, const double* __restrict__ u0, const double* __restrict__ e0,
                        const double* __restrict__ e1, const double* __restrict__ e2, const double* __restrict__ e3,
                        const double* __restrict__ vG, const double* __restrict__ aG, float* __restrict__ X,
                        double* __restrict__ pred, double* __restrict__ scale) {
  count_launch();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const double p = u0[r] + dt * vG[r] + 0.5 * dt * dt * aG[r];
  const double f[4] = {e0[r], e1[r], e2[r], e3[r]};
  double s = 0.0;
  for (int i = 0; i < 4; ++i) s += f[i] * f[i];
  s = sqrt(0.25 * s);
  const bool z = !(s > 0.0) || !isfinite(s);
  for (int i = 0; i < 4; ++i) X[(long long)r * 4 + i] = z ? 0.f : (float)(f[i] / s);
  pred[r] = p;
  scale[r] = z ? 0.0 : s;
}

// Network forward (and, with TRAIN, backward to block-partial gradients and loss).  One thread per
// row; activations of the block's rows live in shared memory for the weight-gradient sums.
template <bool TRAIN>
__global__ void __launch_bounds__(NN_ROWS) k_mlp(int nrows, const float* __restrict__ X, const float* __restrict__ t,
                                                 const __nv_bfloat16* __restrict__ wb, float* __restrict__ y_out,
                                                 float* __restrict__ part, double* __restrict__ loss_part,
                                                 const int* gate) {
  count_launch();
  if (TRAIN && gate && *gate <= 0) return;
  __shared__ float w[NN_NP];
  __shared__ float xs[NN_ROWS][NN_F];
  __shared__ float h1s[NN_ROWS][NN_H + 1];
  __shared__ float h2s[NN_ROWS][NN_H + 1];
  __shared__ float d2s[NN_ROWS][NN_H + 1];
  __shared__ float d1s[NN_ROWS][NN_H + 1];
  __shared__ float dys[NN_ROWS];
  __shared__ double red[NN_ROWS / 32];
  for (int i = threadIdx.x; i < NN_NP; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  const int lr = threadIdx.x;
  const int r = blockIdx.x * NN_ROWS + lr;
  const bool live = r < nrows;
  for (int f = 0; f < NN_F; ++f) xs[lr][f] = live ? X[(long long)r * NN_F + f] : 0.f;
  __syncthreads();
  for (int j = 0; j < NN_H; ++j) {
    float a = w[NN_OB1 + j];
    for (int f = 0; f < NN_F; ++f) a += w[NN_OW1 + j * NN_F + f] * xs[lr][f];
    h1s[lr][j] = tanhf(a);
  }
  float y = w[NN_OB3];
  for (int j = 0; j < NN_H; ++j) {
    float a = w[NN_OB2 + j];
    for (int q = 0; q < NN_H; ++q) a += w[NN_OW2 + j * NN_H + q] * h1s[lr][q];
    const float hv = tanhf(a);
    h2s[lr][j] = hv;
    y += w[NN_OW3 + j] * hv;
  }
  if (!TRAIN) {
    if (live) y_out[r] = y;
    return;
  }
  const float res = live ? y - t[r] : 0.f;
  const float dy = live ? 2.f * res / (float)nrows : 0.f;
  dys[lr] = dy;
  for (int j = 0; j < NN_H; ++j) d2s[lr][j] = dy * w[NN_OW3 + j] * (1.f - h2s[lr][j] * h2s[lr][j]);
  for (int q = 0; q < NN_H; ++q) {
    float a = 0.f;
    for (int j = 0; j < NN_H; ++j) a += d2s[lr][j] * w[NN_OW2 + j * NN_H + q];
    d1s[lr][q] = a * (1.f - h1s[lr][q] * h1s[lr][q]);
  }
  double l = (double)res * (double)res;
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((lr & 31) == 0) red[lr >> 5] = l;
  __syncthreads();
  // block-partial weight gradients: sums over the block's rows in a fixed order
  float* pb = part + (long long)blockIdx.x * NN_NP;
  for (int i = threadIdx.x; i < NN_NP; i += blockDim.x) {
    float s = 0.f;
    if (i < NN_OB1) {
      const int j = (i - NN_OW1) / NN_F, f = (i - NN_OW1) % NN_F;
      for (int q = 0; q < NN_ROWS; ++q) s += d1s[q][j] * xs[q][f];
    } else if (i < NN_OW2) {
      const int j = i - NN_OB1;
      for (int q = 0; q < NN_ROWS; ++q) s += d1s[q][j];
    } else if (i < NN_OB2) {
      const int j = (i - NN_OW2) / NN_H, c = (i - NN_OW2) % NN_H;
      for (int q = 0; q < NN_ROWS; ++q) s += d2s[q][j] * h1s[q][c];
    } else if (i < NN_OW3) {
      const int j = i - NN_OB2;
      for (int q = 0; q < NN_ROWS; ++q) s += d2s[q][j];
    } else if (i < NN_OB3) {
      const int j = i - NN_OW3;
      for (int q = 0; q < NN_ROWS; ++q) s += dys[q] * h2s[q][j];
    } else {
      for (int q = 0; q < NN_ROWS; ++q) s += dys[q];
    }
    pb[i] = s;
  }
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < NN_ROWS / 32; ++q) a += red[q];
    loss_part[blockIdx.x] = a;
  }
}

// Reduce the gradient partials (fixed order) and take one Adam step; refresh the BF16 copy.
__global__ void k_mlp_adam(int nblk, int nrows, WarmCtl c, float lr, const int* gate) {
  count_launch();
  if (gate && *gate <= 0) return;
  __shared__ int it_s;
  if (threadIdx.x == 0) it_s = *c.adam_it + 1;
  __syncthreads();
  const int it = it_s;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)it), c2 = 1.f - powf(b2, (float)it);
  for (int i = threadIdx.x; i < NN_NP; i += blockDim.x) {
    float g = 0.f;
    for (int b = 0; b < nblk; ++b) g += c.part[(long long)b * NN_NP + i];
    const float m = b1 * c.m[i] + (1.f - b1) * g;
    const float v = b2 * c.v[i] + (1.f - b2) * g * g;
    c.m[i] = m;
    c.v[i] = v;
    const float th = c.theta[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    c.theta[i] = th;
    c.wb[i] = __float2bfloat16_rn(th);
  }
  if (threadIdx.x == 0) {
    *c.adam_it = it;
    double l = 0.0;
    for (int b = 0; b < nblk; ++b) l += c.loss_part[b];
    *c.loss = (float)(l / (double)max(nrows, 1));
  }
}

// guess = pred + s y once the network has been trained; otherwise keep the previous solution
// Initial guess u = pred + ar + c: the Taylor predictor, the autoregressive estimate of its error
// ar = sum_k w_k e^{n-k} (weights fitted by least squares on the previous step, k_wsolve), and the
// network's correction c = s y when it beat the AR model alone on the previous step.
__global__ void k_wguess(int nrows, const WarmCtl c, const float* __restrict__ y, const double* __restrict__ pred,
                         const double* __restrict__ scale, const double* __restrict__ e0, const double* __restrict__ e1,
                         const double* __restrict__ e2, const double* __restrict__ e3, double* __restrict__ xG) {
  count_launch();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const double ar = c.arw[0] * e0[r] + c.arw[1] * e1[r] + c.arw[2] * e2[r] + c.arw[3] * e3[r];
  const double cn = (*c.use_net > 0 && isfinite(y[r])) ? scale[r] * (double)y[r] : 0.0;
  xG[r] = pred[r] + ar + cn;
}

// After the solve (xG = u^{n+1}): per-block partials of the least-squares normal equations of the
// predictor-error model (F = [e^n .. e^{n-3}] of the row, target e = u^{n+1} - pred), of the squared
// error of the AR estimate and of AR plus the network's correction (the one this step's guess could
// use); the network's training target t = (e - ar) / s while it trains.  Fixed-order reductions.
__global__ void __launch_bounds__(256) k_wstats(int nrows, const WarmCtl c, const double* __restrict__ xG,
                                                const double* __restrict__ pred, const double* __restrict__ scale,
                                                const float* __restrict__ y, const double* __restrict__ e0,
                                                const double* __restrict__ e1, const double* __restrict__ e2,
                                                const double* __restrict__ e3, float* __restrict__ t) {
  count_launch();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double v[WS_NSTAT];
#pragma unroll
  for (int i = 0; i < WS_NSTAT; ++i) v[i] = 0.0;
  if (r < nrows) {
    const double F[4] = {e0[r], e1[r], e2[r], e3[r]};
    const double e = xG[r] - pred[r];
    const double ar = c.arw[0] * F[0] + c.arw[1] * F[1] + c.arw[2] * F[2] + c.arw[3] * F[3];
    const double r1 = e - ar;
    const double r2 = isfinite(y[r]) ? r1 - scale[r] * (double)y[r] : r1;
    int q = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = i; j < 4; ++j) v[q++] = F[i] * F[j];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[10 + i] = F[i] * e;
    v[14] = r1 * r1;
    v[15] = r2 * r2;
    if (*c.train_left > 0) t[r] = scale[r] > 0.0 ? (float)(r1 / scale[r]) : 0.f;
  }
  __shared__ double red[8][WS_NSTAT];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < WS_NSTAT; ++i) {
    double x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[wid][i] = x;
  }
  __syncthreads();
  if (threadIdx.x < WS_NSTAT) {
    double x = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) x += red[w2][threadIdx.x];
    c.spart[(long long)blockIdx.x * WS_NSTAT + threadIdx.x] = x;
  }
}

// Sum of the partials (each of 256 threads a fixed strided subset of the blocks, then a fixed-order
// tree), the ridge-regularised 4 x 4 least-squares solve for the AR weights of the next guess
// (Gaussian elimination with partial pivoting, one thread), and the network gate: its correction is
// used on the next step when it lowered the last step's error below 0.9 of the AR estimate's.  One
// block of 256 threads.
__global__ void __launch_bounds__(256) k_wsolve(int nblk, const WarmCtl c) {
  count_launch();
  __shared__ double red[256][WS_NSTAT + 1];
  double v[WS_NSTAT];
  for (int i = 0; i < WS_NSTAT; ++i) v[i] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int i = 0; i < WS_NSTAT; ++i) v[i] += c.spart[(long long)b * WS_NSTAT + i];
  for (int i = 0; i < WS_NSTAT; ++i) red[threadIdx.x][i] = v[i];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int i = 0; i < WS_NSTAT; ++i) red[threadIdx.x][i] += red[threadIdx.x + h][i];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  for (int i = 0; i < WS_NSTAT; ++i) v[i] = red[0][i];
  double G[4][5];
  int q = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = i; j < 4; ++j) G[i][j] = G[j][i] = v[q++];
  const double tr = G[0][0] + G[1][1] + G[2][2] + G[3][3];
  for (int i = 0; i < 4; ++i) {
    G[i][i] += 1e-10 * tr;
    G[i][4] = v[10 + i];
  }
  bool ok = tr > 0.0 && isfinite(tr);
  for (int k = 0; k < 4 && ok; ++k) {
    int pv = k;
    for (int i = k + 1; i < 4; ++i)
      if (fabs(G[i][k]) > fabs(G[pv][k])) pv = i;
    if (!(fabs(G[pv][k]) > 0.0)) { ok = false; break; }
    for (int j = 0; j < 5; ++j) { const double tmp = G[k][j]; G[k][j] = G[pv][j]; G[pv][j] = tmp; }
    for (int i = k + 1; i < 4; ++i) {
      const double f = G[i][k] / G[k][k];
      for (int j = k; j < 5; ++j) G[i][j] -= f * G[k][j];
    }
  }
  double wv[4] = {0.0, 0.0, 0.0, 0.0};
  if (ok) {
    for (int i = 3; i >= 0; --i) {
      double x = G[i][4];
      for (int j = i + 1; j < 4; ++j) x -= G[i][j] * wv[j];
      wv[i] = x / G[i][i];
    }
    for (int i = 0; i < 4; ++i) ok = ok && isfinite(wv[i]);
  }
  for (int i = 0; i < 4; ++i) c.arw[i] = ok ? wv[i] : 0.0;
  *c.use_net = (*c.trained > 0 && v[15] < 0.9 * v[14]) ? 1 : 0;
}

// FP32 -> BF16 copy of the parameters
__global__ void k_to_bf16(int n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  count_launch();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// sum of the gradient partials into one vector (fixed order), mean-squared-error loss
__global__ void k_mlp_reduce(int nblk, int nrows, const float* __restrict__ part, const double* __restrict__ loss_part,
                             float* __restrict__ grad, double* __restrict__ loss) {
  count_launch();
  for (int i = threadIdx.x; i < NN_NP; i += blockDim.x) {
    float g = 0.f;
    for (int b = 0; b < nblk; ++b) g += part[(long long)b * NN_NP + i];
    grad[i] = g;
  }
  if (threadIdx.x == 0) {
    double l = 0.0;
    for (int b = 0; b < nblk; ++b) l += loss_part[b];
    *loss = l / (double)max(nrows, 1);
  }
}

// end of a step: history shift (u^{n-2} <- u^{n-1} <- u^n) and training bookkeeping
// history of predictor errors: e3 <- e2 <- e1 <- e0 <- u^{n+1} - pred
__global__ void k_wshift(int nrows, double* __restrict__ e0, double* __restrict__ e1, double* __restrict__ e2,
                         double* __restrict__ e3, const double* __restrict__ xG, const double* __restrict__ pred) {
  count_launch();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  e3[r] = e2[r];
  e2[r] = e1[r];
  e1[r] = e0[r];
  e0[r] = xG[r] - pred[r];
}
__global__ void k_wdone(WarmCtl c) {
  count_launch();
  if (threadIdx.x == 0 && *c.train_left > 0) {
    *c.train_left -= 1;
    *c.trained += 1;
  }
}

// ------------------------------------------------------------------------------------------
// Dense inverse of the mean operator A0 of one pattern (set-up, FP64).  Column c of A0^{-1} is the
// block-tridiagonal solve with right-hand side e_c, by the forward / backward line sweeps of the
// line preconditioner with the stored S_j^{-1}.  A0^{-1} is symmetric, so column c is stored as row c
// of the BF16 copy Ainv[sub][c][node] (row length Kp); rows and columns of nodes outside the
// pattern's free set (class bit not in pat_mask) are zero.  Block (64, INV_CB): x = position along
// a grid line, y = column; grid nsub x ceil(L^2 / INV_CB).
// ------------------------------------------------------------------------------------------
constexpr int INV_CB = 4;
__global__ void __launch_bounds__(256) k_inv_cols(int L, int nl, int Kp, int pat_mask, const uint8_t* __restrict__ cls,
                                                  const double* __restrict__ Sinv, const double* __restrict__ Bd,
                                                  const double* __restrict__ Bu, __nv_bfloat16* __restrict__ out) {
  count_launch();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LL = L * L;
  double* ys = reinterpret_cast<double*>(smem_raw);  // [INV_CB][LL]
  double* ws = ys + (size_t)INV_CB * LL;              // [INV_CB][64]
  const int ngrp = (LL + INV_CB - 1) / INV_CB;
  const int s = blockIdx.x / ngrp;
  const int col = (blockIdx.x % ngrp) * INV_CB + threadIdx.y;
  const int a = threadIdx.x;
  const bool colok = col < LL && ((pat_mask >> cls[(size_t)s * nl + col]) & 1);
  const double* S = Sinv + (size_t)s * LL * L;
  const double* bd = Bd + (size_t)s * LL;
  const double* bu = Bu + (size_t)s * LL;
  double* y = ys + (size_t)threadIdx.y * LL;
  double* w = ws + threadIdx.y * 64;
  const bool ok = a < L;
  for (int j = 0; j < L; ++j) {
    if (ok) {
      double rhs = (colok && col == j * L + a) ? 1.0 : 0.0;
      if (j > 0) {
        rhs -= bd[(j - 1) * L + a] * y[(j - 1) * L + a];
        if (a > 0) rhs -= bu[(j - 1) * L + a - 1] * y[(j - 1) * L + a - 1];
      }
      w[a] = rhs;
    }
    __syncthreads();
    if (ok) {
      const double* row = S + ((size_t)j * L + a) * L;
      double acc = 0.0;
      for (int c2 = 0; c2 < L; ++c2) acc += row[c2] * w[c2];
      y[j * L + a] = acc;
    }
    __syncthreads();
  }
  for (int j = L - 2; j >= 0; --j) {
    if (ok) {
      double t = bd[j * L + a] * y[(j + 1) * L + a];
      if (a + 1 < L) t += bu[j * L + a] * y[(j + 1) * L + a + 1];
      w[a] = t;
    }
    __syncthreads();
    if (ok) {
      const double* row = S + ((size_t)j * L + a) * L;
      double acc = 0.0;
      for (int c2 = 0; c2 < L; ++c2) acc += row[c2] * w[c2];
      y[j * L + a] -= acc;
    }
    __syncthreads();
  }
  if (col < LL) {
    __nv_bfloat16* o = out + ((size_t)s * Kp + col) * Kp;
    for (int nd = a; nd < LL; nd += 64) {
      const bool nok = (pat_mask >> cls[(size_t)s * nl + nd]) & 1;
      o[nd] = __float2bfloat16_rn(colok && nok ? (float)y[nd] : 0.f);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Inner CG update (x += alpha p, r -= alpha q, alpha = r.z / p.q, on all modes of 64 nodes) and
// packing of the updated residual into the image read by k_pre_mma: per right-hand side b and
// 64-node chunk c, the TERMS BF16 terms of r (bf16_split), each a K-major 128-byte-swizzled block
// of NB rows (PCE modes, zero beyond P) x 64 nodes.  Grid: nb x NC blocks.
// init: first call of a solve (x = 0, pack r only).
// ------------------------------------------------------------------------------------------
template <int NB, int TERMS>
__global__ void __launch_bounds__(256) k_cg_pack(int L, int nl, int P, int NC, int NT, float* __restrict__ x,
                                                 float* __restrict__ r, const float* pbuf0, const float* pbuf1,
                                                 const float* __restrict__ q, CgCtl ctl, int init,
                                                 unsigned char* __restrict__ bimg) {
  count_launch();
  __shared__ float rs[64][NB + 1];
  const int b = blockIdx.x / NC, c = blockIdx.x % NC;
  pdl_trigger();
  pdl_wait();
  // control scalars and the p.q partials of the problem in one round trip; the chunk's data loads
  // that do not depend on them are issued before the activity test.  alpha is formed in FP64 by
  // warp 0 alone (partials summed in index order from shuffles, as a sequential loop would) and
  // broadcast through shared memory: FP64 work is slow on this GPU.
  __shared__ float s_alpha;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int actv = 1, par = 0;
  double rzb = 0.0, vq = 0.0;
  if (!init) {
    actv = ctl.active[b];
    par = *ctl.parity;
    if (warp == 0) {
      rzb = ctl.rz[b];
      vq = lane < NT ? ctl.part_pq[(long long)b * NT + lane] : 0.0;
    }
  }
  const int LL = nl;  // nodes per problem (L^2 on the grid, the padded vertex count on a mesh)
  const long long base = (long long)b * nl * P;
  const int n0 = c * 64;
  // values of the chunk's nodes (contiguous); the last chunks of the padded Kp rows may hold none
  const int nv = max(0, min(64, LL - n0)) * P;
  const long long o0 = base + (long long)n0 * P;
  const bool vec = ((nl * P) & 3) == 0 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(r) |
                                            reinterpret_cast<uintptr_t>(q) | reinterpret_cast<uintptr_t>(pbuf0) |
                                            reinterpret_cast<uintptr_t>(pbuf1)) & 15) == 0;
  constexpr int U = 2;
  float4 rv[U], xv[U], pv[U], qv[U];
  const int n4 = vec ? nv >> 2 : 0;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int e4 = threadIdx.x + u * 256;
    if (e4 < n4) {
      rv[u] = reinterpret_cast<const float4*>(r + o0)[e4];
      if (!init) {
        xv[u] = reinterpret_cast<const float4*>(x + o0)[e4];
        qv[u] = reinterpret_cast<const float4*>(q + o0)[e4];
      }
    }
  }
  float alpha = 0.f;
  const float* pc = nullptr;
  if (!init) {
    pc = par ? pbuf0 : pbuf1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e4 = threadIdx.x + u * 256;
      if (e4 < n4) pv[u] = reinterpret_cast<const float4*>(pc + o0)[e4];
    }
    if (warp == 0) {
      double pq = 0.0;
      for (int t0 = 0; t0 < NT; t0 += 32) {
        if (t0 > 0) vq = t0 + lane < NT ? ctl.part_pq[(long long)b * NT + t0 + lane] : 0.0;
        const int n = min(32, NT - t0);
        for (int t = 0; t < n; ++t) pq += __shfl_sync(0xffffffffu, vq, t);
      }
      const double al = (pq > 0.0 && isfinite(pq)) ? rzb / pq : 0.0;
      if (lane == 0) s_alpha = isfinite(al) ? (float)al : 0.f;
    }
  }
  if (!actv) return;  // uniform over the block
  if (!init) {
    __syncthreads();
    alpha = s_alpha;
  }
  if (vec) {
    // 16-byte vectors; every load of a thread is issued before its stores (pc may alias nothing,
    // but the compiler cannot know)
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e4 = threadIdx.x + u * 256;
      if (e4 < n4) {
        if (!init) {
          xv[u].x += alpha * pv[u].x; xv[u].y += alpha * pv[u].y;
          xv[u].z += alpha * pv[u].z; xv[u].w += alpha * pv[u].w;
          rv[u].x -= alpha * qv[u].x; rv[u].y -= alpha * qv[u].y;
          rv[u].z -= alpha * qv[u].z; rv[u].w -= alpha * qv[u].w;
          reinterpret_cast<float4*>(x + o0)[e4] = xv[u];
          reinterpret_cast<float4*>(r + o0)[e4] = rv[u];
        }
        const float vv[4] = {rv[u].x, rv[u].y, rv[u].z, rv[u].w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int e = 4 * e4 + m, i = e / P;
          rs[i][e - i * P] = vv[m];
        }
      }
    }
    for (int e = nv + threadIdx.x; e < 64 * P; e += blockDim.x) rs[e / P][e % P] = 0.f;
    for (int e4 = threadIdx.x + U * 256; e4 < n4; e4 += blockDim.x) {  // chunks beyond U x 256 vectors
      for (int m = 0; m < 4; ++m) {
        const int e = 4 * e4 + m, i = e / P;
        const long long o = o0 + e;
        float v = r[o];
        if (!init) {
          x[o] += alpha * pc[o];
          v -= alpha * q[o];
          r[o] = v;
        }
        rs[i][e - i * P] = v;
      }
    }
  } else {
    for (int e = threadIdx.x; e < 64 * P; e += blockDim.x) {
      const int i = e / P, k = e - i * P;
      float v = 0.f;
      if (e < nv) {
        const long long o = o0 + e;
        v = r[o];
        if (!init) {
          x[o] += alpha * pc[o];
          v -= alpha * q[o];
          r[o] = v;
        }
      }
      rs[i][k] = v;
    }
  }
  if (NB > P)
    for (int e = threadIdx.x; e < 64 * (NB - P); e += blockDim.x) rs[e / (NB - P)][P + e % (NB - P)] = 0.f;
  __syncthreads();
  unsigned char* dst = bimg + ((size_t)b * NC + c) * TERMS * (NB * 128);
  for (int t = threadIdx.x; t < TERMS * NB * 8; t += blockDim.x) {
    const int hl = t / (NB * 8), rem = t - hl * NB * 8, n = rem >> 3, j = rem & 7;
    unsigned h[8];
#pragma unroll
    for (int i2 = 0; i2 < 8; ++i2) {
      __nv_bfloat16 tt[TERMS];
      bf16_split<TERMS>(rs[j * 8 + i2][n], tt);
      __nv_bfloat16 v = tt[0];
#pragma unroll
      for (int q2 = 1; q2 < TERMS; ++q2)
        if (hl == q2) v = tt[q2];
      h[i2] = (unsigned)__bfloat16_as_ushort(v);
    }
    uint4 pk;
    pk.x = h[0] | (h[1] << 16);
    pk.y = h[2] | (h[3] << 16);
    pk.z = h[4] | (h[5] << 16);
    pk.w = h[6] | (h[7] << 16);
    *reinterpret_cast<uint4*>(dst + hl * NB * 128 + sw128_offset(n, j * 8)) = pk;
  }
}

// ------------------------------------------------------------------------------------------
// z = A0^{-1} r on the tensor cores (mma_tile) for every mode of every right-hand side; the image
// holds r, packed by k_cg_pack after the CG update.  The accumulator tile (128 nodes x NB modes) is
// staged through shared memory so that z is stored, and r read back for the partials r.z, r.r, with
// coalesced accesses (the tile's 128 nodes x P modes are contiguous in the [node][mode] layout).
// Then the loop control (line_control, NG = MT row tiles).  Grid: nb x MT CTAs of 256 threads;
// rows of A for (pattern, subdomain) start at row0 + sub * Kp.  err: set to 16 + stage when a
// bounded wait of the pipeline ran out.
// ------------------------------------------------------------------------------------------
// Pipeline of the preconditioner product: 2 chunks per stage; 4 stages with two terms, 3 with three.
// (A recurrence z -= alpha A0^{-1} q on a three-term image of q, which would skip k_cg_pack, was
// measured: 44% more inner iterations on the 128^2 workload and no faster per iteration.)
constexpr int PRE_CPS = 2;
template <int TERMS>
struct PreNst {
  static constexpr int v = TERMS == 3 ? 3 : 4;
};
template <int NB, int TERMS>
using PreShape = MmaShape<NB, TERMS, PreNst<TERMS>::v, PRE_CPS>;

template <int NB>
__global__ void __launch_bounds__(256, 1) k_pre_mma(const __grid_constant__ CUtensorMap tmA, int L, int nl, int P,
                                                    int R, int MT, int NC, int NT, int Kp, int row0, int nb,
                                                    const unsigned char* __restrict__ bimg,
                                                    const float* __restrict__ r, float* __restrict__ z, CgCtl ctl,
                                                    int init, double tol2, double bb_min, int max_it,
                                                    cudaGraphConditionalHandle cond_handle, int use_handle,
                                                    int* err) {
  constexpr int TERMS = 2;
  constexpr int NST = PreNst<TERMS>::v;
  count_launch();
  extern __shared__ unsigned char smem_mma_raw[];
  __shared__ __align__(8) unsigned long long bars[2 * NST + 1];
  __shared__ unsigned tmem_slot;
  __shared__ int s_flags[2];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_mma_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int b = blockIdx.x / MT, tile = blockIdx.x % MT;
  pdl_trigger();
  // prologue before the predecessor has finished: mbarriers, TMEM, the tensor-map descriptor
  const unsigned tmem = mma_begin<NB, TERMS, NST>(bars, &tmem_slot, s_flags);
  if (threadIdx.x == 32)
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&tmA)) : "memory");
  pdl_wait();
  // the tile's residual (rows x P contiguous values, at most NB / 2 per thread) is loaded before the
  // product, so that its latency overlaps the pipeline instead of following it
  constexpr int EPT = MMA_M * NB / 256;
  const int m0 = tile * MMA_M;
  const int rows = min(MMA_M, nl - m0);  // nl = L^2 on the grid
  const int cnt = rows > 0 ? rows * P : 0;
  const long long o = (long long)b * nl * P + (long long)m0 * P;
  float rpre[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int e = threadIdx.x + u * 256;
    rpre[u] = e < cnt ? r[o + e] : 0.f;
  }
  const bool act = init ? true : (ctl.active[b] != 0);
  double s_rz = 0.0, s_rr = 0.0;
  if (!act) mma_tile_end<NB, TERMS, NST>(bars, tmem, s_flags);
  if (act) {
    const int sub = b / R;
    const int y0 = row0 + sub * Kp + tile * MMA_M;
    const unsigned char* bb = bimg + (size_t)b * NC * PreShape<NB, TERMS>::BCHUNK;
    mma_run<NB, TERMS, NST, PRE_CPS>(&tmA, y0, bb, NC, smem, bars, tmem, s_flags, err);
    // every stage has been consumed: stage 0 is free for the accumulator tile [128][NB + 1]
    float* zt = reinterpret_cast<float*>(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= 4) {
      float v[NB];
      mma_row<NB, TERMS>(tmem, warp - 4, v);
      float* zr = zt + ((warp - 4) * 32 + lane) * (NB + 1);
#pragma unroll
      for (int k = 0; k < NB; ++k) zr[k] = v[k];
    }
    mma_tile_end<NB, TERMS, NST>(bars, tmem, s_flags);  // contains __syncthreads
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = threadIdx.x + u * 256;
      if (e < cnt) {
        const int rr_ = e / P, k = e - rr_ * P;
        const float zv = zt[rr_ * (NB + 1) + k];
        z[o + e] = zv;
        const double rv = (double)rpre[u];
        s_rz += rv * (double)zv;
        s_rr += rv * rv;
      }
    }
  }
  line_control(s_rz, s_rr, b, tile, MT, NT, nb, ctl, init, tol2, bb_min, max_it, cond_handle, use_handle);
}

}  // namespace sgk
