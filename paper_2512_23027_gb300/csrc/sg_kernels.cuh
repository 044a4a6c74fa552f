// Device kernels of the SG-DD wave solver (sm_103a).
//
// Vectors of subdomain problems use the local layout [problem b][local node ln][PCE mode k],
// ln = lj * L + li on the (H+1) x (H+1) node grid of a subdomain; problem b belongs to subdomain
// b / R (R right-hand sides per subdomain).  Interface vectors use [global interface node][k].
// Nodes outside a problem's free set always hold 0, so operators never need input masks.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace sgk {

enum : int { DIR = 0, INT = 1, REM = 2, COR = 3 };
constexpr int MASK_I = 1 << INT, MASK_R = 1 << REM, MASK_C = 1 << COR;
constexpr int MASK_G = MASK_R | MASK_C, MASK_FREE = MASK_I | MASK_R | MASK_C, MASK_N = MASK_I | MASK_R;

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
  int L, nl, P, PI;
  T mass_h;              // h^2 / 24: unit entry of the consistent P1 mass on a right triangle
};

// ------------------------------------------------------------------------------------------
// Stochastic Galerkin operator apply:
//   y = add + cm (M (x) I) xm + ck (sum_i K_i (x) G_i) xk     on nodes with class in out_mask
// The stiffness part uses the graph-Laplacian form of P1 on right triangles: for every leg
// (a, b) with weight kappa_i(ab) (half the element coefficient per adjacent element),
//   y_a[k] += sum_{(i,j,k) in G} kappa_i(ab) G_ijk (x_a[j] - x_b[j])       (Sec. 4, Eq. stoksub)
// and the mass part the consistent P1 mass h^2/24 [2 1 1; 1 2 1; 1 1 2] per element, which is
// block diagonal over the modes for a deterministic mass (Sec. 4).
// One thread per (b, ln, k); the G entries of output mode k are contiguous.
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_apply(Op<T> op, int nb, int R, const T* __restrict__ xm,
                        const T* __restrict__ xk, T* __restrict__ y, const T* __restrict__ add,
                        T cm, T ck, int out_mask) {
  const long long total = (long long)nb * op.nl * op.P;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int P = op.P, L = op.L, nl = op.nl;
  const int k = (int)(idx % P);
  const long long t = idx / P;
  const int ln = (int)(t % nl);
  const int b = (int)(t / nl);
  const int sub = b / R;
  const long long so = (long long)sub * nl + ln;
  const int c = op.cls[so];
  if (!((out_mask >> c) & 1)) {
    y[idx] = T(0);
    return;
  }
  const int li = ln % L, lj = ln / L;
  T acc = T(0);
  if (ck != T(0)) {
    const T* xa = xk + ((long long)b * nl + ln) * P;
    const int e0 = op.gk_ptr[k], e1 = op.gk_ptr[k + 1];
    T s = T(0);
    if (li < L - 1) {
      const T* kap = op.kapE + so * op.PI;
      const T* xn = xa + P;
      for (int e = e0; e < e1; ++e) s += kap[op.gk_i[e]] * op.gk_v[e] * (xa[op.gk_j[e]] - xn[op.gk_j[e]]);
    }
    if (li > 0) {
      const T* kap = op.kapE + (so - 1) * op.PI;
      const T* xn = xa - P;
      for (int e = e0; e < e1; ++e) s += kap[op.gk_i[e]] * op.gk_v[e] * (xa[op.gk_j[e]] - xn[op.gk_j[e]]);
    }
    if (lj < L - 1) {
      const T* kap = op.kapN + so * op.PI;
      const T* xn = xa + (long long)L * P;
      for (int e = e0; e < e1; ++e) s += kap[op.gk_i[e]] * op.gk_v[e] * (xa[op.gk_j[e]] - xn[op.gk_j[e]]);
    }
    if (lj > 0) {
      const T* kap = op.kapN + (so - L) * op.PI;
      const T* xn = xa - (long long)L * P;
      for (int e = e0; e < e1; ++e) s += kap[op.gk_i[e]] * op.gk_v[e] * (xa[op.gk_j[e]] - xn[op.gk_j[e]]);
    }
    acc += ck * s;
  }
  if (cm != T(0)) {
    const T* xa = xm + ((long long)b * nl + ln) * P + k;
    const int cb = op.cells[so];
    const long long dN = (long long)L * P;
    T self = T(0), nbs = T(0);
    if (cb & 1) { self += T(4); nbs += T(2) * xa[-dN - P] + xa[-dN] + xa[-P]; }  // cell (li-1, lj-1)
    if (cb & 2) { self += T(2); nbs += xa[-dN] + xa[P]; }                        // cell (li,   lj-1)
    if (cb & 4) { self += T(2); nbs += xa[-P] + xa[dN]; }                        // cell (li-1, lj)
    if (cb & 8) { self += T(4); nbs += xa[P] + T(2) * xa[dN + P] + xa[dN]; }     // cell (li,   lj)
    acc += cm * op.mass_h * (self * xa[0] + nbs);
  }
  if (add) acc += add[idx];
  y[idx] = acc;
}

template <typename T>
void apply(const Op<T>& op, int nb, int R, const T* xm, const T* xk, T* y, const T* add, T cm, T ck,
           int out_mask, cudaStream_t st) {
  const long long total = (long long)nb * op.nl * op.P;
  const int bs = 256;
  const long long grid = (total + bs - 1) / bs;
  k_apply<T><<<(unsigned)grid, bs, 0, st>>>(op, nb, R, xm, xk, y, add, cm, ck, out_mask);
}

// ------------------------------------------------------------------------------------------
// Deterministic per-problem dot products: one block per problem, fixed-order tree.
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_dot(long long len, const T* __restrict__ x, const T* __restrict__ y,
                      const T* __restrict__ z, double* res, double* res2) {
  const int b = blockIdx.x;
  const T* xb = x + (long long)b * len;
  const T* yb = y + (long long)b * len;
  const T* zb = z ? z + (long long)b * len : nullptr;
  double s = 0.0, s2 = 0.0;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) {
    double xv = (double)xb[i];
    s += xv * (double)yb[i];
    if (zb) s2 += xv * (double)zb[i];
  }
  __shared__ double sh[32], sh2[32];
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[w] = s; sh2[w] = s2; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    s = l < nw ? sh[l] : 0.0;
    s2 = l < nw ? sh2[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, o);
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (l == 0) {
      res[b] = s;
      if (res2) res2[b] = s2;
    }
  }
}

template <typename T>
void dot(int nb, long long len, const T* x, const T* y, const T* z, double* res, double* res2,
         cudaStream_t st) {
  k_dot<T><<<nb, 512, 0, st>>>(len, x, y, z, res, res2);
}

// ------------------------------------------------------------------------------------------
// Inner CG vector updates (per-problem scalars live on the device).
// ------------------------------------------------------------------------------------------
// Initialise: active = (bb > 0); rz from the first dot; p = z.
__global__ void k_cg_init(int nb, const double* bb, int* active, int* nactive) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  int a = bb[b] > 0.0;
  active[b] = a;
  if (a) atomicAdd(nactive, 1);
}

// alpha = rz / pq for active problems; x += alpha p; r -= alpha q
template <typename T>
__global__ void k_cg_xr(long long len, int nb, const double* rz, const double* pq, const int* active,
                        const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ x,
                        T* __restrict__ r) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= len * nb) return;
  int b = (int)(idx / len);
  if (!active[b]) return;
  double a = rz[b] / pq[b];
  x[idx] = (T)((double)x[idx] + a * (double)p[idx]);
  r[idx] = (T)((double)r[idx] - a * (double)q[idx]);
}

// convergence: rr <= tol^2 bb deactivates; counts active problems.
__global__ void k_cg_check(int nb, const double* rr, const double* bb, double tol2, int* active,
                           int* nactive, const double* pq) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  if (!active[b]) return;
  if (!(rr[b] > tol2 * bb[b]) || !(pq[b] > 0.0)) {
    active[b] = 0;
    return;
  }
  atomicAdd(nactive, 1);
}

// p = z + beta p with beta = rz_new / rz_old; rz_old <- rz_new
template <typename T>
__global__ void k_cg_p(long long len, int nb, const double* rz_new, const double* rz_old,
                       const int* active, const T* __restrict__ z, T* __restrict__ p) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= len * nb) return;
  int b = (int)(idx / len);
  if (!active[b]) return;
  double beta = rz_new[b] / rz_old[b];
  p[idx] = (T)((double)z[idx] + beta * (double)p[idx]);
}

__global__ void k_copy_scalars(int nb, const double* src, double* dst, const int* active) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb && active[b]) dst[b] = src[b];
}

// ------------------------------------------------------------------------------------------
// Mean-operator preconditioner: exact solve with A0 = cm M + ck K_0 on a free set, applied to
// every PCE mode (the mean-based block-diagonal preconditioner I (x) A0^{-1}).  A0 is block
// tridiagonal over the grid lines lj; the factorisation stores S_j^{-1} (dense L x L) with
//   S_0 = D_0,  S_j = D_j - B_{j-1}^T S_{j-1}^{-1} B_{j-1}
// and the solve is a forward and a backward sweep over the lines.  B_j couples (a, j) to
// (a, j+1) (Bd) and to (a+1, j+1) (Bu).  Non-free nodes carry identity rows.
// Grid: (problem b, mode group); block (L threads, G modes).
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_line_solve(int L, int nl, int P, int R, long long pat_stride, const T* __restrict__ Sinv,
                             const T* __restrict__ Bd, const T* __restrict__ Bu,
                             const T* __restrict__ rin, T* __restrict__ zout, const int* active) {
  extern __shared__ unsigned char smem_raw[];
  T* w = reinterpret_cast<T*>(smem_raw);   // [L][G]
  T* v = w + L * blockDim.y;               // [L][G]
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  const int sub = b / R;
  const int a = threadIdx.x, m = threadIdx.y, G = blockDim.y;
  const int k = blockIdx.y * G + m;
  const bool ok = (a < L) && (k < P);
  const T* S = Sinv + (long long)sub * pat_stride;
  const T* bd = Bd + (long long)sub * L * L;
  const T* bu = Bu + (long long)sub * L * L;
  const T* rb = rin + (long long)b * nl * P;
  T* zb = zout + (long long)b * nl * P;
  // forward sweep: y_j = S_j^{-1} (r_j - B_{j-1}^T y_{j-1})
  for (int j = 0; j < L; ++j) {
    T rhs = T(0);
    if (ok) {
      rhs = rb[(long long)(j * L + a) * P + k];
      if (j > 0) {
        rhs -= bd[(j - 1) * L + a] * v[a * G + m];
        if (a > 0) rhs -= bu[(j - 1) * L + a - 1] * v[(a - 1) * G + m];
      }
    }
    __syncthreads();
    if (a < L) w[a * G + m] = rhs;
    __syncthreads();
    if (ok) {
      const T* Sj = S + (long long)j * L * L + (long long)a * L;
      T s0 = T(0), s1 = T(0);
      int c = 0;
      for (; c + 1 < L; c += 2) {
        s0 += Sj[c] * w[c * G + m];
        s1 += Sj[c + 1] * w[(c + 1) * G + m];
      }
      if (c < L) s0 += Sj[c] * w[c * G + m];
      T yv = s0 + s1;
      zb[(long long)(j * L + a) * P + k] = yv;
      v[a * G + m] = yv;
    }
    __syncthreads();
  }
  // backward sweep: x_j = y_j - S_j^{-1} B_j x_{j+1}; v holds x_{j+1}
  for (int j = L - 2; j >= 0; --j) {
    T tv = T(0);
    if (ok) {
      tv = bd[j * L + a] * v[a * G + m];
      if (a + 1 < L) tv += bu[j * L + a] * v[(a + 1) * G + m];
    }
    __syncthreads();
    if (a < L) w[a * G + m] = tv;
    __syncthreads();
    if (ok) {
      const T* Sj = S + (long long)j * L * L + (long long)a * L;
      T s0 = T(0), s1 = T(0);
      int c = 0;
      for (; c + 1 < L; c += 2) {
        s0 += Sj[c] * w[c * G + m];
        s1 += Sj[c + 1] * w[(c + 1) * G + m];
      }
      if (c < L) s0 += Sj[c] * w[c * G + m];
      const long long o = (long long)(j * L + a) * P + k;
      T xv = zb[o] - (s0 + s1);
      zb[o] = xv;
      v[a * G + m] = xv;
    }
    __syncthreads();
  }
}

// Line factorisation, FP64: one block per (subdomain, pattern).  D (within-line tridiagonal)
// diag Dd[j][a], upper Du[j][a]; coupling Bd, Bu as above.  Writes Sinv[j] (L x L).
// status[blk] = 1 when a pivot is not positive (the matrix is not SPD).
__global__ void k_line_factor(int L, const double* __restrict__ Dd, const double* __restrict__ Du,
                              const double* __restrict__ Bd, const double* __restrict__ Bu,
                              double* __restrict__ Sinv, int* status) {
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
      for (int r = threadIdx.x; r < L; r += nt) {
        col[r] = S[r * L + piv];
        prow[r] = S[piv * L + r];
      }
      __syncthreads();
      const double inv = 1.0 / d;
      for (int e = threadIdx.x; e < L * L; e += nt) {
        const int r = e / L, c = e % L;
        double val;
        if (r == piv && c == piv) val = inv;
        else if (r == piv) val = prow[c] * inv;
        else if (c == piv) val = -col[r] * inv;
        else val = S[e] - col[r] * prow[c] * inv;
        S[e] = val;
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < L * L; e += nt) out[(long long)j * L * L + e] = S[e];
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// Interface gathers / scatters.
// ------------------------------------------------------------------------------------------
// x_loc[b][ln][k] = (class in mask) ? src[gidx][k] * (useD ? D[g] : 1) : 0
template <typename T>
__global__ void k_gather(int nb, int R, int nl, int P, const uint8_t* cls, const int* gidx, const double* D,
                         const double* __restrict__ src, T* __restrict__ dst, int mask, int useD) {
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

// dst[g][k] = sum over owners o of src[o][k] (* D[g] when useD); owners are (sub * nl + ln), R = 1
template <typename T>
__global__ void k_scatter(int nG, int P, const int* owners, const double* D, const T* __restrict__ src,
                          double* __restrict__ dst, int useD) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nG * P) return;
  const int k = (int)(idx % P), g = (int)(idx / P);
  double s = 0.0;
  for (int q = 0; q < 4; ++q) {
    const int o = owners[g * 4 + q];
    if (o >= 0) s += (double)src[(long long)o * P + k];
  }
  if (useD) s *= D[g];
  dst[idx] = s;
}

// Sum the interface values of all owners and write the sum back to every owner (global
// assembly of a local-layout vector on the interface).
__global__ void k_assemble_gamma(int nG, int P, const int* owners, double* __restrict__ v) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nG * P) return;
  const int k = (int)(idx % P), g = (int)(idx / P);
  double s = 0.0;
  for (int q = 0; q < 4; ++q) {
    const int o = owners[g * 4 + q];
    if (o >= 0) s += v[(long long)o * P + k];
  }
  for (int q = 0; q < 4; ++q) {
    const int o = owners[g * 4 + q];
    if (o >= 0) v[(long long)o * P + k] = s;
  }
}

// weight for counting each global dof once in local-layout dots: 1 on interior, D on interface
__global__ void k_node_weight(int n, const uint8_t* cls, const int* gidx, const double* D, double* w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = cls[i];
  w[i] = c == DIR ? 0.0 : (c == INT ? 1.0 : D[gidx[i]]);
}

// res = sum_i w[node(i)] x_i y_i over a local-layout vector (single block, fixed order)
__global__ void k_dot_w(long long nnodes, int P, const double* w, const double* x, const double* y,
                        double* res) {
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
__global__ void k_coarse_extend(int nsub, int nl, int P, int nGam, int maxc, const uint8_t* cls,
                                const int* cidx, const int* gam_ln, const int* n_gam, const int* loc_corner,
                                const int* n_loc_corner, const double* __restrict__ Phi,
                                const double* __restrict__ uc, const double* __restrict__ v,
                                double* __restrict__ zloc) {
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
    val = v[so * P + k];
    const int nc = n_loc_corner[sub];
    const int ncolmax = maxc * P;
    for (int lc = 0; lc < nc; ++lc) {
      const int cg = cidx[(long long)sub * nl + loc_corner[sub * 4 + lc]];
      for (int m = 0; m < P; ++m) {
        const int col = lc * P + m;
        val += Phi[(((long long)sub * ncolmax + col) * nGam + q) * P + k] * uc[(long long)cg * P + m];
      }
    }
  }
  zloc[so * P + k] = val;
}

// d[c][k] = sum over owners o of (wc - y)[o][k]
__global__ void k_corner_rhs(int nC, int P, const int* cowners, const double* __restrict__ wc,
                             const double* __restrict__ y, double* __restrict__ d) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nC * P) return;
  const int k = (int)(idx % P), c = (int)(idx / P);
  double s = 0.0;
  for (int q = 0; q < 4; ++q) {
    const int o = cowners[c * 4 + q];
    if (o >= 0) s += wc[(long long)o * P + k] - y[(long long)o * P + k];
  }
  d[idx] = s;
}

// y = A x for a dense n x n row-major matrix (one warp per row)
__global__ void k_gemv(int n, const double* __restrict__ A, const double* __restrict__ x,
                       double* __restrict__ y) {
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
__global__ void k_coarse_units(int nsub, int R, int nl, int P, int sub0, const int* loc_corner,
                               const int* n_loc_corner, double* e) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nsc = nsub;
  if (idx >= (long long)nsc * R) return;
  const int col = (int)(idx % R), sl = (int)(idx / R);
  const int sub = sub0 + sl;
  const int lc = col / P, m = col % P;
  if (lc >= n_loc_corner[sub]) return;
  const int ln = loc_corner[sub * 4 + lc];
  e[(((long long)sl * R + col) * nl + ln) * P + m] = 1.0;
}

// Phi[sub][col][q][k] = v[b][gam_ln[q]][k] on remaining nodes (0 on corners)
__global__ void k_coarse_phi(int nsub_chunk, int sub0, int R, int nl, int P, int nGam, const uint8_t* cls,
                             const int* gam_ln, const int* n_gam, const double* __restrict__ v,
                             double* __restrict__ Phi) {
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
    if (cls[(long long)sub * nl + ln] == REM) val = v[(((long long)sl * R + col) * nl + ln) * P + k];
  }
  Phi[(((long long)sub * R + col) * nGam + q) * P + k] = val;
}

// local coarse matrix entries: Fs[sub][row = lc'*P+m'][col] = y[b(col)][loc_corner[lc']][m']
__global__ void k_coarse_fs(int nsub_chunk, int sub0, int R, int nl, int P, const int* loc_corner,
                            const int* n_loc_corner, const double* __restrict__ y, double* __restrict__ Fs) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nsub_chunk * R * R) return;
  const int col = (int)(idx % R);
  long long t = idx / R;
  const int row = (int)(t % R), sl = (int)(t / R);
  const int sub = sub0 + sl;
  const int lr = row / P, mr = row % P;
  double val = 0.0;
  if (lr < n_loc_corner[sub] && col / P < n_loc_corner[sub]) {
    const int ln = loc_corner[sub * 4 + lr];
    val = y[(((long long)sl * R + col) * nl + ln) * P + mr];
  }
  Fs[((long long)sub * R + row) * R + col] = val;
}

// ------------------------------------------------------------------------------------------
// Newmark and loads.
// ------------------------------------------------------------------------------------------
// um = (U + dt V)/(zeta dt^2) + (1 - 2 zeta) A/(2 zeta); uc = gamma dt um - V - (1-gamma) dt A
// xm = um + alpha0 uc (mass input of the effective load), all on free nodes (Eqs. UmCm)
__global__ void k_newmark_pre(long long n, double dt, double alpha0, const double* __restrict__ U,
                              const double* __restrict__ V, const double* __restrict__ A,
                              double* __restrict__ um, double* __restrict__ uc, double* __restrict__ xm) {
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
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double zeta = 0.25, gamma = 0.5;
  const double an = Un[i] / (zeta * dt * dt) - um[i];
  V[i] = V[i] + dt * ((1.0 - gamma) * A[i] + gamma * an);
  A[i] = an;
  U[i] = Un[i];
}

// point source: f[node][0] += w * amp * ricker(t)  (amp folded into w)
__global__ void k_point_load(int n, const int* node, const double* w, double t, double freq, int P,
                             double* f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double pi = 3.14159265358979323846;
  const double tau = t - 1.0 / freq;
  const double a = (pi * freq * tau) * (pi * freq * tau);
  f[(long long)node[i] * P] += w[i] * (1.0 - 2.0 * a) * exp(-a);
}

// external nodal load (mode 0) split over the owners with D_s
__global__ void k_ext_load(long long nloc, int P, const int* free_of_local, const uint8_t* cls,
                           const int* gidx, const double* D, const double* __restrict__ fext,
                           double* __restrict__ f) {
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
__global__ void k_scatter_free(long long nloc, int P, const int* free_of_local, const double* __restrict__ src,
                               double* __restrict__ dst) {
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
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

template <typename T, typename U>
__global__ void k_convert(long long n, const T* __restrict__ x, U* __restrict__ y) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (U)x[i];
}

// keep values on nodes whose class is in mask, zero elsewhere (R right-hand sides per subdomain)
template <typename T>
__global__ void k_mask(int nb, int R, int nl, int P, const uint8_t* cls, const T* __restrict__ x,
                       T* __restrict__ y, int mask) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nb * nl * P) return;
  const long long t = idx / P;
  const int ln = (int)(t % nl), b = (int)(t / nl);
  y[idx] = ((mask >> cls[(long long)(b / R) * nl + ln]) & 1) ? x[idx] : T(0);
}

template <typename T>
__global__ void k_finite(long long n, const T* __restrict__ x, int* bad) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite((double)x[i])) *bad = 1;
}

}  // namespace sgk
