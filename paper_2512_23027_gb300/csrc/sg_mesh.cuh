// Kernels of the general-partition path (unstructured triangle meshes, any element partition).
//
// The local layout of a subdomain is the list of its free vertices (interior, remaining, corners;
// Sec. 3 classes), padded to nl rows; the operators are sparse rows of that layout (sgm::Rows), the
// subdomain solves (local Dirichlet and Neumann problems of Sec. 3, in the stochastic form of Sec. 5)
// are a batched CG preconditioned by the dense inverse of the subdomain's mean operator
// am M + bk K_0 (the same preconditioner as the line sweeps of the structured path, which solve that
// operator exactly).  Everything else of the step (interface PCG, two-level preconditioner, coarse
// solve, Newmark update) is the structured path's code on the same generic tables.
#pragma once
#include "sg_mesh_rows.h"

namespace sgk {

// y = add + cm (M (x) I) xm + ck (sum_i K_i (x) G_i) xk on rows whose class is in out_mask, 0 on the
// other rows; nb problems of nl * P values, problem b on subdomain s0 + b / R.  With `active`, the
// problems whose flag is 0 are skipped (y keeps its values).  y may alias add, not xm or xk.
template <typename T, typename TO>
__global__ void __launch_bounds__(256) k_mapply(sgm::Rows<T> r, const uint8_t* __restrict__ cls, int s0, int nb,
                                                int R, const T* __restrict__ xm, const T* __restrict__ xk, TO* y,
                                                const TO* add, T cm, T ck, int out_mask, const int* active) {
  count_launch();
  const long long len = (long long)r.nl * r.P;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= len * nb) return;
  const int b = (int)(idx / len);
  if (active && !active[b]) return;
  const long long t = idx - (long long)b * len;
  const int a = (int)(t / r.P), k = (int)(t - (long long)a * r.P);
  const long long row = (long long)(s0 + b / R) * r.nl + a;
  TO out = TO(0);
  if ((out_mask >> cls[row]) & 1) {
    out = (TO)sgm::apply_row(r, row, k, xm + (long long)b * len, xk + (long long)b * len, cm, ck);
    if (add) out += add[idx];
  }
  y[idx] = out;
}

// z = (I (x) A0^{-1}) rv per problem on the rows of its pattern (the first npat[sub] local rows), 0 on
// the other rows; Ainv holds nl x nl per subdomain (zero beyond npat).  Inactive problems are skipped.
template <typename T>
__global__ void __launch_bounds__(256) k_mdense(const T* __restrict__ Ainv, const int* __restrict__ npat, int s0,
                                                int nb, int R, int nl, int P, const T* __restrict__ rv,
                                                T* __restrict__ z, const int* active) {
  count_launch();
  const long long len = (long long)nl * P;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= len * nb) return;
  const int b = (int)(idx / len);
  if (active && !active[b]) return;
  const long long t = idx - (long long)b * len;
  const int a = (int)(t / P), k = (int)(t - (long long)a * P);
  const int sub = s0 + b / R;
  const int n = npat[sub];
  T v = T(0);
  if (a < n) v = sgm::dense_row(Ainv + ((long long)sub * nl + a) * nl, rv + (long long)b * len, n, P, k);
  z[idx] = v;
}

// out1[b] = x1 . y1 and, when x2 is given, out2[b] = x2 . y2 over problem b's vector of len values:
// FP64 sums in a fixed order (strided per thread, then a tree over the block).  One block of
// MDOT_THREADS threads per problem; inactive problems are skipped.
constexpr int MDOT_THREADS = 256;
template <typename T>
__global__ void __launch_bounds__(MDOT_THREADS) k_mdot2(long long len, const T* __restrict__ x1,
                                                        const T* __restrict__ y1, double* out1,
                                                        const T* __restrict__ x2, const T* __restrict__ y2,
                                                        double* out2, const int* active) {
  count_launch();
  const int b = blockIdx.x;
  if (active && !active[b]) return;  // uniform over the block
  const long long o = (long long)b * len;
  double s1 = 0.0, s2 = 0.0;
  for (long long i = threadIdx.x; i < len; i += MDOT_THREADS) {
    s1 += (double)x1[o + i] * (double)y1[o + i];
    if (x2) s2 += (double)x2[o + i] * (double)y2[o + i];
  }
  __shared__ double r1[MDOT_THREADS], r2[MDOT_THREADS];
  r1[threadIdx.x] = s1;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int w = MDOT_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      r1[threadIdx.x] += r1[threadIdx.x + w];
      r2[threadIdx.x] += r2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out1[b] = r1[0];
    if (x2) out2[b] = r2[0];
  }
}

// CG step of every active problem: alpha = rz / pq, x += alpha p, r -= alpha q (pq in part_pq[b]).
// A problem whose pq is not positive keeps x and r; the control kernel then stops it.
template <typename T>
__global__ void __launch_bounds__(256) k_mcg_upd(long long len, int nb, CgCtl ctl, T* __restrict__ x,
                                                 T* __restrict__ r, const T* __restrict__ p,
                                                 const T* __restrict__ q) {
  count_launch();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= len * nb) return;
  const int b = (int)(idx / len);
  if (!ctl.active[b]) return;
  const double pq = ctl.part_pq[b];
  if (!(pq > 0.0) || !isfinite(pq)) return;
  const T alpha = (T)(ctl.rz[b] / pq);
  x[idx] += alpha * p[idx];
  r[idx] -= alpha * q[idx];
}

// Per-problem control after the preconditioner (one block): r.r and r.z in part_rr[b], part_rz[b].
// init: ||b||^2 and r.z of the start, active when the right-hand side is above the underflow level;
// otherwise a problem stops when ||r||^2 <= tol2 ||b||^2 or at a breakdown (p.q or r.z not positive,
// non-finite values, which also set the breakdown flag), else beta = rz_new / rz.  Sets the loop
// condition (some problem active and fewer than max_it iterations) on the device mirror and, inside a
// captured graph, on the conditional node.
__global__ void __launch_bounds__(256) k_mcg_ctl(int nb, CgCtl ctl, int init, double tol2, double bb_min,
                                                 int max_it, cudaGraphConditionalHandle cond_handle,
                                                 int use_handle) {
  count_launch();
  __shared__ int n_act;
  if (threadIdx.x == 0) n_act = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double rr = ctl.part_rr[b], rz = ctl.part_rz[b];
    if (init) {
      ctl.bb[b] = rr;
      ctl.rz[b] = rz;
      ctl.beta[b] = 0.0;
      if (!isfinite(rr) || !isfinite(rz)) ctl.breakdown[0] = 1;
      const int ac = rr > bb_min && isfinite(rr) && rz > 0.0;
      ctl.active[b] = ac;
      if (ac) atomicAdd(&n_act, 1);
    } else if (ctl.active[b]) {
      const double pq = ctl.part_pq[b];
      if (!isfinite(rr) || !isfinite(rz)) ctl.breakdown[0] = 1;
      const bool stop = !(pq > 0.0) || !isfinite(pq) || !isfinite(rr) || !(rz > 0.0);
      if (stop || !(rr > tol2 * ctl.bb[b])) {
        ctl.active[b] = 0;
      } else {
        ctl.beta[b] = rz / ctl.rz[b];
        ctl.rz[b] = rz;
        atomicAdd(&n_act, 1);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int itn = init ? 0 : (*ctl.it + 1);
    *ctl.it = itn;
    if (!init) *ctl.it_total += 1;
    const int cond = (n_act > 0) && (itn < max_it);
    *ctl.cond = cond;
    if (use_handle) cudaGraphSetConditional(cond_handle, cond ? 1u : 0u);
  }
}

// Search direction of every active problem: p = z (init) or p = z + beta p.
template <typename T>
__global__ void __launch_bounds__(256) k_mcg_dir(long long len, int nb, CgCtl ctl, int init, const T* __restrict__ z,
                                                 T* __restrict__ p) {
  count_launch();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= len * nb) return;
  const int b = (int)(idx / len);
  if (!ctl.active[b]) return;
  p[idx] = init ? z[idx] : z[idx] + (T)ctl.beta[b] * p[idx];
}

// Direction and product of the tensor-core CG loop (the contract of the structured fused apply, which
// k_cg_pack and k_pre_mma follow): p_new = z + beta p_old with p_old = parity ? p1 : p0 and p_new the
// other buffer, q = A p_new on the pattern rows (0 elsewhere; p_new at the neighbours is formed on
// the fly from z and p_old), and the partial of p_new . q of block (b, tile) in part_pq[b * NT + tile].
// Grid: nb x NT blocks of 256 threads, block tile covering entries [256 tile, 256 tile + 256) of the
// problem's nl * P values.  Inactive problems are skipped.
template <typename T>
__global__ void __launch_bounds__(256) k_mapply_cg(sgm::Rows<T> r, const uint8_t* __restrict__ cls, int s0, int R,
                                                   int NT, const T* __restrict__ z, T* p0, T* p1, T* __restrict__ q,
                                                   T am, T bk, int out_mask, CgCtl ctl) {
  count_launch();
  const int b = blockIdx.x / NT, tile = blockIdx.x - (blockIdx.x / NT) * NT;
  if (!ctl.active[b]) return;  // uniform over the block
  const int par = *ctl.parity;
  const T* pold = par ? p1 : p0;
  T* pnew = par ? p0 : p1;
  const T bet = (T)ctl.beta[b];
  const long long len = (long long)r.nl * r.P;
  const long long t = (long long)tile * 256 + threadIdx.x;
  double s = 0.0;
  if (t < len) {
    const long long o = (long long)b * len;
    const int a = (int)(t / r.P), k = (int)(t - (long long)a * r.P);
    const long long row = (long long)(s0 + b / R) * r.nl + a;
    const T pn = bet != T(0) ? z[o + t] + bet * pold[o + t] : z[o + t];
    pnew[o + t] = pn;
    T out = T(0);
    if ((out_mask >> cls[row]) & 1) out = sgm::apply_row_dir(r, row, k, z + o, pold + o, bet, am, bk);
    q[o + t] = out;
    s = (double)pn * (double)out;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) ctl.part_pq[(long long)b * NT + tile] = red[0];
}

}  // namespace sgk
