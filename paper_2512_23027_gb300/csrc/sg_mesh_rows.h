// Per-row arithmetic of the general-partition (unstructured mesh) path: the SG operator apply and
// the dense mean-operator preconditioner on the sparse-row layout built by sgh::mesh_to_problem.
// Host/device neutral: the CUDA kernels of sg_mesh.cuh call these functions, and so can a host
// program that checks them.
#pragma once

#ifdef __CUDACC__
#define SG_HD __host__ __device__ __forceinline__
#else
#define SG_HD inline
#endif

namespace sgm {

// Sparse rows of the local layout (nl rows per subdomain) and the triple-product table grouped by
// the output mode k (entries [gk_ptr[k], gk_ptr[k+1]) hold the input mode i, the vector mode j and
// the value G_ijk).
template <typename T>
struct Rows {
  const int* rp;        // row pointers, nsub * nl + 1
  const int* col;       // local column, same subdomain
  const T* kv;          // entries x PI: K_i[a][b]
  const T* mv;          // entries: M[a][b]
  const int* gk_ptr;
  const int* gk_i;
  const int* gk_j;
  const T* gk_v;
  int nl, P, PI;
};

// Mode k of row `row` (= sub * nl + a) of cm (M (x) I) xm + ck (sum_i K_i (x) G_i) xk, where xm and xk
// point at the first row of the problem's local vectors (node-major, P modes per node):
//   sum_b cm M[a][b] xm[b][k] + ck sum_b sum_{(i,j) : G_ijk != 0} G_ijk K_i[a][b] xk[b][j]
// (Sec. 4, Eq. stok: [K]_{jk} = sum_i G_ijk K_i; deterministic mass block-diagonal over the modes).
template <typename T>
SG_HD T apply_row(const Rows<T>& r, long long row, int k, const T* xm, const T* xk, T cm, T ck) {
  T acc = T(0);
  const int e0 = r.rp[row], e1 = r.rp[row + 1];
  const int g0 = r.gk_ptr[k], g1 = r.gk_ptr[k + 1];
  for (int e = e0; e < e1; ++e) {
    const long long cb = (long long)r.col[e] * r.P;
    if (cm != T(0)) acc += cm * r.mv[e] * xm[cb + k];
    if (ck != T(0)) {
      const T* kw = r.kv + (long long)e * r.PI;
      T s = T(0);
      for (int g = g0; g < g1; ++g) s += r.gk_v[g] * kw[r.gk_i[g]] * xk[cb + r.gk_j[g]];
      acc += ck * s;
    }
  }
  return acc;
}

// Mode k of row `row` of (am M (x) I + bk sum_i K_i (x) G_i) p for a CG direction formed on the fly,
// p = z + bet pold (pold is read only when bet != 0, so that it may hold anything before the first
// direction): am sum_b M[a][b] p[b][k] + bk sum_b sum_{(i,j)} G_ijk K_i[a][b] p[b][j].
template <typename T>
SG_HD T apply_row_dir(const Rows<T>& r, long long row, int k, const T* z, const T* pold, T bet, T am, T bk) {
  T acc = T(0);
  const int e0 = r.rp[row], e1 = r.rp[row + 1];
  const int g0 = r.gk_ptr[k], g1 = r.gk_ptr[k + 1];
  const bool usep = bet != T(0);
  for (int e = e0; e < e1; ++e) {
    const long long cb = (long long)r.col[e] * r.P;
    const T pk = usep ? z[cb + k] + bet * pold[cb + k] : z[cb + k];
    T s = T(0);
    const T* kw = r.kv + (long long)e * r.PI;
    for (int g = g0; g < g1; ++g) {
      const long long j = cb + r.gk_j[g];
      const T pj = usep ? z[j] + bet * pold[j] : z[j];
      s += r.gk_v[g] * kw[r.gk_i[g]] * pj;
    }
    acc += am * r.mv[e] * pk + bk * s;
  }
  return acc;
}

// Mode k of row a of (I (x) A0^{-1}) rv on a pattern of n rows: sum_{c < n} Ainv[a][c] rv[c][k], with
// `arow` row a of the subdomain's inverse (nl columns, zero beyond n) and rv the problem's vector.
template <typename T>
SG_HD T dense_row(const T* arow, const T* rv, int n, int P, int k) {
  T acc = T(0);
  for (int c = 0; c < n; ++c) acc += arow[c] * rv[(long long)c * P + k];
  return acc;
}

}  // namespace sgm
