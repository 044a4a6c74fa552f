// Compile-time structure of the Galerkin triple products for fixed PCE sizes.
//
// The SG stiffness flux of an edge e is z_e[k] = sum_{(i,j,k)} kappa_i(e) G_ijk d_e[j] (Sec. 4,
// Eq. stoksub).  Which (i, j, k) are nonzero depends only on the number of random variables M, the
// output order p and the input order p_in: for orthonormal Hermite chaos, G_ijk factorises over the
// variables and the 1-D factor <psi_a psi_b psi_c> is nonzero exactly when a + b + c is even and
// s = (a + b + c) / 2 >= max(a, b, c).  This header enumerates the multi-indices (graded, descending
// lexicographic inside a degree, the order the host set-up uses) and the nonzero triples (grouped by
// output mode k, then i, then j) as constant expressions, so that a kernel instantiated for one
// (M, p, p_in) addresses its register arrays with constant indices and reads each G value as a
// constant-bank operand.  The values themselves are uploaded by the host into c_gvf / c_gvd.
#pragma once
#include <utility>

namespace sgk {
namespace gfix {

constexpr int MAXM = 5;    // random variables
constexpr int MAXN = 56;   // multi-indices (M = 5, p = 3)

struct MSet {
  int n;
  signed char a[MAXN][MAXM];
};

// multi-indices |alpha| <= p in graded order; inside a degree, descending lexicographic
constexpr MSet multi(int M, int p) {
  MSet r{};
  r.n = 0;
  for (int d = 0; d <= p; ++d) {
    int t[MAXM] = {0, 0, 0, 0, 0};
    for (int m = 0; m < M; ++m) t[m] = d;
    for (;;) {  // odometer over [0, d]^M, counting down from (d, ..., d)
      int s = 0;
      for (int m = 0; m < M; ++m) s += t[m];
      if (s == d) {
        for (int m = 0; m < M; ++m) r.a[r.n][m] = (signed char)t[m];
        ++r.n;
      }
      int m = M - 1;
      while (m >= 0 && t[m] == 0) --m;
      if (m < 0) break;
      --t[m];
      for (int q = m + 1; q < M; ++q) t[q] = d;
    }
  }
  return r;
}

constexpr bool nonzero(const MSet& in, int i, const MSet& out, int j, int k, int M) {
  for (int m = 0; m < M; ++m) {
    const int a = in.a[i][m], b = out.a[j][m], c = out.a[k][m];
    const int t = a + b + c;
    if (t & 1) return false;
    const int s = t / 2;
    if (s < a || s < b || s < c) return false;
  }
  return true;
}

constexpr int count(int M, int p, int pin) {
  const MSet out = multi(M, p), in = multi(M, pin);
  int n = 0;
  for (int k = 0; k < out.n; ++k)
    for (int i = 0; i < in.n; ++i)
      for (int j = 0; j < out.n; ++j) n += nonzero(in, i, out, j, k, M) ? 1 : 0;
  return n;
}

template <int N>
struct Tab {
  short i[N], j[N], k[N];
  int kptr[MAXN + 1];
};

template <int N>
constexpr Tab<N> table(int M, int p, int pin) {
  const MSet out = multi(M, p), in = multi(M, pin);
  Tab<N> t{};
  int n = 0;
  for (int k = 0; k < out.n; ++k) {
    t.kptr[k] = n;
    for (int i = 0; i < in.n; ++i)
      for (int j = 0; j < out.n; ++j)
        if (nonzero(in, i, out, j, k, M)) {
          t.i[n] = (short)i;
          t.j[n] = (short)j;
          t.k[n] = (short)k;
          ++n;
        }
  }
  t.kptr[out.n] = n;
  return t;
}

// One compiled PCE size.  OFF: offset of its values in the constant-memory G table.  KG: output-mode
// groups per edge (work items per edge in the flux phase), split at mode boundaries with about
// NNZ / KG entries each.
template <int M_, int P_ORD, int PIN, int OFF_>
struct Cfg {
  static constexpr bool fixed = true;
  static constexpr bool nods = false;
  static constexpr bool gglob = false;
  static constexpr int M = M_, p = P_ORD, pin = PIN, OFF = OFF_;
  static constexpr int P = multi(M_, P_ORD).n, PI = multi(M_, PIN).n;
  static constexpr int NNZ = count(M_, P_ORD, PIN);
  static constexpr int KG = NNZ >= 300 ? 4 : NNZ >= 100 ? 2 : 1;
  static constexpr Tab<NNZ> tab = table<NNZ>(M_, P_ORD, PIN);
  static constexpr int ti(int e) { return tab.i[e]; }
  static constexpr int tj(int e) { return tab.j[e]; }
  static constexpr int tk(int e) { return tab.k[e]; }
  static constexpr int kptr(int k) { return tab.kptr[k]; }
  // first output mode of group g: smallest k whose entries start at or after g * NNZ / KG
  static constexpr int kbeg(int g) {
    if (g <= 0) return 0;
    if (g >= KG) return P;
    int k = 0;
    while (k < P && tab.kptr[k] * KG < g * NNZ) ++k;
    return k;
  }
};

// The compiled sizes: every (M, p) of the workloads, input order p_in = p.
using C0 = Cfg<2, 2, 2, 0>;
using C1 = Cfg<2, 3, 3, C0::OFF + C0::NNZ>;
using C2 = Cfg<3, 2, 2, C1::OFF + C1::NNZ>;
using C3 = Cfg<3, 3, 3, C2::OFF + C2::NNZ>;
using C4 = Cfg<4, 2, 2, C3::OFF + C3::NNZ>;
using C5 = Cfg<4, 3, 3, C4::OFF + C4::NNZ>;
using C6 = Cfg<5, 2, 2, C5::OFF + C5::NNZ>;
constexpr int NCFG = 7;
constexpr int GV_CAP = C6::OFF + C6::NNZ;

}  // namespace gfix

__constant__ float c_gvf[gfix::GV_CAP];   // G values of every compiled size (FP32 copy)
__constant__ double c_gvd[gfix::GV_CAP];  // the same values in FP64
__constant__ float c_gvf_lo[gfix::GV_CAP];  // G - (double) c_gvf: the low part of a float-float G

template <typename T>
__device__ __forceinline__ T gval(int e);
template <>
__device__ __forceinline__ float gval<float>(int e) { return c_gvf[e]; }
template <>
__device__ __forceinline__ double gval<double>(int e) { return c_gvd[e]; }

// Scalar constant members (usable in device code) for entry E and for mode group G of a size C;
// the table itself is only read during compile-time evaluation.
template <class C, int E>
struct Ent {
  static constexpr int I = C::ti(E), J = C::tj(E), K = C::tk(E);
};
template <class C, int G>
struct Grp {
  static constexpr int K0 = C::kbeg(G), K1 = C::kbeg(G + 1);
  static constexpr int E0 = C::kptr(K0), E1 = C::kptr(K1);
};

// one triple-product term: z[k] += G_ijk * (kappa[i] * d[j]) with constant i, j, k
template <class C, typename T, int E>
__device__ __forceinline__ void gterm(const T (&kap)[C::PI], const T (&d)[C::P], T (&z)[C::P]) {
  using X = Ent<C, E>;
  z[X::K] = fma(gval<T>(C::OFF + E), kap[X::I] * d[X::J], z[X::K]);
}

template <class C, typename T, int E0, int... E>
__device__ __forceinline__ void gterms(const T (&kap)[C::PI], const T (&d)[C::P], T (&z)[C::P],
                                       std::integer_sequence<int, E...>) {
  (gterm<C, T, E0 + E>(kap, d, z), ...);
}

// Flux of one edge for the output modes of group G: reads kappa(e) from global memory (kp) and the
// two end-point values from shared memory (xa - xb), writes z_e[k] for the group's modes to zo.
template <class C, typename T, int G>
__device__ __forceinline__ void gflux_group(const T* __restrict__ kp, const T* xa, const T* xb, T* zo, bool live) {
  constexpr int K0 = Grp<C, G>::K0, K1 = Grp<C, G>::K1;
  constexpr int E0 = Grp<C, G>::E0, E1 = Grp<C, G>::E1;
  T z[C::P];
#pragma unroll
  for (int k = K0; k < K1; ++k) z[k] = T(0);
  if (live) {
    T kap[C::PI], d[C::P];
#pragma unroll
    for (int i = 0; i < C::PI; ++i) kap[i] = __ldg(kp + i);
#pragma unroll
    for (int j = 0; j < C::P; ++j) d[j] = xa[j] - xb[j];
    gterms<C, T, E0>(kap, d, z, std::make_integer_sequence<int, E1 - E0>{});
  }
#pragma unroll
  for (int k = K0; k < K1; ++k) zo[k] = z[k];
}

template <class C, typename T>
__device__ __forceinline__ void gflux(int g, const T* __restrict__ kp, const T* xa, const T* xb, T* zo, bool live) {
  switch (g) {
    case 0: gflux_group<C, T, 0>(kp, xa, xb, zo, live); break;
    case 1: if constexpr (C::KG > 1) gflux_group<C, T, 1>(kp, xa, xb, zo, live); break;
    case 2: if constexpr (C::KG > 2) gflux_group<C, T, 2>(kp, xa, xb, zo, live); break;
    case 3: if constexpr (C::KG > 3) gflux_group<C, T, 3>(kp, xa, xb, zo, live); break;
    default: break;
  }
}

// ---- float-float flux (unevaluated sums of two FP32 values, ~2^-44 relative) for FP64 applies ----
// Error-free transformations: TwoSum (Knuth) for sums, the fused multiply-add for the exact rounding
// error of a product.  A value is (h, l) with |l| <= ulp(h) / 2 after normalisation; the inner loop
// keeps the accumulator's low part unnormalised (it only collects error terms).  The explicitly
// rounded intrinsics (__fadd_rn, __fmul_rn) keep the compiler from contracting a rounded product
// into a following sum, which would break the transformations.
struct f2 {
  float h, l;
};
__device__ __forceinline__ f2 f2_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double f2_to(f2 a) { return (double)a.h + (double)a.l; }

// FP64 <-> float-float with a power-of-two scale, by integer operations on the bit patterns (FP64
// instructions, conversions included, issue at a small fraction of the FP32 rate on this part).
// f2_split_scaled(x, ex) = x 2^-ex as (h, l): h is x's leading 24 significant bits (truncated), l the
// rest of its 53 rounded to 24 bits, so h + l = x 2^-ex to about 2^-47 relative.  Values whose scaled
// magnitude is below the FP32 normal range give 0 (l alone below it gives l = 0); Inf and NaN give NaN.
__device__ __forceinline__ f2 f2_split_scaled(double x, int ex) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sgn = hi & 0x80000000u;
  const int E = (int)((hi >> 20) & 0x7ffu);
  if (E == 0x7ff) return {__uint_as_float(0x7fc00000u), 0.f};
  const int Ef = E - ex - 1023 + 127;               // biased FP32 exponent of h
  if (Ef <= 0) return {0.f, 0.f};
  const float h = __uint_as_float(sgn | ((unsigned)Ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  float l = 0.f;
  if (Ef > 52) l = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), __uint_as_float((unsigned)(Ef - 52) << 23));
  return {h, __uint_as_float(__float_as_uint(l) ^ sgn)};
}
// a (normal) FP32 value times 2^ex as FP64, exactly; FP32 zeros and subnormals give 0, overflow Inf
__device__ __forceinline__ double f32_to_f64_scaled(float f, int ex) {
  const unsigned u = __float_as_uint(f);
  const unsigned sgn = u & 0x80000000u;
  const int e8 = (int)((u >> 23) & 0xffu);
  if (e8 == 0) return 0.0;
  if (e8 == 0xff) return __hiloint2double((int)(sgn | 0x7ff80000u), 0);
  const int E = e8 - 127 + 1023 + ex;
  if (E <= 0) return 0.0;
  if (E >= 0x7ff) return __hiloint2double((int)(sgn | 0x7ff00000u), 0);
  const unsigned m = u & 0x7fffffu;
  return __hiloint2double((int)(sgn | ((unsigned)E << 20) | (m >> 3)), (int)(m << 29));
}
__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 s = two_sum(a.h, b.h);
  s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) { return f2_add(a, {-b.h, -b.l}); }
// product with normalisation
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}

// one triple-product term in float-float: z[k] += G_ijk * (kappa[i] * d[j])
template <class C, int E>
__device__ __forceinline__ void gterm_f2(const f2 (&kap)[C::PI], const f2 (&d)[C::P], f2 (&z)[C::P]) {
  using X = Ent<C, E>;
  const f2 a = kap[X::I], b = d[X::J];
  // t = a * b, unnormalised (p, e)
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  // u = G * t
  const float gh = c_gvf[C::OFF + E], gl = c_gvf_lo[C::OFF + E];
  const float uh = __fmul_rn(gh, p);
  float ue = fmaf(gh, p, -uh);
  ue = fmaf(gh, e, ue);
  ue = fmaf(gl, p, ue);
  // z += u: TwoSum on the high parts, error terms into the low part
  const f2 s = two_sum(z[X::K].h, uh);
  z[X::K].h = s.h;
  z[X::K].l = __fadd_rn(z[X::K].l, __fadd_rn(s.l, ue));
}

template <class C, int E0, int... E>
__device__ __forceinline__ void gterms_f2(const f2 (&kap)[C::PI], const f2 (&d)[C::P], f2 (&z)[C::P],
                                          std::integer_sequence<int, E...>) {
  (gterm_f2<C, E0 + E>(kap, d, z), ...);
}

// Flux of one edge for the output modes of group G in float-float: kappa(e) from the float-float
// copy of the edge weights (kp: PI pairs), end-point values from shared memory (pairs).
template <class C, int G>
__device__ __forceinline__ void gflux_group_f2(const float2* __restrict__ kp, const f2* xa, const f2* xb, f2* zo,
                                               bool live) {
  constexpr int K0 = Grp<C, G>::K0, K1 = Grp<C, G>::K1;
  constexpr int E0 = Grp<C, G>::E0, E1 = Grp<C, G>::E1;
  f2 z[C::P];
#pragma unroll
  for (int k = K0; k < K1; ++k) z[k] = {0.f, 0.f};
  if (live) {
    f2 kap[C::PI], d[C::P];
#pragma unroll
    for (int i = 0; i < C::PI; ++i) {
      const float2 v = __ldg(kp + i);
      kap[i] = {v.x, v.y};
    }
#pragma unroll
    for (int j = 0; j < C::P; ++j) d[j] = f2_sub(xa[j], xb[j]);
    gterms_f2<C, E0>(kap, d, z, std::make_integer_sequence<int, E1 - E0>{});
  }
#pragma unroll
  for (int k = K0; k < K1; ++k) zo[k] = fast_two_sum(z[k].h, z[k].l);
}

template <class C>
__device__ __forceinline__ void gflux_f2(int g, const float2* __restrict__ kp, const f2* xa, const f2* xb, f2* zo,
                                         bool live) {
  switch (g) {
    case 0: gflux_group_f2<C, 0>(kp, xa, xb, zo, live); break;
    case 1: if constexpr (C::KG > 1) gflux_group_f2<C, 1>(kp, xa, xb, zo, live); break;
    case 2: if constexpr (C::KG > 2) gflux_group_f2<C, 2>(kp, xa, xb, zo, live); break;
    case 3: if constexpr (C::KG > 3) gflux_group_f2<C, 3>(kp, xa, xb, zo, live); break;
    default: break;
  }
}

// the generic (runtime-G) variant of the apply kernel
struct GDyn {
  static constexpr bool fixed = false;
  static constexpr bool nods = false;
  static constexpr bool gglob = false;
  static constexpr int KG = 1;
};
// runtime table without the staged edge differences (subdomains too wide for the staging tiles)
struct GDynNoDS {
  static constexpr bool fixed = false;
  static constexpr bool nods = true;
  static constexpr bool gglob = false;
  static constexpr int KG = 1;
};
// the same with the triple-product table read from global memory (through L1) instead of staged:
// input lines and fluxes of a one-line tile of the widest FP64 subdomains fill shared memory alone
struct GDynNoDSG {
  static constexpr bool fixed = false;
  static constexpr bool nods = true;
  static constexpr bool gglob = true;
  static constexpr int KG = 1;
};

}  // namespace sgk
