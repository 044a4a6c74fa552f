// Mean-operator preconditioner of the FP32 subdomain CG as a dense tensor-core product (sm_103a).
//
// The inner CG of the subdomain solves is preconditioned by I (x) A0^{-1}, A0 = a_m M + b_k K_0 on the
// pattern's free nodes (the mean of the SG operator, Sec. 4).  For subdomains of up to about 40 x 40
// nodes the whole inverse fits comfortably in HBM (and mostly in L2), and z = A0^{-1} r for all PCE
// modes of a subdomain is one dense product Z[n x P] = Ainv[n x n] R[n x P].  It runs on the 5th-
// generation tensor cores: Ainv is stored once in BF16 (rows padded to Kp, a multiple of 128); R is
// split into two BF16 terms R = R_hi + R_lo (about 17 significant bits together) so that the product
// is a fixed linear operator up to that precision; both products accumulate in FP32 in tensor memory.
//
// Per CTA: one 128-row tile of one right-hand side.  A warp-specialised pipeline streams 64-column
// chunks of the Ainv tile by TMA (128-byte swizzle) and the matching chunks of the pre-packed R image
// by bulk copy into NST shared-memory stages guarded by mbarriers; one thread issues
// tcgen05.mma (M = 128, N = NB, K = 16) into a TMEM accumulator and frees each stage with
// tcgen05.commit; four warps read the accumulator back with tcgen05.ld.  Every wait is bounded (1 s)
// and reports through an error word instead of hanging.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace sgk {

constexpr int MMA_M = 128;                    // rows per CTA tile (TMEM lanes)
constexpr int MMA_KC = 64;                    // K elements per chunk: one 128-byte swizzle row of BF16
constexpr int MMA_ABYTES = MMA_M * MMA_KC * 2;  // 16 KB of A per stage
constexpr int MMA_NST = 6;                    // pipeline stages
constexpr unsigned long long MMA_WAIT_NS = 1000000000ull;  // bound of every wait

// NB: PCE modes padded to 16 or 32; TERMS: BF16 terms of the right-hand side (2: r = hi + lo, about
// 17 significant bits; 3: hi + mid + lo, about 25).  The B operand of one chunk is the TERMS x NB
// rows [term 0; term 1; ...], so one MMA of N = TERMS x NB per K step covers all terms (the
// epilogue adds the column blocks).  CPS: 64-column chunks per pipeline stage.
template <int NB, int TERMS = 2, int NST = MMA_NST, int CPS = 1>
struct MmaShape {
  static constexpr int BBYTES = NB * 128;                      // one term of one chunk (NB rows)
  static constexpr int BCHUNK = TERMS * BBYTES;                // all terms of one chunk
  static constexpr int STAGE = CPS * (MMA_ABYTES + BCHUNK);    // A chunks, then B chunks (x 1024)
  static constexpr int SMEM = NST * STAGE + 1024;              // + alignment slack
  static constexpr unsigned TX = STAGE;                        // bytes landing per stage
  static constexpr int N = TERMS * NB;                         // MMA N
  static constexpr unsigned TCOLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;  // TMEM alloc
};

// Programmatic dependent launch: let the next kernel of the stream start its prologue, and wait
// until every predecessor grid has completed and its memory is visible (no-ops without PDL).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// one bounded probe of the phase (the thread may be suspended for a short hardware-defined time)
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait until the phase of the given parity has completed; false after MMA_WAIT_NS
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (;;) {
    if (mbar_test(bar, parity)) return true;
    if (gtimer() - t0 > MMA_WAIT_NS) return false;
  }
}

// TMA: 2-D tile (x = inner element coordinate, y = row) into shared memory, completion on bar
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, unsigned bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
// bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned), completion on bar
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle layout (8-row atoms of
// 1024 bytes, atoms 1024-aligned, consecutive atoms 1024 bytes apart).
__device__ __forceinline__ unsigned long long sdesc_sw128(unsigned saddr) {
  unsigned long long d = (unsigned long long)((saddr & 0x3FFFFu) >> 4);  // start address / 16
  d |= (unsigned long long)(16 >> 4) << 16;                             // leading offset (unused here)
  d |= (unsigned long long)(1024 >> 4) << 32;                           // stride offset: next 8-row atom
  d |= 1ull << 46;                                                      // descriptor version
  d |= 2ull << 61;                                                      // 128-byte swizzle
  return d;
}
// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                          unsigned idesc, unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 lanes x NB columns of FP32 from TMEM (warp w reads lanes 32 (w % 4) ...)
template <int NB>
__device__ __forceinline__ void tmem_ld(unsigned taddr, float (&v)[NB]) {
  unsigned u[NB];
  if constexpr (NB == 32) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
          "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
          "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
        : "r"(taddr));
  } else {
    static_assert(NB == 16, "NB is 16 or 32");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < NB; ++i) v[i] = __uint_as_float(u[i]);
}

// Byte offset of element (row n, k) inside one K-major 128-byte-swizzled chunk (64 BF16 per row).
__host__ __device__ constexpr unsigned sw128_offset(int n, int k) {
  return (unsigned)((n >> 3) * 1024 + (n & 7) * 128 + ((((k >> 3) ^ (n & 7)) & 7) << 4) + (k & 7) * 2);
}

// ------------------------------------------------------------------------------------------
// Dense product core shared by the preconditioner kernel: accumulates
//   D[128 x 2NB] = sum_c A[y0 .. y0+127][64c .. 64c+63] * [Bhi_c; Blo_c]^T
// into TMEM (columns 0..NB-1: hi term, NB..2NB-1: lo term).  Roles: warp 0 allocates TMEM and its
// lane 0 produces (TMA for A, one bulk copy for the B chunks of a stage); warp 1 lane 0 issues the
// MMAs; on return (all threads) the accumulator is complete, or *err is set.  smem: 1024-aligned
// stage area; bars: 2 NST + 1 mbarriers.  NC must be a multiple of CPS.  Returns the TMEM base.
// ------------------------------------------------------------------------------------------
// Prologue (all threads): mbarriers and the TMEM accumulator (TERMS x NB columns, allocated as a
// power of two).  Needs no input data,
// so it may run before the wait on the predecessor grid.  Returns the TMEM base address.
template <int NB, int TERMS = 2, int NST = MMA_NST>
__device__ __forceinline__ unsigned mma_begin(unsigned long long* bars, unsigned* tmem_slot, volatile int* s_flags) {
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    const unsigned full0 = smem_u32(bars), empty0 = smem_u32(bars + NST), done = smem_u32(bars + 2 * NST);
    for (int s = 0; s < NST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    s_flags[0] = 0;  // stages issued by the producer
    s_flags[1] = 0;  // stages consumed by the MMA issuer
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(MmaShape<NB, TERMS, NST>::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *tmem_slot;
}

// Main loop (all threads; call after mma_begin): accumulates
//   D[128 x TERMS NB] = sum_c A[y0 .. y0+127][64c .. 64c+63] * [B_c,0; B_c,1; ...]^T
// into TMEM (column block t: term t).  Warp 0 lane 0 produces (TMA for A, one
// bulk copy for the B chunks of a stage), warp 1 lane 0 issues the MMAs; on return the accumulator
// is complete, or *err is set.  smem: 1024-aligned stage area.  NC must be a multiple of CPS.
template <int NB, int TERMS = 2, int NST = MMA_NST, int CPS = 1, bool MMA = true>
__device__ __forceinline__ void mma_run(const CUtensorMap* tmA, int y0, const unsigned char* __restrict__ bimg, int NC,
                                        unsigned char* smem, unsigned long long* bars, unsigned tmem,
                                        volatile int* s_flags, int* err) {
  using S = MmaShape<NB, TERMS, NST, CPS>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned full0 = smem_u32(bars), empty0 = smem_u32(bars + NST), done = smem_u32(bars + 2 * NST);
  const int NS = NC / CPS;  // stages to stream
  const unsigned sbase = smem_u32(smem);
  if (warp == 0 && lane == 0) {
    // producer
    for (int g = 0; g < NS; ++g) {
      const int s = g % NST, u = g / NST;
      if (g >= NST && !mbar_wait(empty0 + 8 * s, (unsigned)((u - 1) & 1))) {
        atomicExch(err, 17);
        break;
      }
      const unsigned st = sbase + (unsigned)(s * S::STAGE);
      mbar_expect_tx(full0 + 8 * s, S::TX);
#pragma unroll
      for (int j = 0; j < CPS; ++j) tma_load_2d(st + j * MMA_ABYTES, tmA, full0 + 8 * s, (g * CPS + j) * MMA_KC, y0);
      bulk_load(st + CPS * MMA_ABYTES, bimg + (size_t)g * CPS * S::BCHUNK, CPS * S::BCHUNK, full0 + 8 * s);
      s_flags[0] = g + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr unsigned idesc = idesc_bf16(MMA_M, S::N);
    for (int g = 0; g < NS; ++g) {
      const int s = g % NST, u = g / NST;
      if (!mbar_wait(full0 + 8 * s, (unsigned)(u & 1))) {
        atomicExch(err, 18);
        break;
      }
      tc_fence_after();
      const unsigned st = sbase + (unsigned)(s * S::STAGE);
      if (!MMA) {  // data movement only (timing of the pipeline without the products)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(empty0 + 8 * s) : "memory");
        s_flags[1] = g + 1;
        continue;
      }
#pragma unroll
      for (int j = 0; j < CPS; ++j) {
#pragma unroll
        for (int k = 0; k < MMA_KC / 16; ++k) {
          const unsigned long long a = sdesc_sw128(st + j * MMA_ABYTES + 32 * k);
          const unsigned long long bb = sdesc_sw128(st + CPS * MMA_ABYTES + j * S::BCHUNK + 32 * k);
          umma_bf16(tmem, a, bb, idesc, (g | j | k) != 0 ? 1u : 0u);
        }
      }
      umma_commit(empty0 + 8 * s);
      s_flags[1] = g + 1;
    }
    if (MMA) umma_commit(done);  // arrives when every MMA issued above has completed
    else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(done) : "memory");
  }
  __syncwarp();
  // everyone: wait for the accumulator
  if (!mbar_wait(done, 0u)) atomicExch(err, 19);
  __syncwarp();
  tc_fence_after();
}

// mma_begin + mma_run
template <int NB, int TERMS = 2, int NST = MMA_NST, int CPS = 1, bool MMA = true>
__device__ __forceinline__ unsigned mma_tile(const CUtensorMap* tmA, int y0, const unsigned char* __restrict__ bimg,
                                             int NC, unsigned char* smem, unsigned long long* bars,
                                             unsigned* tmem_slot, volatile int* s_flags, int* err) {
  const unsigned tmem = mma_begin<NB, TERMS, NST>(bars, tmem_slot, s_flags);
  mma_run<NB, TERMS, NST, CPS, MMA>(tmA, y0, bimg, NC, smem, bars, tmem, s_flags, err);
  return tmem;
}

// Row of the accumulator for this thread's lane (warp quarter wq owns lanes 32 wq ...): the sum of
// the TERMS column blocks.
template <int NB, int TERMS = 2>
__device__ __forceinline__ void mma_row(unsigned tmem, int wq, float (&v)[NB]) {
  const unsigned t = tmem + ((unsigned)(wq * 32) << 16);
  tmem_ld<NB>(t, v);
#pragma unroll
  for (int term = 1; term < TERMS; ++term) {
    float w[NB];
    tmem_ld<NB>(t + term * NB, w);
#pragma unroll
    for (int i = 0; i < NB; ++i) v[i] += w[i];
  }
}

// After the accumulator has been read: drain copies that were issued but never consumed (error
// path only), then free TMEM.  All threads call this.
template <int NB, int TERMS = 2, int NST = MMA_NST>
__device__ __forceinline__ void mma_tile_end(unsigned long long* bars, unsigned tmem, volatile int* s_flags) {
  tc_fence_before();
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    const unsigned full0 = smem_u32(bars);
    for (int g = s_flags[1]; g < s_flags[0]; ++g)
      (void)mbar_wait(full0 + 8 * (g % NST), (unsigned)((g / NST) & 1));
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(MmaShape<NB, TERMS, NST>::TCOLS)
                 : "memory");
  }
}

}  // namespace sgk
