// Split-precision tile tasks on the tcgen05 tensor cores.
//
// The tile tasks C_ij += A_ik B_kj (paper Sec. 2.1) are computed with
// error-free Ozaki-style slicing (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms
// 59, 2012), one power-of-two scale per tile:
//   e = smallest integer with max|x| < 2^e over the tile, rho_0 = x 2^-e,
//   N_t = rint(rho_{t-1} 2^(7t)), rho_t = rho_{t-1} - N_t 2^(-7t),  t = 1..s,
// so every slice is an integer of at most 8 bits, exact in bfloat16 and float16.
// For one tile pair the diagonal sums S_d = sum_{p+q=d} NA_p NB_q (d = 2..s+1)
// are integer matrices; with |S_d| <= 2^24 (inner blocks up to 512 elements for
// s = 6) the FP32 tensor-core accumulator holds them exactly. The epilogue forms
// T = sum_d S_d 2^(7(s+1-d)) exactly in int64 and adds T, shifted to its binary
// position e_A + e_B - 7(s+1), into an exact 128-bit integer accumulator per C
// element (no floating-point rounding and no FP64 instruction in the k loop; GB300's
// FP64 pipe is narrow). The sum is rounded once to FP64 at the end of the unit, so
// the result is fixed bit for bit, independent of schedule, unit order and k order.
//
// Kernels, in launch order:
//   1. split_exp_kernel   per stored tile: the exponent e (integer max reduction);
//      split_emax_kernel  per row / column block: the largest tile exponent;
//      split_class_kernel per (k block, row block / column block): the per-row /
//                         per-column offsets from it and the scale classes.
//   2. split_pack_kernel  per (128-row block, k block) of A and (k block, tn-column
//                         block) of B: the s slices, stored as bf16/fp16 in the
//                         exact shared-memory image the tensor core reads (K-major,
//                         64-byte swizzle, 32-element chunks), so the contraction
//                         kernel moves them with plain 1-D bulk copies.
//   3. split_mma_kernel   persistent, one CTA per SM, warp-specialised:
//                         warp 0 streams packed chunks into an S-stage shared-memory
//                         ring with cp.async.bulk (several k panels in flight -- the
//                         on-chip form of the paper's multiple-issue SUMMA
//                         iterations, Sec. 3.2); warps 1..3 share the issue of the
//                         tcgen05.mma slice products into double-buffered TMEM
//                         accumulators; warps 4..11 drain TMEM (zeroing it behind
//                         them), recombine in integer arithmetic and store
//                         C = alpha*fl(sum) + beta*C.
//   4. split_reduce_kernel only for a plan that cut k-lists (split k, Sec. 3.2, Fig. 2):
//                         adds each cut region's exact partial sums and stores C.
// A work unit is a 128-row x tn-column block of the global C index space over its
// k-list (or one piece of it); the CTA that owns it runs its inner blocks in ascending
// order. Float32 and complex elements use the same kernels: the exponent and pack
// kernels read the element type, the epilogue rounds and stores it.
// wait_selftest_kernel exercises the bounded waits and the abort protocol (diagnostics).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math_constants.h>

#include <nvtx3/nvToolsExt.h>

#include <climits>
#include <cstdint>
#include <type_traits>

#include "bsmm_internal.h"

namespace bsmm {

namespace {

constexpr int64_t kWaitNs = 4000000000LL;  // bounded waits: 4 s, then error + abort
constexpr int kEpiThreads = kSplitEpiWarps * 32;
// MMA issue: one thread issues tcgen05.mma instructions about one per 100 cycles, whatever
// their N, so the slice products of a step are spread over kMmaWarps issuing warps.
constexpr int kMmaWarps = 3;
constexpr int kEpiWarp0 = 1 + kMmaWarps;                 // first epilogue warp (warpgroups 1 and 2)
constexpr int kStoreWarps = 4;                           // C store warps (warpgroup 3), when present
constexpr int kStoreWarp0 = kEpiWarp0 + kSplitEpiWarps;  // first store warp
// Two forms of the contraction kernel: without store warps (the epilogue warps store each
// unit's C themselves) and with them (the C store of a unit runs while the epilogue drains
// the next one; it pays off when units are short).
template <bool SW>
constexpr int threads_of() {
  return 32 * (kStoreWarp0 + (SW ? kStoreWarps : 0));
}
// Register split with setmaxnreg (form with store warps): the CTA is launched with
// kThreadsSW x kRegsLaunch registers (the whole register file); the producer and MMA warps
// (warpgroup 0) and the store warps (warpgroup 3) give registers back and the epilogue warps
// take them. The shares add up to the launch's total exactly, so every setmaxnreg.inc is
// satisfiable.
constexpr int kThreadsSW = threads_of<true>();  // 512
constexpr int kRegsLaunch = 65536 / kThreadsSW;  // 128
constexpr int kRegsCtl = 80, kRegsEpi = 168, kRegsStore = 96;
static_assert(kEpiWarp0 % 4 == 0 && kStoreWarp0 % 4 == 0, "roles start on warpgroup boundaries");
static_assert(4 * 32 * kRegsCtl + kSplitEpiWarps * 32 * kRegsEpi + kStoreWarps * 32 * kRegsStore ==
                  kThreadsSW * kRegsLaunch,
              "the warpgroups' register shares must add up to the launch's registers");
constexpr uint32_t kTmemCols = 512;
constexpr int kAChunk = kSplitBM * kSplitKC * 2;  // bytes of one slice of a 128x32 A chunk

__device__ __forceinline__ int64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (int64_t)t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Single-thread bounded wait. False on timeout (sets the error word and the abort
// flag) or when another role aborted.
__device__ bool wait1(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int32_t* err,
                      int64_t limit = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const int64_t t0 = gtimer();
  for (uint32_t spin = 1;; spin++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if ((spin & 63) == 0 && gtimer() - t0 > limit) {
      *abort_flag = 1;
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
}

constexpr uint32_t kGroupPollNs = 128;  // the epilogue's sleep between polls for the next group

// Warp-uniform bounded wait (every lane polls; the decision is taken by the warp). A warp
// whose wait is not on the critical path passes sleep_ns > 0: it sleeps between polls,
// leaving the issue slots to the warps that are.
__device__ bool wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int32_t* err,
                          int64_t limit = kWaitNs, uint32_t sleep_ns = 0) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  const int64_t t0 = gtimer();
  for (uint32_t spin = 1;; spin++) {
    if (sleep_ns) __nanosleep(sleep_ns);
    const bool ok = mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, ok)) return true;
    int stop = *abort_flag;
    if ((spin & 63) == 0 && gtimer() - t0 > limit) stop = 2;
    if (__any_sync(0xffffffffu, stop != 0)) {
      if (stop == 2 && (threadIdx.x & 31) == 0) {
        *abort_flag = 1;
        atomicOr(err, kErrTimeout);
      }
      __syncwarp();
      return false;
    }
  }
}

// ---------------------------------------------------------------- bulk copy
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}


// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (bf16 or fp16 in, fp32 accumulate)
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_zero4(uint32_t taddr) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%1,%1,%1};" ::"r"(taddr), "r"(0u) : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_zero8(uint32_t taddr) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr), "r"(0u) : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row groups of
// 64-byte rows (stride between 8-row groups = 512 bytes).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address (16-byte units)
  d |= (uint64_t)0 << 16;                   // leading byte offset: unused (one swizzle atom along K)
  d |= (uint64_t)(512u >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;                   // descriptor version for tcgen05
  d |= (uint64_t)4 << 61;                   // layout: 64-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D fp32, A and B bf16 (or fp16), both K-major.
__device__ __forceinline__ uint32_t idesc_f16(int M, int N, bool fp16) {
  const uint32_t fmt = fp16 ? 0u : 1u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) inside one 64-byte-swizzled chunk slice (rows of 32 elements)
__device__ __forceinline__ uint32_t swz64(int row, int k) {
  const int ch = k >> 3;
  return (uint32_t)(row * 64 + ((ch ^ ((row >> 1) & 3)) << 4) + ((k & 7) << 1));
}


// ---------------------------------------------------------------- kernel 1: exponents
// The caller's offset of stored tile t of A (isA) or B; transposed storage indexes the
// tables (k,i) / (j,k) (the maximum does not depend on the element order in a tile).
__device__ __forceinline__ void tile_geometry(const SplitArgs& a, bool isA, int t, int& rows, int& cols,
                                              int64_t& off) {
  if (isA) {
    const int i = t / a.K, k = t % a.K;
    rows = a.r[i];
    cols = a.q[k];
    off = a.transa ? a.a_off[(int64_t)k * a.M + i] : a.a_off[t];
  } else {
    const int k = t / a.N, j = t % a.N;
    rows = a.q[k];
    cols = a.c[j];
    off = a.transb ? a.b_off[(int64_t)j * a.K + k] : a.b_off[t];
  }
}

// Magnitude of a double as its bit pattern without the sign: for non-negative doubles the
// bit patterns order like the values, so maxima are taken with integer instructions
// (GB300's FP64 pipe is narrow). A pattern at or above kInfBits is an infinity or a NaN.
constexpr unsigned long long kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;
__device__ __forceinline__ unsigned long long mag_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & kAbsMask;
}

// Smallest e with m < 2^e for the magnitude bits m of a finite nonzero double
// (m = f 2^e with f in [0.5, 1), as frexp gives; subnormals included).
__device__ __forceinline__ int exponent_above(unsigned long long m) {
  const int be = (int)(m >> 52);
  if (be) return be - 1022;
  return -1022 - (__clzll((long long)m) - 12);  // subnormal: leading one at bit 63 - clz
}

// The same for the magnitude bits of a finite nonzero float (subnormals included).
constexpr uint32_t kInfBits32 = 0x7F800000u;
__device__ __forceinline__ int exponent_above32(uint32_t m) {
  const int be = (int)(m >> 23);
  if (be) return be - 126;
  return -126 - (__clz((int)m) - 8);  // subnormal: leading one at bit 31 - clz
}

__global__ void __launch_bounds__(256) split_exp_kernel(SplitArgs a) {
  const int b = blockIdx.x;
  const bool isA = b < a.n_a_tiles;
  const int t = isA ? a.a_tiles[b] : a.b_tiles[b - a.n_a_tiles];
  int rows, cols;
  int64_t off;
  tile_geometry(a, isA, t, rows, cols, off);
  // complex elements: the tile's doubles (both parts) at twice its complex offset; an A
  // tile holds r x q' doubles (q' = 2q), a B tile q' x c' / 2 (c' = 2c)
  const double* x = (isA ? a.A : a.B) + (off < 0 ? 0 : (a.cplx ? 2 * off : off));
  const int64_t n = (int64_t)rows * cols / (a.cplx && !isA ? 2 : 1);
  // the largest magnitude as bits: at or above kInfBits when a NaN or infinity is there
  unsigned long long mx = 0;
  if (a.f32 && off >= 0) {
    // float32 tiles start 16-byte aligned (offsets multiples of 4): four floats per load;
    // the float maximum's bits are turned into a double's (both order like the values)
    const float* xf = (isA ? a.Af : a.Bf) + off;
    uint32_t m32 = 0;
    if (off & 3) {
      if (threadIdx.x == 0) atomicOr(a.err, kErrBadOffset);
    } else {
      const uint4* x4 = reinterpret_cast<const uint4*>(xf);
      const int64_t n4 = n >> 2;
      const int64_t bd = blockDim.x;
      for (int64_t e = threadIdx.x; e < n4; e += 4 * bd) {  // four loads in flight
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = e + u * bd < n4 ? __ldg(x4 + e + u * bd) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < 4; u++)
          m32 = max(m32, max(max(v[u].x & 0x7FFFFFFFu, v[u].y & 0x7FFFFFFFu),
                             max(v[u].z & 0x7FFFFFFFu, v[u].w & 0x7FFFFFFFu)));
      }
      for (int64_t e = (n4 << 2) + threadIdx.x; e < n; e += blockDim.x)
        m32 = max(m32, __float_as_uint(__ldg(xf + e)) & 0x7FFFFFFFu);
    }
    // as a double's magnitude bits: equal exponent of the top bit, so exponent_above agrees
    if (m32 >= kInfBits32)
      mx = kInfBits;
    else if (m32)
      mx = (unsigned long long)(exponent_above32(m32) + 1022) << 52;
  } else if (off >= 0) {
    // tiles start 16-byte aligned (even offsets): pairs of doubles, four pairs in flight
    const longlong2* x2 = reinterpret_cast<const longlong2*>(x);
    const int64_t n2 = n >> 1;
    const int64_t bd = blockDim.x;
    for (int64_t e = threadIdx.x; e < n2; e += 4 * bd) {
      longlong2 v[4];
#pragma unroll
      for (int u = 0; u < 4; u++) v[u] = e + u * bd < n2 ? __ldg(x2 + e + u * bd) : make_longlong2(0, 0);
#pragma unroll
      for (int u = 0; u < 4; u++) {
        mx = max(mx, (unsigned long long)v[u].x & kAbsMask);
        mx = max(mx, (unsigned long long)v[u].y & kAbsMask);
      }
    }
    if ((n & 1) && threadIdx.x == 0) mx = max(mx, mag_bits(__ldg(x + n - 1)));
  }
  __shared__ unsigned long long red[8];
  for (int o = 16; o; o >>= 1) mx = max(mx, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = max(m, red[w]);
    int e = 0;
    if (off < 0 || m >= kInfBits) {
      atomicOr(a.err, off < 0 ? kErrBadOffset : kErrNonFinite);
    } else if (m > 0) {
      e = exponent_above(m);  // smallest e with max|x| < 2^e
    }
    if (isA)
      a.eA[t] = e;
    else
      a.eB[t] = e;
  }
}

// Row/column scaling: one exponent per row of each stored A tile and per column of each
// stored B tile (kZeroLine for an all-zero line); a non-finite value is reported by
// split_exp_kernel. One block per tile, one thread per line.
__global__ void __launch_bounds__(256) split_exp_lines_kernel(SplitArgs a) {
  const int b = blockIdx.x;
  const bool isA = b < a.n_a_tiles;
  const int t = isA ? a.a_tiles[b] : a.b_tiles[b - a.n_a_tiles];
  int rows, cols;
  int64_t off;
  tile_geometry(a, isA, t, rows, cols, off);
  if (off < 0) return;
  const double* x = (isA ? a.A : a.B) + off;
  const int i_or_k = isA ? t / a.K : t / a.N;
  const int k_or_j = isA ? t % a.K : t % a.N;
  const int nl = isA ? rows : cols;   // lines
  const int len = isA ? cols : rows;  // elements per line
  const bool tr = isA ? a.transa != 0 : a.transb != 0;
  // element u of line l: A row l is (l, u), B column l is (u, l); stored transposed or not
  const int64_t lstep = isA ? (tr ? 1 : cols) : (tr ? rows : 1);
  const int64_t ustep = isA ? (tr ? rows : 1) : (tr ? 1 : cols);
  if (a.cplx) {
    // complex elements: the plan's inner and column tilings count both parts, so an A tile
    // is rows x (2 qc) and a B tile (2 qc) x (2 cc) of the real product; a line's exponent
    // is that of the complex row (column) over both parts, and the B column cl and its
    // partner cl + cc (the same complex column's other part) share it
    const int qc = (isA ? cols : rows) >> 1;
    const int nlc = isA ? rows : cols >> 1;  // complex lines
    const int64_t cl_step = isA ? (tr ? 1 : qc) : (tr ? qc : 1);           // between lines
    const int64_t cu_step = isA ? (tr ? rows : 1) : (tr ? 1 : (cols >> 1));  // along a line
    const double* xc = (isA ? a.A : a.B) + 2 * off;
    for (int l = threadIdx.x; l < nlc; l += blockDim.x) {
      unsigned long long lm = 0;
      const double* line = xc + 2 * (l * cl_step);
      for (int u = 0; u < qc; u++) {
        lm = max(lm, mag_bits(__ldg(line + 2 * u * cu_step)));
        lm = max(lm, mag_bits(__ldg(line + 2 * u * cu_step + 1)));
      }
      const int e = (lm > 0 && lm < kInfBits) ? exponent_above(lm) : kZeroLine;
      if (isA) {
        a.eArow[(int64_t)k_or_j * a.Mtot + a.ro[i_or_k] + l] = e;
      } else {
        a.eBcol[(int64_t)i_or_k * a.Ntot + a.co[k_or_j] + l] = e;
        a.eBcol[(int64_t)i_or_k * a.Ntot + a.co[k_or_j] + nlc + l] = e;
      }
    }
    return;
  }
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    int e = kZeroLine;
    if (a.f32) {
      uint32_t lm = 0;
      const float* line = (isA ? a.Af : a.Bf) + off + l * lstep;
      for (int u = 0; u < len; u++) lm = max(lm, __float_as_uint(__ldg(line + u * ustep)) & 0x7FFFFFFFu);
      if (lm > 0 && lm < kInfBits32) e = exponent_above32(lm);
    } else {
      unsigned long long lm = 0;
      const double* line = x + l * lstep;
      for (int u = 0; u < len; u++) lm = max(lm, mag_bits(__ldg(line + u * ustep)));
      if (lm > 0 && lm < kInfBits) e = exponent_above(lm);
    }
    if (isA)
      a.eArow[(int64_t)k_or_j * a.Mtot + a.ro[i_or_k] + l] = e;
    else
      a.eBcol[(int64_t)i_or_k * a.Ntot + a.co[k_or_j] + l] = e;
  }
}

// ---------------------------------------------------------------- kernel 1b: largest exponents
// Per row block i: Emax_A(i) = the largest exponent of its stored A tiles (0 when none);
// the same per column block for B. One block per row or column block, its threads
// spread over the K inner blocks. The contraction adds each tile pair's exact integer at
// the binary position GUARD + rowexp + colexp of a 128-bit accumulator whose unit is
// 2^(Emax_A(i) + Emax_B(j) - 7(s+1) - GUARD); the class kernel writes rowexp and colexp.
__global__ void __launch_bounds__(256) split_emax_kernel(SplitArgs a) {
  const bool isA = (int)blockIdx.x < a.M;
  const int t = isA ? blockIdx.x : blockIdx.x - a.M;
  int em = INT_MIN;
  if (isA ? a.r[t] > 0 : a.c[t] > 0) {
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
      if (a.q[k] <= 0) continue;
      if (isA) {
        if (a.am[(int64_t)t * a.K + k]) em = max(em, a.eA[(int64_t)t * a.K + k]);
      } else {
        if (a.bm[(int64_t)k * a.N + t]) em = max(em, a.eB[(int64_t)k * a.N + t]);
      }
    }
  }
  __shared__ int red[8];
  for (int o = 16; o; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = em;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) em = max(em, red[w]);
    if (em == INT_MIN) em = 0;
    if (isA)
      a.eAmax[t] = em;
    else
      a.eBmax[t] = em;
  }
}

// ---------------------------------------------------------------- kernel 1b': line scales
// Row/column scaling: one thread per row m of A (per column n of B): Emax = the largest
// exponent of that line over its stored tiles (all-zero lines excluded; 0 when none), and
// rowexp[k][m] = e(m, k) - Emax (colexp likewise), 0 where there is no tile or the line is
// zero there (its slices are zero).
__global__ void __launch_bounds__(256) split_scale_lines_kernel(SplitArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < a.Mtot) {
    const int64_t m = t;
    const int i = a.row_tile[m];
    int em = INT_MIN;
    for (int k = 0; k < a.K; k++) {
      const int e = a.eArow[(int64_t)k * a.Mtot + m];
      if (a.am[(int64_t)i * a.K + k] && a.q[k] > 0 && e != kZeroLine) em = max(em, e);
    }
    if (em == INT_MIN) em = 0;
    a.eAmaxr[m] = em;
    for (int k = 0; k < a.K; k++) {
      const int e = a.eArow[(int64_t)k * a.Mtot + m];
      const bool pres = a.am[(int64_t)i * a.K + k] && a.q[k] > 0 && e != kZeroLine;
      a.rowexp[(int64_t)k * a.Mtot + m] = (int16_t)(pres ? e - em : 0);
    }
  } else if (t < a.Mtot + a.Ntot) {
    const int64_t n = t - a.Mtot;
    const int j = a.col_tile[n];
    int em = INT_MIN;
    for (int k = 0; k < a.K; k++) {
      const int e = a.eBcol[(int64_t)k * a.Ntot + n];
      if (a.bm[(int64_t)k * a.N + j] && a.q[k] > 0 && e != kZeroLine) em = max(em, e);
    }
    if (em == INT_MIN) em = 0;
    a.eBmaxc[n] = em;
    for (int k = 0; k < a.K; k++) {
      const int e = a.eBcol[(int64_t)k * a.Ntot + n];
      const bool pres = a.bm[(int64_t)k * a.N + j] && a.q[k] > 0 && e != kZeroLine;
      a.colexp[(int64_t)k * a.colexp_ld + n] = (int16_t)(pres ? e - em : 0);
    }
  }
}

// ---------------------------------------------------------------- kernel 1c: offsets and scale classes
// One warp per (k block, row block) and per (k block, column block). With one scale per
// tile it first writes the offsets of its rows, rowexp[k][m] = e_A(i,k) - Emax_A(i) for a
// stored tile (0 for an absent one), or of its columns (colexp); with one scale per row
// and column the line kernel wrote them.
// Then the scale class. The products of k block k land at element (m, n) at the binary
// position e_A(m,k) + e_B(n,k) - Emax_A(m) - Emax_B(n) (exponents of the row's and the
// column's tile, or line, at k, and their maxima). When the rows of the row block that
// have a tile at k share one exponent e_A(k) (the columns likewise e_B(k)), that position
// is e_A(k) + e_B(k) plus a part that depends only on the row and the column, not on k:
//   urow[k][rb] = e_A(k) - maxE_A(rb),  rowadj[m] = maxE_A(rb) - Emax_A(m) >= 0
// (maxE_A(rb) = the largest Emax_A over the block's rows; the same for columns), so two
// k blocks whose urow + ucol agree may share one TMEM accumulation, drained at
// guard + urow + ucol + rowadj[m] + coladj[n]. kNonUniform marks a k block whose rows (or
// columns) at k have different exponents; rows without a tile (or all-zero lines) there
// take no part.
__global__ void __launch_bounds__(256) split_class_kernel(SplitArgs a) {
  // one warp per (k block, row block) and per (k block, column block); lanes over the lines
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nr = (int64_t)a.K * a.RB, nc = (int64_t)a.K * a.CB;
  int lo = INT_MAX, hi = INT_MIN, emx = INT_MIN;
  if (wid < nr) {
    const int k = (int)(wid / a.RB), rb = (int)(wid % a.RB);
    const int64_t m0 = (int64_t)rb * kSplitBM;
    const int64_t m1 = m0 + kSplitBM < a.Mtot ? m0 + kSplitBM : a.Mtot;
    for (int64_t m = m0 + lane; m < m1; m += 32) {
      const int i = a.row_tile[m];
      const int emax_m = a.rowscale ? a.eAmaxr[m] : a.eAmax[i];
      emx = max(emx, emax_m);
      bool pres = a.q[k] > 0 && a.am[(int64_t)i * a.K + k];
      int eabs = 0;
      if (!a.rowscale) {
        eabs = pres ? a.eA[(int64_t)i * a.K + k] : 0;
        a.rowexp[(int64_t)k * a.Mtot + m] = (int16_t)(pres ? eabs - emax_m : 0);
      } else if (pres) {
        eabs = a.eArow[(int64_t)k * a.Mtot + m];
        pres = eabs != kZeroLine;
      }
      if (pres) {
        lo = min(lo, eabs);
        hi = max(hi, eabs);
      }
    }
    for (int o = 16; o; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      emx = max(emx, __shfl_xor_sync(0xffffffffu, emx, o));
    }
    if (k == 0)
      for (int64_t m = m0 + lane; m < m1; m += 32) {
        const int e = a.rowscale ? a.eAmaxr[m] : a.eAmax[a.row_tile[m]];
        a.emaxr[m] = e;
        if (a.urow) a.rowadj[m] = (int16_t)(emx - e);
      }
    if (a.urow && lane == 0) a.urow[wid] = (int16_t)(lo > hi ? 0 : lo == hi ? lo - emx : kNonUniform);
  } else if (wid < nr + nc) {
    const int64_t u = wid - nr;
    const int k = (int)(u / a.CB), cb = (int)(u % a.CB);
    const int64_t n0 = (int64_t)cb * a.tn;
    const int64_t n1 = n0 + a.tn < a.Ntot ? n0 + a.tn : a.Ntot;
    for (int64_t n = n0 + lane; n < n1; n += 32) {
      const int j = a.col_tile[n];
      const int emax_n = a.rowscale ? a.eBmaxc[n] : a.eBmax[j];
      emx = max(emx, emax_n);
      bool pres = a.q[k] > 0 && a.bm[(int64_t)k * a.N + j];
      int eabs = 0;
      if (!a.rowscale) {
        eabs = pres ? a.eB[(int64_t)k * a.N + j] : 0;
        a.colexp[(int64_t)k * a.colexp_ld + n] = (int16_t)(pres ? eabs - emax_n : 0);
      } else if (pres) {
        eabs = a.eBcol[(int64_t)k * a.Ntot + n];
        pres = eabs != kZeroLine;
      }
      if (pres) {
        lo = min(lo, eabs);
        hi = max(hi, eabs);
      }
    }
    for (int o = 16; o; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      emx = max(emx, __shfl_xor_sync(0xffffffffu, emx, o));
    }
    if (k == 0)
      for (int64_t n = n0 + lane; n < n1; n += 32) {
        const int e = a.rowscale ? a.eBmaxc[n] : a.eBmax[a.col_tile[n]];
        a.emaxc[n] = e;
        if (a.ucol) a.coladj[n] = (int16_t)(emx - e);
      }
    if (a.ucol && lane == 0) a.ucol[u] = (int16_t)(lo > hi ? 0 : lo == hi ? lo - emx : kNonUniform);
  }
}

// ---------------------------------------------------------------- kernel 2: slices
// Slice 8 consecutive inner elements (one 16-byte chunk of a swizzled row) of one
// packed row and store the s chunks.
// The slicing recurrence N_t = rint(rho_{t-1} 2^(7t)), rho_t = rho_{t-1} - N_t 2^(-7t)
// telescopes: with Z_t = sum_{u<=t} N_u 2^(7(t-u)) one has Z_t = rint(x 2^(7t-e)) (the
// subtracted 128 Z_{t-1} is even, so round-half-even commutes with it), hence
// N_t = Z_t - 128 Z_{t-1}. Each Z_t is computed exactly from the mantissa with integer
// shifts and a round-half-even step; no floating-point operation is involved.
// All Z_t of one element come from one window of its significand: x 2^-e = +-m 2^ex with
// an integer m < 2^53; at the finest level t = S the window is W = floor(m 2^-k),
// k = -(ex + 7S), with the round bit R (bit k-1 of m) and the sticky flag (any lower bit
// set); level t < S drops a = 7(S-t) more bits of W, rounding with bit a-1 of W and the
// bits below it (the finest level's fraction included). The window's shifts are
// compile-time constants. Only the low 32 bits of Z_t are kept: N_t is small, so
// Z_t - 128 Z_(t-1) is exact in 32-bit wrap-around arithmetic.
struct SliceWindow {
  unsigned long long W;  // floor(m 2^-k)
  bool R, T, F;          // round bit and sticky bits at the finest level; F = any bit below W
  __device__ __forceinline__ void init(unsigned long long m, int k) {
    if (k <= 0) {  // exact (a subnormal tile's elements, or a non-finite input already reported)
      W = -k >= 63 ? 0ull : m << -k;
      R = T = F = false;
    } else if (k >= 64) {
      W = 0ull;
      R = false;
      T = F = m != 0ull;
    } else {
      W = m >> k;
      R = (m >> (k - 1)) & 1ull;
      T = (m & ((1ull << (k - 1)) - 1ull)) != 0ull;
      F = R || T;
    }
  }
  // low 32 bits of Z at the level a bits coarser than the finest. For A > 0 the rounding
  // is one addition: with h = 2^(A-1) and b = (bit A of W) | F, W + h - 1 + b carries into
  // bit A exactly when the dropped part exceeds h, or equals h with an odd quotient or a
  // nonzero fraction below W (round half to even).
  template <int A>
  __device__ __forceinline__ uint32_t z() const {
    if constexpr (A == 0) {
      return (uint32_t)W + ((R && (T || (W & 1ull))) ? 1u : 0u);
    } else {
      const unsigned long long b = ((W >> A) & 1ull) | (F ? 1ull : 0ull);
      return (uint32_t)((W + ((1ull << (A - 1)) - 1ull) + b) >> A);
    }
  }
};

template <typename T>
__device__ __forceinline__ uint16_t small_int_bits(int n) {  // |n| <= 256, exact in bf16/fp16
  const float f = __int_as_float(0x4B400000 + n) - 12582912.0f;  // exact for |n| < 2^22
  if constexpr (std::is_same<T, __nv_bfloat16>::value) {
    return (uint16_t)(__float_as_uint(f) >> 16);  // <= 8 significant bits: truncation is exact
  } else {
    return __half_as_ushort(__float2half_rn(f));
  }
}

template <typename T, int S, int t>
__device__ __forceinline__ void slice_level(const SliceWindow (&w)[8], const bool (&neg)[8], uint32_t (&zp)[8],
                                            uint8_t* base, int slice_stride, uint32_t soff) {
  if constexpr (t <= S) {
    uint16_t h[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      uint32_t zt = w[u].template z<kSplitBeta * (S - t)>();
      if (neg[u]) zt = 0u - zt;
      h[u] = small_int_bits<T>((int)(zt - (zp[u] << kSplitBeta)));
      zp[u] = zt;
    }
    *reinterpret_cast<uint4*>(base + (size_t)(t - 1) * slice_stride + soff) = *reinterpret_cast<uint4*>(h);
    slice_level<T, S, t + 1>(w, neg, zp, base, slice_stride, soff);
  }
}

// x 2^-e = +-m 2^ex with an integer significand m, from the bits of a double or a float
__device__ __forceinline__ void decode(double x, int e, bool& neg, unsigned long long& m, int& ex) {
  const long long b = __double_as_longlong(x);
  neg = b < 0;
  const int be = (int)((b >> 52) & 0x7FF);
  const unsigned long long frac = (unsigned long long)b & ((1ull << 52) - 1ull);
  m = be ? (frac | (1ull << 52)) : frac;
  ex = (be ? be : 1) - 1075 - e;
}
__device__ __forceinline__ void decode(float x, int e, bool& neg, unsigned long long& m, int& ex) {
  const uint32_t b = __float_as_uint(x);
  neg = (b >> 31) != 0;
  const int be = (int)((b >> 23) & 0xFF);
  const uint32_t frac = b & 0x7FFFFFu;
  m = be ? (frac | 0x800000u) : frac;
  ex = (be ? be : 1) - 150 - e;
}

template <typename T, int S, typename E>
__device__ __forceinline__ void slice_store8(const E (&x)[8], int e, uint8_t* base, int slice_stride, uint32_t soff) {
  SliceWindow w[8];
  bool neg[8];
  uint32_t zp[8];
#pragma unroll
  for (int u = 0; u < 8; u++) {
    unsigned long long m;
    int ex;
    decode(x[u], e, neg[u], m, ex);
    w[u].init(m, -(ex + kSplitBeta * S));
    zp[u] = 0u;
  }
  slice_level<T, S, 1>(w, neg, zp, base, slice_stride, soff);
}

// Complex elements (CPLX): the real product's A tile is [Ar, -Ai] (inner index kk' < q
// takes the real part of column kk', kk' >= q the negated imaginary part of column kk' - q)
// and its B tile [[Br, Bi], [Bi, -Br]] (row half and column half pick the part and the
// sign); q and c below are the doubled sizes, the stored complex tile is q/2 and c/2 wide.
__device__ __forceinline__ double neg_if(double v, bool n) {  // sign flip as bits (no FP64 op)
  return n ? __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull) : v;
}

template <typename T, int S, typename E, bool CPLX = false>
__global__ void __launch_bounds__(256) split_pack_kernel(SplitArgs a) {
  constexpr int s = S;
  const E* Ae = reinterpret_cast<const E*>(std::is_same<E, float>::value ? (const void*)a.Af : (const void*)a.A);
  const E* Be = reinterpret_cast<const E*>(std::is_same<E, float>::value ? (const void*)a.Bf : (const void*)a.B);
  if ((int)blockIdx.x < a.n_a_blocks) {
    // A block (rb, kt): chunks of 128 rows x 32 inner elements
    const int blk = a.a_blocks[blockIdx.x];
    const int rb = blk / a.K, kt = blk % a.K;
    const int q = a.q[kt];
    const int nkc = (q + kSplitKC - 1) / kSplitKC;
    uint8_t* out = a.apk + a.apk_off[blk];
    for (int item = threadIdx.x; item < nkc * kSplitBM * 4; item += blockDim.x) {
      const int ch = item & 3, rr = (item >> 2) % kSplitBM, kc = (item >> 2) / kSplitBM;
      const int64_t m = (int64_t)rb * kSplitBM + rr;
      E x[8];
      int e = 0;
      bool present = false;
      int64_t off = -1;
      int i = 0;
      if (m < a.Mtot) {
        i = a.row_tile[m];
        present = a.am[(int64_t)i * a.K + kt] != 0;
        off = a.transa ? a.a_off[(int64_t)kt * a.M + i] : a.a_off[(int64_t)i * a.K + kt];
        if (present && off < 0) {
          atomicOr(a.err, kErrBadOffset);
          present = false;
        }
        e = a.rowscale ? a.eArow[(int64_t)kt * a.Mtot + m] : a.eA[(int64_t)i * a.K + kt];
      }
      const int64_t lr = m - (m < a.Mtot ? a.ro[i] : 0);
      // element (lr, k) of A_ik at line + k * step, stored transposed or not
      const int64_t step = a.transa ? (m < a.Mtot ? a.r[i] : 0) : 1;
      const int k0 = kc * kSplitKC + ch * 8;
      if constexpr (CPLX) {
        // complex element (lr, kc) of the tile at row + 2 kc cstep (cstep = 1, or the tile's
        // row count when stored transposed); part 0 real, 1 imaginary
        const int qc = q >> 1;
        const int64_t cstep = a.transa ? step : 1;
        const double* row = a.A + 2 * (off + (a.transa ? lr : lr * qc));
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const int kk = k0 + u, part = kk >= qc;
          x[u] = (present && kk < q) ? neg_if(__ldg(row + 2 * (kk - part * qc) * cstep + part), part) : 0.0;
        }
      } else {
        const E* line = Ae + off + (a.transa ? lr : lr * q);
#pragma unroll
        for (int u = 0; u < 8; u++) x[u] = (present && k0 + u < q) ? __ldg(line + (k0 + u) * step) : E(0);
      }
      slice_store8<T, S>(x, e, out + (size_t)kc * s * kAChunk, kAChunk, swz64(rr, ch * 8));
    }
  } else {
    // B block (kt, cb): chunks of tn rows (columns of B) x 32 inner elements, transposed
    const int blk = a.b_blocks[blockIdx.x - a.n_a_blocks];
    const int kt = blk / a.CB, cb = blk % a.CB;
    const int q = a.q[kt];
    const int tn = a.tn;
    const int nkc = (q + kSplitKC - 1) / kSplitKC;
    const int bchunk = tn * kSplitKC * 2;
    uint8_t* out = a.bpk + a.bpk_off[blk];
    for (int item = threadIdx.x; item < nkc * tn * 4; item += blockDim.x) {
      const int nn = item % tn, ch = (item / tn) & 3, kc = (item / tn) >> 2;
      const int64_t n = (int64_t)cb * tn + nn;
      E x[8];
      int e = 0;
      bool present = false;
      int64_t off = -1;
      int j = 0, cj = 0;
      if (n < a.Ntot) {
        j = a.col_tile[n];
        cj = a.c[j];
        present = a.bm[(int64_t)kt * a.N + j] != 0;
        off = a.transb ? a.b_off[(int64_t)j * a.K + kt] : a.b_off[(int64_t)kt * a.N + j];
        if (present && off < 0) {
          atomicOr(a.err, kErrBadOffset);
          present = false;
        }
        e = a.rowscale ? a.eBcol[(int64_t)kt * a.Ntot + n] : a.eB[(int64_t)kt * a.N + j];
      }
      const int64_t lc = n - (n < a.Ntot ? a.co[j] : 0);
      // element (k, lc) of B_kj at line + k * step, stored transposed or not
      const int64_t step = a.transb ? 1 : cj;
      const int k0 = kc * kSplitKC + ch * 8;
      if constexpr (CPLX) {
        // complex element (kc, c) of the tile at col + 2 kc kstep: kstep = the tile's complex
        // column count, or 1 when stored transposed (then column c starts c * qc in)
        const int qc = q >> 1, cc = cj >> 1;
        const int cpart = lc >= cc;
        const int64_t kstep = a.transb ? 1 : cc;
        const double* col = a.B + 2 * (off + (lc - cpart * cc) * (a.transb ? qc : 1));
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const int kk = k0 + u, rpart = kk >= qc;
          x[u] = (present && kk < q)
                     ? neg_if(__ldg(col + 2 * (int64_t)(kk - rpart * qc) * kstep + (rpart ^ cpart)), rpart & cpart)
                     : 0.0;
        }
      } else {
        const E* line = Be + off + (a.transb ? lc * q : lc);
#pragma unroll
        for (int u = 0; u < 8; u++) x[u] = (present && k0 + u < q) ? __ldg(line + (k0 + u) * step) : E(0);
      }
      slice_store8<T, S>(x, e, out + (size_t)kc * s * bchunk, bchunk, swz64(nn, ch * 8));
    }
  }
}

// ---------------------------------------------------------------- exact accumulation
// w (four 32-bit words, two's complement) += T * 2^sh, with floor(T / 2^-sh) for sh < 0.
// |T| < 2^59 and sh <= kSplitGuard for every accumulation group (its depth keeps each FP32
// partial sum below 2^24); an absent tile pair has T = 0.
__device__ __forceinline__ void acc_add(uint32_t (&w)[4], long long T, int sh) {
  const int sl = min(max(sh, 0), 63);
  long long lo = T << sl;
  long long hi = sl ? (T >> (64 - sl)) : (T >> 63);
  if (sh < 0) {
    lo = T >> min(-sh, 63);
    hi = T >> 63;
  }
  asm("add.cc.u32 %0, %0, %4;\n\t"
      "addc.cc.u32 %1, %1, %5;\n\t"
      "addc.cc.u32 %2, %2, %6;\n\t"
      "addc.u32 %3, %3, %7;"
      : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3])
      : "r"((uint32_t)lo), "r"((uint32_t)((unsigned long long)lo >> 32)), "r"((uint32_t)hi),
        "r"((uint32_t)((unsigned long long)hi >> 32)));
}

// 64-bit window of a 128-bit magnitude shifted right by r (0 <= r < 128)
__device__ __forceinline__ unsigned long long shr128(unsigned long long hi, unsigned long long lo, int r) {
  if (r == 0) return lo;
  if (r < 64) return (lo >> r) | (hi << (64 - r));
  return hi >> (r - 64);
}

// |w| of the 128-bit two's-complement integer w rounded to P significant bits (ties to
// even): |w| ~ mant 2^r with mant in [2^(P-1), 2^P), in integer arithmetic. False for w = 0.
template <int P>
__device__ __forceinline__ bool acc_round(const uint32_t (&w)[4], bool& neg, unsigned long long& mant, int& r) {
  unsigned long long lo = ((unsigned long long)w[1] << 32) | w[0];
  unsigned long long hi = ((unsigned long long)w[3] << 32) | w[2];
  neg = (long long)hi < 0;
  if (neg) {
    lo = ~lo;
    hi = ~hi;
    lo += 1;
    if (lo == 0) hi += 1;
  }
  if (hi == 0 && lo == 0) return false;
  const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  r = msb - (P - 1);
  if (r <= 0) {
    mant = lo << (-r);  // exact
  } else {
    mant = shr128(hi, lo, r);
    const bool round = shr128(hi, lo, r - 1) & 1;
    bool sticky;
    if (r - 1 <= 64)
      sticky = (r - 1 == 64) ? lo != 0 : (lo & ((1ull << (r - 1)) - 1)) != 0;
    else
      sticky = lo != 0 || (hi & ((1ull << (r - 1 - 64)) - 1)) != 0;
    if (round && (sticky || (mant & 1))) {
      mant += 1;
      if (mant >> P) {
        mant >>= 1;
        r += 1;
      }
    }
  }
  return true;
}

// Bit b of the 128-bit magnitude (hi, lo), and whether any of its bits below b is set.
__device__ __forceinline__ bool bit128(unsigned long long hi, unsigned long long lo, int b) {
  return b < 64 ? (lo >> b) & 1 : (hi >> (b - 64)) & 1;
}
__device__ __forceinline__ bool low128(unsigned long long hi, unsigned long long lo, int b) {  // bits [0, b)
  if (b <= 0) return false;
  if (b <= 64) return (b == 64 ? lo : lo & ((1ull << b) - 1)) != 0;
  if (b >= 128) return (lo | hi) != 0;
  return lo != 0 || (hi & ((1ull << (b - 64)) - 1)) != 0;
}

// A result below the smallest normal number (rare): w * 2^L rounded once, ties to even,
// to a multiple of the format's smallest subnormal 2^emin_sub, returned as that multiple
// (at most 2^P-1: the next normal number's pattern when it rounds up). Callers pass only
// values below the smallest normal, so |w| < 2^(emin_sub - L + P - 1). Out of line, with
// the words passed by value (no address of the caller's accumulators is taken). The sign
// bit of the result's pattern is added by the caller.
template <int P>
__device__ __noinline__ unsigned long long acc_round_subnormal(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                                               int L, int emin_sub) {
  unsigned long long lo = ((unsigned long long)w1 << 32) | w0;
  unsigned long long hi = ((unsigned long long)w3 << 32) | w2;
  const bool neg = (long long)hi < 0;
  if (neg) {
    lo = ~lo;
    hi = ~hi;
    lo += 1;
    if (lo == 0) hi += 1;
  }
  const int sh = emin_sub - L;  // the grid step in units of w
  if (sh <= 0) return lo << (-sh);  // exact (then |w| < 2^(P-1+sh), so hi = 0)
  if (sh > 128) return 0;           // |w| < 2^128 <= half a step
  unsigned long long q = sh < 128 ? shr128(hi, lo, sh) : 0ull;
  const bool round = bit128(hi, lo, sh - 1);
  if (round && (low128(hi, lo, sh - 1) || (q & 1))) q += 1;
  return q;
}

// The integer w times 2^L rounded to the nearest double: the 53-bit significand and the
// exponent are assembled into the double's bit pattern (GB300's FP64 pipe is narrow, so
// no FP64 instruction is spent per element). A result below the normal range is rounded
// once on the subnormal grid (not first to 53 bits); one beyond it is an infinity.
__device__ __forceinline__ double acc_to_double(const uint32_t (&w)[4], int L) {
  bool neg;
  unsigned long long mant;
  int r;
  if (!acc_round<53>(w, neg, mant, r)) return 0.0;
  const int biased = r + L + 52 + 1023;
  if (biased >= 1 && biased <= 2046)  // sign, exponent and significand assembled as bits
    return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)biased << 52) |
                                            (mant & ((1ull << 52) - 1))));
  if (biased > 2046) return neg ? -CUDART_INF : CUDART_INF;
  const unsigned long long q = acc_round_subnormal<53>(w[0], w[1], w[2], w[3], L, -1074);
  return __longlong_as_double((long long)(((unsigned long long)neg << 63) | q));
}

// The same rounded once to float32 (24-bit significand), for float32 elements.
__device__ __forceinline__ float acc_to_float(const uint32_t (&w)[4], int L) {
  bool neg;
  unsigned long long mant;
  int r;
  if (!acc_round<24>(w, neg, mant, r)) return 0.0f;
  const int biased = r + L + 23 + 127;
  if (biased >= 1 && biased <= 254)
    return __uint_as_float(((uint32_t)neg << 31) | ((uint32_t)biased << 23) | ((uint32_t)mant & 0x7FFFFFu));
  if (biased > 254) return neg ? -CUDART_INF_F : CUDART_INF_F;
  const unsigned long long q = acc_round_subnormal<24>(w[0], w[1], w[2], w[3], L, -149);
  return __uint_as_float(((uint32_t)neg << 31) | (uint32_t)q);
}

// A float32 result travels through the double staging buffer as its bit pattern.
__device__ __forceinline__ double f32_slot(float f) { return __longlong_as_double((long long)__float_as_uint(f)); }
__device__ __forceinline__ float f32_of_slot(double d) { return __uint_as_float((uint32_t)__double_as_longlong(d)); }

// w += v, 128-bit two's complement
__device__ __forceinline__ void add128(uint32_t (&w)[4], const uint4& v) {
  asm("add.cc.u32 %0, %0, %4;\n\t"
      "addc.cc.u32 %1, %1, %5;\n\t"
      "addc.cc.u32 %2, %2, %6;\n\t"
      "addc.u32 %3, %3, %7;"
      : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3])
      : "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w));
}

template <int R>
__device__ __forceinline__ void regs_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(R));
}
template <int R>
__device__ __forceinline__ void regs_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(R));
}

// True when v is true in every thread of the kEpiThreads epilogue threads (named barrier 1
// with an AND reduction; all of them must call it).
__device__ __forceinline__ bool epi_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(kEpiThreads)
      : "memory");
  return r != 0;
}

// C = alpha*v + beta*C for a 128 x TN region staged in shared memory (row stride TN + 1),
// on the elements that lie in S_C tiles. Warp w of NW stores rows w*(128/NW) .. with
// lane = column (TN == 32), so a store instruction writes one or two contiguous row
// segments; per pass of up to 16 rows, lanes fetch the rows' tile and row-in-tile and
// shuffles hand them out.
template <int TN, int NW, int ELEM>  // ELEM: 0 float64, 1 float32, 2 complex (one part per column)
__device__ __forceinline__ void store_region(const SplitArgs& P, const double* cstage, int rb, int cb, int w, int lane,
                                             int32_t* err) {
  static_assert(TN == 32, "one column per lane");
  constexpr int kRowsPerWarp = kSplitBM / NW;
  constexpr int kPass = kRowsPerWarp < 16 ? kRowsPerWarp : 16;  // rows whose offsets are in flight together
  static_assert(kRowsPerWarp % kPass == 0, "whole passes");
  const int64_t nl = (int64_t)cb * TN + lane;
  const bool col_ok = nl < P.Ntot;
  const int jl = col_ok ? P.col_tile[nl] : 0;
  const int64_t lcl = col_ok ? nl - P.co[jl] : 0;
  const int64_t cjl = col_ok ? P.c[jl] : 0;
  const double alpha = P.alpha, beta = P.beta;
  const float alpha32 = (float)alpha, beta32 = (float)beta;  // float32 elements: exact (given as floats)
#pragma unroll 1
  for (int r0 = 0; r0 < kRowsPerWarp; r0 += kPass) {
    const int64_t mr = (int64_t)rb * kSplitBM + w * kRowsPerWarp + r0 + (lane % kPass);
    const int ir = mr < P.Mtot ? P.row_tile[mr] : 0;
    const int lrr = mr < P.Mtot ? (int)(mr - P.ro[ir]) : 0;
    // every row's C tile offset first (independent loads, all in flight), then the stores
    int64_t offs[kPass];
    int lr2s[kPass];
#pragma unroll
    for (int rr = 0; rr < kPass; rr++) {
      const int64_t m2 = (int64_t)rb * kSplitBM + w * kRowsPerWarp + r0 + rr;
      const int i2 = __shfl_sync(0xffffffffu, ir, rr);
      lr2s[rr] = __shfl_sync(0xffffffffu, lrr, rr);
      offs[rr] = -2;
      if (m2 < P.Mtot && col_ok) {
        const int64_t tile = (int64_t)i2 * P.N + jl;
        offs[rr] = P.cs[tile] ? P.c_off[tile] : -2;
      }
    }
#pragma unroll
    for (int rr = 0; rr < kPass; rr++) {
      const int r2 = w * kRowsPerWarp + r0 + rr;
      const int lr2 = lr2s[rr];
      const int64_t off = offs[rr];
      if (off == -1) atomicOr(err, kErrBadOffset);
      if (off < 0) continue;
      if constexpr (ELEM == 2) {
        // column lcl of the doubled tile: the real part of complex column lcl, or the
        // imaginary part of column lcl - c_j / 2
        const int64_t cc = cjl >> 1;
        const int64_t part = lcl >= cc;
        double* dst = P.C + 2 * (off + (int64_t)lr2 * cc + lcl - part * cc) + part;
        double vv = cstage[r2 * (TN + 1) + lane];
        if (alpha != 1.0) vv = __dmul_rn(alpha, vv);
        if (beta != 0.0) vv = __dadd_rn(vv, __dmul_rn(beta, *dst));
        *dst = vv;
      } else if constexpr (ELEM == 1) {
        float* dst = P.Cf + off + (int64_t)lr2 * cjl + lcl;
        float vv = f32_of_slot(cstage[r2 * (TN + 1) + lane]);
        if (alpha32 != 1.0f) vv = __fmul_rn(alpha32, vv);
        if (beta32 != 0.0f) vv = __fadd_rn(vv, __fmul_rn(beta32, *dst));
        *dst = vv;
      } else {
        double* dst = P.C + off + (int64_t)lr2 * cjl + lcl;
        double vv = cstage[r2 * (TN + 1) + lane];
        if (alpha != 1.0) vv = __dmul_rn(alpha, vv);
        if (beta != 0.0) vv = __dadd_rn(vv, __dmul_rn(beta, *dst));
        *dst = vv;
      }
    }
  }
}

// One thread's row of a unit's sums rounded into the staging buffer: doubles, or float32
// bit patterns for float32 elements (zero outside the product).
template <int TH, bool F32>
__device__ __forceinline__ void round_row(const uint32_t (&acc)[TH][4], double* srow, const SplitArgs& P, bool row_ok,
                                          int64_t n0, int Lrow) {
  // the TH columns' maxima with a few 16-byte loads (n0 is a multiple of TH)
  int emc[TH];
#pragma unroll
  for (int w = 0; w < TH / 4; w++) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(P.emaxc + n0) + w);
    emc[4 * w] = v.x;
    emc[4 * w + 1] = v.y;
    emc[4 * w + 2] = v.z;
    emc[4 * w + 3] = v.w;
  }
#pragma unroll
  for (int c = 0; c < TH; c++) {
    const int64_t n = n0 + c;
    double v = 0.0;
    if (row_ok && n < P.Ntot) {
      const int L = Lrow + emc[c];
      if constexpr (F32)
        v = f32_slot(acc_to_float(acc[c], L));
      else
        v = acc_to_double(acc[c], L);
    }
    srow[c] = v;
  }
}

// ---------------------------------------------------------------- kernel 3: contraction
// Ascending k blocks of one unit (a 128-row block times a group of cl column blocks):
// presA[rb] & presBg[group], within the unit's inner-block range [k0, k1) (all of it, or
// one piece under split k). Each CTA of the group takes from it, with next_own(), the k
// blocks where its own column block has a B tile.
struct UnitIter {
  const uint64_t* pa;
  const uint64_t* pb;
  const uint64_t* po;  // this CTA's own column block (null: beyond the last one)
  int kwords, wd, kend;
  uint64_t bits;
  __device__ void init(const SplitArgs& a, const SplitUnit& un, int cb) {
    pa = a.presA + (size_t)un.rb * a.kwords;
    pb = a.presBg + (size_t)un.cb * a.kwords;
    po = cb < a.CB ? a.presB + (size_t)cb * a.kwords : nullptr;
    kwords = a.kwords;
    kend = un.k1;
    wd = un.k0 >> 6;
    bits = wd < kwords ? (pa[wd] & pb[wd]) & (~0ull << (un.k0 & 63)) : 0ull;
  }
  __device__ bool own_b(int k) const { return po && ((po[k >> 6] >> (k & 63)) & 1); }
  __device__ int next_own() {  // next k block that also has a B tile in this CTA's column block
    for (int k = next(); k >= 0; k = next())
      if (own_b(k)) return k;
    return -1;
  }
  __device__ int next() {  // -1 when done
    while (!bits) {
      if (++wd >= kwords) return -1;
      bits = pa[wd] & pb[wd];
    }
    const int k = wd * 64 + __ffsll((long long)bits) - 1;
    if (k >= kend) {  // past the unit's range
      bits = 0;
      wd = kwords;
      return -1;
    }
    bits &= bits - 1;
    return k;
  }
};

// Accumulation groups: consecutive k blocks of a CTA's own list (those where its column
// block has a B tile) share one TMEM accumulation when each has a uniform scale class
// for the unit, the classes add up to the same binary position, and the total inner depth
// keeps every FP32 partial sum exact. The MMA warps and the epilogue apply the same rule
// to the same list, so they agree on where the accumulator is drained.
// The scale class of k block k for the unit's row block rb and column block cb: true
// and the binary offset sig of its products when both classes are uniform.
// A class more than kSplitGuard binades below the unit's largest scale is not uniform
// either: its products enter the accumulator rounded down (floor) to its unit, and the
// floor of a sum is not the sum of the floors, so such k blocks are drained one by one,
// each product taking its own floor as the exact sum's definition states.
__device__ __forceinline__ bool scale_class(const SplitArgs& P, int k, int rb, int cb, int& sig) {
  if (!P.urow) return false;
  const int u = P.urow[(size_t)k * P.RB + rb], v = P.ucol[(size_t)k * P.CB + cb];
  if (u == kNonUniform || v == kNonUniform || u + v < -kSplitGuard) return false;
  sig = u + v;
  return true;
}

struct GroupRule {
  bool uni;
  int sig, depth, kdepth;
  __device__ void start(bool uni_, int sig_, int q, int kdepth_) {
    uni = uni_;
    sig = sig_;
    depth = q;
    kdepth = kdepth_;
  }
  __device__ bool joins(bool uni_, int sig_, int q) {  // true: the k block joins (its depth is added)
    if (!uni || !uni_ || sig_ != sig || depth + q > kdepth) return false;
    depth += q;
    return true;
  }
};

// A group is complete: its descriptor goes to the epilogue (from the first MMA warp),
// then every MMA warp's commit marks the buffer full once its MMAs have finished.
__device__ __forceinline__ void close_group(bool first, int4* gdesc, uint64_t* gready, uint64_t* tfull, uint32_t buf,
                                            int gk0, const GroupRule& grp, bool last) {
  if (first) {
    gdesc[buf] = make_int4(gk0, grp.sig, (grp.uni ? 1 : 0) | (last ? 2 : 0), 0);
    mbar_arrive(&gready[buf]);
  }
  umma_commit(&tfull[buf]);
}

// The values of one own k block of a unit's list that the MMA warps need, loaded ahead.
struct KAhead {
  int k, q;
  bool uni;
  int sig;
  __device__ void load(const SplitArgs& P, int k_, int rb, int cb) {  // k_: an own k block, or -1
    k = k_;
    q = 0;
    uni = false;
    sig = 0;
    if (k < 0) return;
    q = P.q[k];
    uni = scale_class(P, k, rb, cb, sig);
  }
};

// The chunks of one CTA's unit list in order: unit by unit, k block by k block
// (ascending; only the k blocks where the CTA's own column block has a B tile), 32-deep
// chunk by chunk.
struct ChunkCursor {
  const SplitArgs* P;  // the product of the current unit (the batch-wide args for one product)
  int idx, uend;
  int rb, cb;  // this CTA's row block and column block
  UnitIter it;
  int kt, kc, nkc;
  bool in_unit;
  const uint8_t* asrc;
  const uint8_t* bsrc;
  __device__ void start(int beg, int end) {
    idx = beg - 1;
    uend = end;
    in_unit = false;
    kc = 0;
    nkc = 0;
  }
  __device__ bool advance(const SplitArgs& a, int cl, int rank) {  // false when exhausted
    if (++kc < nkc) return true;
    for (;;) {
      if (in_unit) {
        kt = it.next_own();
        if (kt >= 0) {
          nkc = (P->q[kt] + kSplitKC - 1) / kSplitKC;  // >= 1: blocks with q = 0 are never present
          kc = 0;
          asrc = P->apk + P->apk_off[(size_t)rb * P->K + kt];
          bsrc = P->bpk + P->bpk_off[(size_t)kt * P->CB + cb];
          return true;
        }
        in_unit = false;
      }
      if (++idx >= uend) return false;
      int g = a.sched_units[idx];
      P = a.prods ? &a.prods[a.unit_prod[g]] : &a;
      if (a.prods) g = a.unit_local[g];
      const SplitUnit un = P->units[g];
      rb = un.rb;
      cb = un.cb * cl + rank;
      it.init(*P, un, cb);
      in_unit = true;
    }
  }
};

// a.cl consecutive CTAs form a column-block group: they take the same units (a 128-row
// block times cl column blocks), each its own column block, at about the same time, so
// the A panel they all read is served from L2. Every CTA loads its own operands; no CTA
// reads or signals another's shared memory.
// WALK: the epilogue finds the accumulation groups on its own k list (products of long
// k lists) instead of taking the MMA warps' descriptors; the two ways share no code path,
// so each form keeps its own register allocation.
// DEEP: some inner block is deeper than the exact FP32 depth; such a block (it always
// starts a group of its own) is cut into groups of kdepth / 32 whole 32-deep chunks, the
// last of which may take the following blocks. A form of its own, because any extra work
// in the MMA-issuing loop slows every product.
template <int S, int TN, bool SW, bool WALK, bool DEEP>
__global__ void __launch_bounds__(threads_of<SW>(), 1) split_mma_kernel(const __grid_constant__ SplitArgs a) {
  constexpr int TH = TN / 2;                    // columns per epilogue thread
  constexpr int A_STAGE = S * kAChunk;          // bytes of A per stage
  constexpr int B_STAGE = S * TN * kSplitKC * 2;
  constexpr int STAGE = A_STAGE + B_STAGE;
  constexpr int BUF_COLS = S * TN;              // TMEM columns per accumulator buffer
  constexpr int W = S < kMmaWarps ? S : kMmaWarps;  // MMA warps with work: warp 1+w issues slices p = w+1, w+1+W, ...
  static_assert(A_STAGE % 16 == 0 && B_STAGE % 16 == 0, "bulk copies move multiples of 16 bytes");
  static_assert(TN == 32, "the coalesced C store maps one column to each lane");

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int stages = a.stages;
  uint64_t* bars = (uint64_t*)(smem + (size_t)stages * STAGE);
  uint64_t* full = bars;
  uint64_t* empty = bars + stages;
  uint64_t* tfull = bars + 2 * stages;
  uint64_t* tempty = tfull + 2;
  uint64_t* gready = tempty + 2;  // a group's descriptor is in gdesc[buf]
  uint64_t* cready = gready + 2;  // the unit's rounded results are in cstage
  uint64_t* cfree = cready + 1;   // the store warps are done with cstage
  uint64_t* drain = cfree + 1;    // one per MMA warp
  uint32_t* tmem_slot = (uint32_t*)(drain + kMmaWarps);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  // the accumulation group in TMEM buffer b: first k block, binary offset of a uniform
  // group, flags (1: uniform scale class, 2: the unit's last group); written by the first
  // MMA warp when it closes the group
  int4* gdesc = (int4*)(((uintptr_t)(tmem_slot + 2) + 15) & ~(uintptr_t)15);
  // the unit's results on their way to C: 128 rows x (TN + 1) doubles (padded rows)
  double* cstage = (double*)(smem + (size_t)stages * STAGE + kSplitBarBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int CL = a.cl;
  const int cta = blockIdx.x / CL;   // the group: schedules are per group
  const int rank = blockIdx.x % CL;  // this CTA's column block within the group's units
  const int ubeg = a.sched_ptr[cta], uend = a.sched_ptr[cta + 1];

  if (threadIdx.x == 0) {
    for (int st = 0; st < stages; st++) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], W);  // released by every MMA warp
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&tfull[b], W);
      mbar_init(&tempty[b], kSplitEpiWarps);
      mbar_init(&gready[b], 1);
    }
    mbar_init(cready, kEpiThreads);         // every epilogue thread, after its row
    mbar_init(cfree, kStoreWarps * 32);     // every store thread, after its rows
    for (int w = 0; w < kMmaWarps; w++) mbar_init(&drain[w], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // Roles by warpgroup; with store warps each warpgroup first takes its register share
  // (every warp of the warpgroup executes the setmaxnreg, and it dominates the role's code).
  if (warp < kEpiWarp0) {
    if constexpr (SW) regs_dec<kRegsCtl>();
  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued = 0;  // bit st: stage st holds an issued copy; its parity in issued_par
      uint32_t issued_par = 0;
      bool ok = true;
      ChunkCursor cur;
      cur.start(ubeg, uend);
      while (ok && cur.advance(a, CL, rank)) {
        if (!wait1(&empty[stage], phase ^ 1, abort_flag, a.err)) {
          ok = false;
          break;
        }
        uint8_t* sa = smem + (size_t)stage * STAGE;
        mbar_arrive_expect_tx(&full[stage], STAGE);
        bulk_g2s(sa, cur.asrc + (size_t)cur.kc * A_STAGE, A_STAGE, &full[stage]);
        bulk_g2s(sa + A_STAGE, cur.bsrc + (size_t)cur.kc * B_STAGE, B_STAGE, &full[stage]);
        issued |= 1u << stage;
        issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
        if (++stage == stages) {
          stage = 0;
          phase ^= 1;
        }
      }
      // drain: every copy this thread issued has landed before the CTA may exit
      for (int st = 0; st < stages; st++) {
        if (!(issued >> st & 1)) continue;
        const uint32_t par = issued_par >> st & 1;
        const int64_t t0 = gtimer();
        while (!mbar_try_wait(&full[st], par)) {
          if (gtimer() - t0 > kWaitNs) {
            atomicOr(a.err, kErrTimeout);
            break;
          }
        }
      }
    }
  } else if (warp <= W) {
    // ------------------------------------------------------------ MMA issuers
    // Every MMA warp walks the same chunks and issues its share of each step's slice
    // products; all of them accumulate (the epilogue zeroes a buffer once drained), and
    // the order in which the tensor core applies them does not matter: every partial sum
    // is an integer below 2^24, exact in FP32.
    if (lane == 0) {
      const int mw = warp - 1;
      int stage = 0;
      uint32_t phase = 0;
      uint32_t tcount = 0;
      bool ok = true;
      bool any = false;
      // Descriptors are built once: within a stage, slice p of A starts (p-1)*kAChunk bytes
      // in and the second 16-deep step 32 bytes in, i.e. fixed additions to the 16-byte
      // start-address field (which cannot carry: shared addresses are below 256 KB).
      const uint64_t adesc0 = sdesc_sw64(smem_u32(smem));
      const uint64_t bdesc0 = sdesc_sw64(smem_u32(smem) + A_STAGE);
      constexpr int NP = (S + W - 1) / W;  // slices per warp (upper bound)
      uint32_t idp[NP];
      uint32_t dcol[NP];
      uint64_t aoff[NP];
#pragma unroll
      for (int j = 0; j < NP; j++) {
        const int p = mw + 1 + j * W;
        idp[j] = idesc_f16(kSplitBM, (S + 1 - (p <= S ? p : S)) * TN, a.fp16 != 0);
        dcol[j] = (uint32_t)((p - 1) * TN);
        aoff[j] = (uint64_t)((p - 1) * (kAChunk >> 4));
      }
      for (int idx = ubeg; idx < uend && ok; idx++) {
        int g = a.sched_units[idx];
        const SplitArgs& P = a.prods ? a.prods[a.unit_prod[g]] : a;
        if (a.prods) g = a.unit_local[g];
        const SplitUnit un = P.units[g];
        const int cb = un.cb * CL + rank;
        UnitIter it;
        it.init(P, un, cb);
        GroupRule grp;
        bool in_group = false;
        uint32_t buf = 0;
        int gk0 = 0;  // the current group's first k block
        // per-k values are loaded one k block ahead, so their latency hides behind the
        // current block's MMAs; a group is closed when the next own k block does not join
        KAhead cur, nxt;
        cur.load(P, it.next_own(), un.rb, cb);
        while (cur.k >= 0 && ok) {
          nxt.load(P, it.next_own(), un.rb, cb);
          const int kt = cur.k;
          const int q = cur.q;
          const int nkc = (q + kSplitKC - 1) / kSplitKC;
          if (!(in_group && grp.joins(cur.uni, cur.sig, cur.q))) {
            if (in_group) {  // the previous group is complete
              close_group(mw == 0, gdesc, gready, tfull, buf, gk0, grp, false);
              tcount++;
            }
            buf = tcount & 1;
            const uint32_t use = tcount >> 1;
            // the buffer was drained and zeroed by the epilogue (use 0: zeroed at start)
            if (!wait1(&tempty[buf], use & 1, abort_flag, a.err)) {
              ok = false;
              in_group = false;
              break;
            }
            tc_fence_after();
            grp.start(cur.uni, cur.sig, cur.q, P.kdepth);
            gk0 = kt;
            in_group = true;
          }
          uint32_t dbase = tmem_base + buf * BUF_COLS;
          for (int kc = 0; kc < nkc; kc++) {
            if constexpr (DEEP) {
              const int cpg = P.kdepth >= kSplitKC ? P.kdepth / kSplitKC : 1;
              if (kc > 0 && q > P.kdepth && kc % cpg == 0) {  // the block's next group
                close_group(mw == 0, gdesc, gready, tfull, buf, gk0, grp, false);
                tcount++;
                buf = tcount & 1;
                if (!wait1(&tempty[buf], (tcount >> 1) & 1, abort_flag, a.err)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                dbase = tmem_base + buf * BUF_COLS;
              }
            }
            if (!wait1(&full[stage], phase, abort_flag, a.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            {
              const uint64_t soff = (uint64_t)((stage * STAGE) >> 4);
              const uint64_t ad = adesc0 + soff, bd = bdesc0 + soff;
              const bool two = q - kc * kSplitKC > 16;  // second 16-deep step of the 32-deep chunk
#pragma unroll
              for (int j = 0; j < NP; j++) {
                if (mw + 1 + j * W > S) break;
                umma_f16(dbase + dcol[j], ad + aoff[j], bd, idp[j], 1u);
                if (two) umma_f16(dbase + dcol[j], ad + aoff[j] + 2, bd + 2, idp[j], 1u);
              }
            }
            umma_commit(&empty[stage]);  // the stage is free once these MMAs have finished
            any = true;
            if (++stage == stages) {
              stage = 0;
              phase ^= 1;
            }
          }
          if constexpr (DEEP) {
            const int cpg = P.kdepth >= kSplitKC ? P.kdepth / kSplitKC : 1;
            if (q > P.kdepth) grp.depth = q - kSplitKC * cpg * ((nkc - 1) / cpg);  // its last group's depth
          }
          cur = nxt;
        }
        if (in_group && ok) {  // the unit's last group
          close_group(mw == 0, gdesc, gready, tfull, buf, gk0, grp, true);
          tcount++;
        }
      }
      // drain: every MMA this thread issued has completed before TMEM is released
      if (any) {
        umma_commit(&drain[mw]);
        const int64_t t0 = gtimer();
        while (!mbar_try_wait(&drain[mw], 0)) {
          if (gtimer() - t0 > kWaitNs) {
            atomicOr(a.err, kErrTimeout);
            break;
          }
        }
      }
    }
  }
  } else if (warp < kStoreWarp0) {
    if constexpr (SW) regs_inc<kRegsEpi>();
    // ------------------------------------------------------------ epilogue warps
    const int ew = warp - kEpiWarp0;   // 0..7
    const int quad = warp & 3;         // TMEM lane quadrant this warp may access
    const int half = ew >> 2;          // which half of the tn columns
    const int row = quad * 32 + lane;  // row inside the unit
    const uint32_t tq = tmem_base + ((uint32_t)(quad * 32) << 16) + half * TH;  // this warp's lanes and columns
    // both accumulator buffers start at zero; the MMA warps only ever accumulate
#pragma unroll 1
    for (int b = 0; b < 2; b++)
#pragma unroll
      for (int d = 0; d < S; d++)
#pragma unroll
        for (int cc = 0; cc < TH / 8; cc++) tmem_zero8(tq + b * BUF_COLS + d * TN + cc * 8);
    tmem_st_wait();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&tempty[0]);
      mbar_arrive(&tempty[1]);
    }
    uint32_t tcount = 0;
    uint32_t ncs = 0;  // uses of cstage so far
    bool ok = true;
    for (int idx = ubeg; idx < uend && ok; idx++) {
      int u = a.sched_units[idx];
      const SplitArgs& P = a.prods ? a.prods[a.unit_prod[u]] : a;
      if (a.prods) u = a.unit_local[u];
      const SplitUnit un = P.units[u];
      const int cb = un.cb * CL + rank;
      if (cb >= P.CB) continue;  // a group's CTA past the last column block has no work
      // timing record: the unit's start (the group's first CTA) and the longest time any CTA
      // of the group spends on it
      const int64_t t_unit = a.timings && ew == 0 && lane == 0 ? gtimer() : 0;
      if (a.timings && rank == 0 && ew == 0 && lane == 0) a.timings[2 * (int64_t)u] = t_unit;
      const int64_t m = (int64_t)un.rb * kSplitBM + row;
      const bool row_ok = m < P.Mtot;
      const int64_t n0 = (int64_t)cb * TN + half * TH;
      uint32_t acc[TH][4];  // exact 128-bit two's-complement sums, unit 2^L per column
#pragma unroll
      for (int c = 0; c < TH; c++) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0u;
      // The unit's accumulation groups, in the order the MMA warps fill them. With WALK the
      // epilogue walks the CTA's own k list with the MMA warps' rule, ahead of them;
      // otherwise it takes each group's descriptor when the first MMA warp closes it (none
      // when this CTA's column block has no B tile in the unit's inner range: the planner's
      // own mask). Either way the groups are the same, in the same order.
      UnitIter it;
      int kt = -1;
      [[maybe_unused]] int sub = 0;  // DEEP: groups already taken from k block kt
      if constexpr (WALK) {
        it.init(P, un, cb);
        kt = it.next_own();
      }
      bool more = WALK ? kt >= 0 : ((un.own >> rank) & 1) != 0;
      while (more) {
        const uint32_t buf = tcount & 1, use = tcount >> 1;
        int gk0, gsig;  // the group's first k block and, for a uniform group, its class
        bool guni;
        if constexpr (WALK) {
          GroupRule grp;
          {
            int sg = 0;
            const bool uni = scale_class(P, kt, un.rb, cb, sg);
            grp.start(uni, sg, P.q[kt], P.kdepth);
          }
          gk0 = kt;
          guni = grp.uni;
          gsig = grp.sig;
          bool whole = true;  // DEEP: a deep block's groups but its last take no other block
          if constexpr (DEEP) {
            const int qk = P.q[kt];
            if (qk > P.kdepth) {
              const int cpg = P.kdepth >= kSplitKC ? P.kdepth / kSplitKC : 1;
              const int nsub = ((qk + kSplitKC - 1) / kSplitKC + cpg - 1) / cpg;
              if (++sub < nsub) {
                whole = false;
              } else {
                grp.depth = qk - kSplitKC * cpg * (nsub - 1);
                sub = 0;
              }
            }
          }
          if (whole) {
            int kn = it.next_own();
            for (; kn >= 0; kn = it.next_own()) {
              int sg = 0;
              const bool uni = scale_class(P, kn, un.rb, cb, sg);
              if (!grp.joins(uni, sg, P.q[kn])) break;
            }
            kt = kn;
          }
          more = kt >= 0;
        } else {
          // (the epilogue warps sleep between polls here: while the MMA warps fill a group
          // they would otherwise take issue slots from the producer and MMA threads)
          if (!wait_warp(&gready[buf], use & 1, abort_flag, a.err, kWaitNs, kGroupPollNs)) {
            ok = false;
            break;
          }
          const int4 gd = gdesc[buf];
          more = (gd.z & 2) == 0;
          gk0 = gd.x;
          guni = (gd.z & 1) != 0;
          gsig = gd.y;
        }
        // the binary position of the group's integers: one shift for a uniform group (its
        // common class plus the row's and the columns' parts), per-row and per-column
        // offsets for a lone k block; loaded while the tensor core finishes the group
        int shr = kSplitGuard;
        uint4 cx[TH / 8];
        if (guni) {
          shr += gsig + (row_ok ? (int)P.rowadj[m] : 0);
          const uint4* src = reinterpret_cast<const uint4*>(P.coladj + n0);
#pragma unroll
          for (int w = 0; w < TH / 8; w++) cx[w] = __ldg(src + w);
        } else {
          shr += row_ok ? (int)P.rowexp[(int64_t)gk0 * P.Mtot + m] : 0;
          const uint4* src = reinterpret_cast<const uint4*>(P.colexp + (int64_t)gk0 * P.colexp_ld + n0);
#pragma unroll
          for (int w = 0; w < TH / 8; w++) cx[w] = __ldg(src + w);
        }
        if (!wait_warp(&tfull[buf], use & 1, abort_flag, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tq + buf * BUF_COLS;
        // columns in batches of CW (4 for s >= 5 keeps the TMEM values and the 128-bit
        // sums within the register budget)
        constexpr int CW = S >= 5 ? 4 : 8;
#pragma unroll
        for (int cc = 0; cc < TH / CW; cc++) {
          uint32_t v[S][CW];
#pragma unroll
          for (int d = 0; d < S; d++) {
            if constexpr (CW == 8)
              tmem_ld8(taddr + d * TN + cc * CW, v[d]);
            else
              tmem_ld4(taddr + d * TN + cc * CW, v[d]);
          }
          tmem_ld_wait();
#pragma unroll
          for (int d = 0; d < S; d++) {  // ready for the buffer's next use
            if constexpr (CW == 8)
              tmem_zero8(taddr + d * TN + cc * CW);
            else
              tmem_zero4(taddr + d * TN + cc * CW);
          }
#pragma unroll
          for (int c = 0; c < CW; c++) {
            // T = sum_d S_d 2^(7(S+1-d)), exact: the tensor core's FP32 sums are integers
            long long T = 0;
#pragma unroll
            for (int d = 0; d < S; d++) {
              int iv;
              asm("cvt.rni.s32.f32 %0, %1;" : "=r"(iv) : "f"(__uint_as_float(v[d][c])));
              T += (long long)iv * (1ll << (kSplitBeta * (S - 1 - d)));
            }
            const int col = cc * CW + c;  // column within this thread's TH
            const uint4& w4 = cx[col >> 3];
            const int e = col & 7;
            const uint32_t wd = e < 2 ? w4.x : e < 4 ? w4.y : e < 6 ? w4.z : w4.w;
            acc_add(acc[col], T, shr + (int)(int16_t)(wd >> (16 * (e & 1))));
          }
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
        tcount++;
      }
      // (a warp whose wait gave up still passes the barriers below, so that no other
      // epilogue warp waits at them for it; every wait before them is bounded and sees the
      // abort flag, so all eight warps reach them, and the last one agrees on the outcome,
      // so all eight leave the unit loop together)
      if (un.slot < 0) {
        // C = alpha*fl(sum) + beta*C on the unit's elements that lie in S_C tiles: each
        // thread rounds its row's sums to doubles into the staging buffer (with store warps,
        // once they are done with the previous unit's); then whole rows are stored, lane =
        // column, so a store instruction writes one or two contiguous row segments. With
        // store warps the store runs while this warp drains the next unit.
        if constexpr (SW)
          if (ok && !wait_warp(cfree, (ncs & 1) ^ 1, abort_flag, a.err)) ok = false;
        if (ok) {
          // the accumulator's unit 2^L: per row block and column block of tiles, or per row
          // and column with row/column scaling
          const int Lrow = row_ok ? P.emaxr[m] - kSplitBeta * (S + 1) - kSplitGuard : 0;
          double* srow = cstage + row * (TN + 1) + half * TH;
          if (P.f32)
            round_row<TH, true>(acc, srow, P, row_ok, n0, Lrow);
          else
            round_row<TH, false>(acc, srow, P, row_ok, n0, Lrow);
        }
        if constexpr (SW) {
          mbar_arrive(cready);  // every thread: its row is in cstage (release)
          ncs++;
        } else {
          asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory");
          if (ok && !*abort_flag) {
            if (P.f32)
              store_region<TN, kSplitEpiWarps, 1>(P, cstage, un.rb, cb, ew, lane, a.err);
            else if (P.cplx)
              store_region<TN, kSplitEpiWarps, 2>(P, cstage, un.rb, cb, ew, lane, a.err);
            else
              store_region<TN, kSplitEpiWarps, 0>(P, cstage, un.rb, cb, ew, lane, a.err);
          }
        }
      } else if (ok) {
        // a piece of a split k-list: its exact partial sums go to the workspace (column-
        // major, so the 32 rows of a warp write 512 contiguous bytes per column)
        uint4* dst = P.part + ((size_t)un.slot * CL + rank) * (TN * kSplitBM) + (size_t)half * TH * kSplitBM + row;
#pragma unroll
        for (int c = 0; c < TH; c++) dst[(size_t)c * kSplitBM] = make_uint4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
      }
      ok = epi_all(ok);  // every epilogue warp has the same outcome (and, without store warps,
                         // cstage is free again)
      if (!ok) break;
      if (a.timings && ew == 0 && lane == 0) {
        atomicMax(reinterpret_cast<unsigned long long*>(&a.timings[2 * (int64_t)u + 1]),
                  (unsigned long long)(gtimer() - t_unit));
        if (rank == 0) a.unit_cta[u] = cta;
      }
    }
  } else if constexpr (SW) {
    regs_dec<kRegsStore>();
    // ------------------------------------------------------------ C store warps
    // The units' rounded results from the staging buffer to C, in the epilogue's unit
    // order, while the epilogue warps drain the next unit.
    const int sw = warp - kStoreWarp0;
    uint32_t ncs = 0;
    for (int idx = ubeg; idx < uend; idx++) {
      int u = a.sched_units[idx];
      const SplitArgs& P = a.prods ? a.prods[a.unit_prod[u]] : a;
      if (a.prods) u = a.unit_local[u];
      const SplitUnit un = P.units[u];
      const int cb = un.cb * CL + rank;
      if (cb >= P.CB || un.slot >= 0) continue;  // units that do not use the staging buffer
      if (!wait_warp(cready, ncs & 1, abort_flag, a.err, kWaitNs, 200)) break;
      if (!*abort_flag) {
        if (P.f32)
          store_region<TN, kStoreWarps, 1>(P, cstage, un.rb, cb, sw, lane, a.err);
        else if (P.cplx)
          store_region<TN, kStoreWarps, 2>(P, cstage, un.rb, cb, sw, lane, a.err);
        else
          store_region<TN, kStoreWarps, 0>(P, cstage, un.rb, cb, sw, lane, a.err);
      }
      mbar_arrive(cfree);  // every thread: done reading cstage (release)
      ncs++;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, kTmemCols);
}

// ---------------------------------------------------------------- kernel 4: split-k reduction
// The reduction task of a region whose k-list was cut into pieces (Sec. 3.2, Fig. 2).
// The pieces' partial sums are exact 128-bit integers in the same unit 2^L, so adding
// them is exact in any order and the rounded result equals the unsplit one bit for bit;
// it is rounded once and stored like the contraction's epilogue. One CTA of 256 threads
// per (region, column block of the region's group); thread = (row, half of the columns).
template <int TN>
__global__ void __launch_bounds__(256) split_reduce_kernel(const __grid_constant__ SplitArgs a) {
  constexpr int TH = TN / 2;
  __shared__ double cstage[kSplitBM * (TN + 1)];
  const SplitRed rd = a.red[blockIdx.x / a.cl];
  const int rank = blockIdx.x % a.cl;
  const int cb = rd.cb * a.cl + rank;
  if (cb >= a.CB) return;
  const int row = threadIdx.x % kSplitBM, half = threadIdx.x / kSplitBM;
  const int64_t m = (int64_t)rd.rb * kSplitBM + row;
  const bool row_ok = m < a.Mtot;
  const int Lrow =
      row_ok ? (a.rowscale ? a.eAmaxr[m] : a.eAmax[a.row_tile[m]]) - kSplitBeta * (a.s + 1) - kSplitGuard : 0;
  const int64_t n0 = (int64_t)cb * TN + half * TH;
  const size_t piece_stride = (size_t)a.cl * TN * kSplitBM;
  const uint4* src = a.part + ((size_t)rd.slot0 * a.cl + rank) * (TN * kSplitBM) + (size_t)half * TH * kSplitBM + row;
  for (int c = 0; c < TH; c++) {
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    for (int p = 0; p < rd.n; p++) add128(w, src[p * piece_stride + (size_t)c * kSplitBM]);
    const int64_t n = n0 + c;
    double v = 0.0;
    if (row_ok && n < a.Ntot) {
      const int L = Lrow + (a.rowscale ? a.eBmaxc[n] : a.eBmax[a.col_tile[n]]);
      v = a.f32 ? f32_slot(acc_to_float(w, L)) : acc_to_double(w, L);
    }
    cstage[row * (TN + 1) + half * TH + c] = v;
  }
  __syncthreads();
  if (a.f32)
    store_region<TN, 8, 1>(a, cstage, rd.rb, cb, threadIdx.x >> 5, threadIdx.x & 31, a.err);
  else if (a.cplx)
    store_region<TN, 8, 2>(a, cstage, rd.rb, cb, threadIdx.x >> 5, threadIdx.x & 31, a.err);
  else
    store_region<TN, 8, 0>(a, cstage, rd.rb, cb, threadIdx.x >> 5, threadIdx.x & 31, a.err);
}

// ---------------------------------------------------------------- bounded-wait self-test
// Two mbarriers that no thread ever arrives at. Warp 0 (one thread) waits on the first
// with the given limit, runs out, sets the error word and the abort flag; warps 1 and 2
// wait on the second (warp-uniform waits, a 20x longer limit) and leave as soon as they
// see the abort flag. The kernel then exits normally: the contraction's wait functions
// and its abort protocol, exercised without a hang.
__global__ void __launch_bounds__(96) wait_selftest_kernel(int32_t* err, int64_t limit_ns) {
  __shared__ uint64_t bars[2];
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) wait1(&bars[0], 0, &abort_flag, err, limit_ns);
  } else {
    wait_warp(&bars[1], 0, &abort_flag, err, 20 * limit_ns);
  }
  __syncthreads();
}

template <int S, int TN, bool SW, bool WALK, bool DEEP = false>
cudaError_t launch_mma(const SplitArgs& a, int groups, cudaStream_t st) {
  const size_t smem = split_smem_bytes(S, TN, a.stages);
  cudaError_t e = cudaFuncSetAttribute(split_mma_kernel<S, TN, SW, WALK, DEEP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (SW) {
    // the register split assumes exactly kRegsLaunch registers per thread at launch (a
    // smaller allocation could not satisfy the epilogue's setmaxnreg.inc): refuse otherwise
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, split_mma_kernel<S, TN, SW, WALK, DEEP>);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != kRegsLaunch) return cudaErrorInvalidConfiguration;
  }
  split_mma_kernel<S, TN, SW, WALK, DEEP><<<(unsigned)(groups * a.cl), threads_of<SW>(), smem, st>>>(a);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_mma_sw(const SplitArgs& a, int groups, cudaStream_t st) {
  if (a.cl != 1 && a.cl != 2 && a.cl != 4) return cudaErrorInvalidValue;
  // the walking epilogue is built for the forms with store warps and 3 to 6 slices (the
  // dense products' default); other forms take the descriptors whatever epi_walk says
  if (a.deep) {  // products with inner blocks deeper than the exact depth: store-warp forms
    if (!a.sw) return cudaErrorInvalidConfiguration;
    if constexpr (S >= 3)
      if (a.epi_walk) return launch_mma<S, 32, true, true, true>(a, groups, st);
    return launch_mma<S, 32, true, false, true>(a, groups, st);
  }
  if constexpr (S >= 3)
    if (a.sw && a.epi_walk) return launch_mma<S, 32, true, true>(a, groups, st);
  return a.sw ? launch_mma<S, 32, true, false>(a, groups, st) : launch_mma<S, 32, false, false>(a, groups, st);
}

// Groups of cl CTAs that are resident at once: the persistent grid (one CTA per SM at
// this shared-memory size) divided into groups.
template <int S, bool SW>
int max_groups_for(int cl, int stages) {
  const size_t smem = split_smem_bytes(S, 32, stages);
  if (cudaFuncSetAttribute(split_mma_kernel<S, 32, SW, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, split_mma_kernel<S, 32, SW, false, false>, threads_of<SW>(), smem) !=
      cudaSuccess)
    return 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return cl > 0 ? per_sm * sms / cl : 0;
}

template <int S>
int max_groups_s(int cl, int stages, bool sw) {
  return sw ? max_groups_for<S, true>(cl, stages) : max_groups_for<S, false>(cl, stages);
}

}  // namespace

template <typename E, bool C = false>
cudaError_t launch_pack(const SplitArgs& a, unsigned g, cudaStream_t st) {
  switch (a.s * 2 + (a.fp16 ? 1 : 0)) {
    case 2: split_pack_kernel<__nv_bfloat16, 1, E, C><<<g, 256, 0, st>>>(a); break;
    case 3: split_pack_kernel<__half, 1, E, C><<<g, 256, 0, st>>>(a); break;
    case 4: split_pack_kernel<__nv_bfloat16, 2, E, C><<<g, 256, 0, st>>>(a); break;
    case 5: split_pack_kernel<__half, 2, E, C><<<g, 256, 0, st>>>(a); break;
    case 6: split_pack_kernel<__nv_bfloat16, 3, E, C><<<g, 256, 0, st>>>(a); break;
    case 7: split_pack_kernel<__half, 3, E, C><<<g, 256, 0, st>>>(a); break;
    case 8: split_pack_kernel<__nv_bfloat16, 4, E, C><<<g, 256, 0, st>>>(a); break;
    case 9: split_pack_kernel<__half, 4, E, C><<<g, 256, 0, st>>>(a); break;
    case 10: split_pack_kernel<__nv_bfloat16, 5, E, C><<<g, 256, 0, st>>>(a); break;
    case 11: split_pack_kernel<__half, 5, E, C><<<g, 256, 0, st>>>(a); break;
    case 12: split_pack_kernel<__nv_bfloat16, 6, E, C><<<g, 256, 0, st>>>(a); break;
    case 13: split_pack_kernel<__half, 6, E, C><<<g, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int split_prep_kernels(const SplitArgs& a) {  // the kernels launch_split_prep launches
  int n = 0;
  if (a.n_a_tiles + a.n_b_tiles > 0) n += a.rowscale ? 2 : 1;
  if (a.rowscale ? a.Mtot + a.Ntot > 0 : a.M + a.N > 0) n++;
  if ((a.urow || !a.rowscale) && (int64_t)a.K * (a.RB + a.CB) > 0) n++;
  if (a.n_a_blocks + a.n_b_blocks > 0) n++;
  return n;
}

cudaError_t launch_split_prep(const SplitArgs& a, cudaStream_t st, cudaEvent_t* ev, int* k) {
  if (a.n_a_tiles + a.n_b_tiles > 0) {
    split_exp_kernel<<<a.n_a_tiles + a.n_b_tiles, 256, 0, st>>>(a);
    if (a.rowscale) split_exp_lines_kernel<<<a.n_a_tiles + a.n_b_tiles, 256, 0, st>>>(a);
  }
  if (a.rowscale) {
    // the per-tile maxima (eAmax/eBmax) are not used in this mode; the line kernel writes
    // rowexp/colexp and the line maxima
    const int64_t lines = a.Mtot + a.Ntot;
    if (lines > 0) split_scale_lines_kernel<<<(unsigned)((lines + 255) / 256), 256, 0, st>>>(a);
  } else if (a.M + a.N > 0) {
    split_emax_kernel<<<a.M + a.N, 256, 0, st>>>(a);
  }
  // tile scaling: the offsets rowexp/colexp; both: the scale classes (when kept)
  const int64_t ncls = (int64_t)a.K * (a.RB + a.CB);
  if ((a.urow || !a.rowscale) && ncls > 0) split_class_kernel<<<(unsigned)((ncls * 32 + 255) / 256), 256, 0, st>>>(a);
  if (ev) cudaEventRecord(ev[++*k], st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.n_a_blocks + a.n_b_blocks > 0) {
    const unsigned g = (unsigned)(a.n_a_blocks + a.n_b_blocks);
    cudaError_t pe = a.f32 ? launch_pack<float>(a, g, st)
                           : a.cplx ? launch_pack<double, true>(a, g, st) : launch_pack<double>(a, g, st);
    if (pe != cudaSuccess) return pe;
  }
  if (ev) cudaEventRecord(ev[++*k], st);
  return cudaGetLastError();
}

// NVTX ranges name the phases of a product for a timeline tool (host-side enqueue spans).
cudaError_t launch_split(const SplitArgs& a, int ctas, cudaStream_t st, cudaEvent_t* ev, int* nk) {
  int k = 0;
  if (ev) cudaEventRecord(ev[0], st);
  nvtxRangePushA("bsmm split: exponents, scales, slices");
  cudaError_t e = launch_split_prep(a, st, ev, &k);
  nvtxRangePop();
  if (e != cudaSuccess) return e;
  nvtxRangePushA("bsmm split: contraction");
  e = launch_split_mma(a, ctas, st);
  nvtxRangePop();
  if (ev) cudaEventRecord(ev[++k], st);
  if (e == cudaSuccess && !a.prods && a.n_red > 0) {  // a batch launches its products' reductions
    nvtxRangePushA("bsmm split: split-k reduction");
    e = launch_split_reduce(a, st);
    nvtxRangePop();
    if (ev) cudaEventRecord(ev[++k], st);
  }
  if (nk) *nk = k;
  return e;
}

cudaError_t launch_wait_selftest(int32_t* err, int64_t limit_ns, cudaStream_t st) {
  wait_selftest_kernel<<<1, 96, 0, st>>>(err, limit_ns);
  return cudaGetLastError();
}

cudaError_t launch_split_reduce(const SplitArgs& a, cudaStream_t st) {
  if (a.n_red <= 0) return cudaSuccess;
  split_reduce_kernel<32><<<(unsigned)(a.n_red * a.cl), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_split_mma(const SplitArgs& a, int ctas, cudaStream_t st) {
  cudaError_t e;
  switch (a.s) {  // `ctas` counts groups of a.cl CTAs
    case 1: e = launch_mma_sw<1>(a, ctas, st); break;
    case 2: e = launch_mma_sw<2>(a, ctas, st); break;
    case 3: e = launch_mma_sw<3>(a, ctas, st); break;
    case 4: e = launch_mma_sw<4>(a, ctas, st); break;
    case 5: e = launch_mma_sw<5>(a, ctas, st); break;
    case 6: e = launch_mma_sw<6>(a, ctas, st); break;
    default: e = cudaErrorInvalidValue;
  }
  return e;
}

int split_max_clusters(int s, int cl, int stages, bool sw) {
  switch (s) {
    case 1: return max_groups_s<1>(cl, stages, sw);
    case 2: return max_groups_s<2>(cl, stages, sw);
    case 3: return max_groups_s<3>(cl, stages, sw);
    case 4: return max_groups_s<4>(cl, stages, sw);
    case 5: return max_groups_s<5>(cl, stages, sw);
    case 6: return max_groups_s<6>(cl, stages, sw);
    default: return 0;
  }
}

}  // namespace bsmm
