// Plain FP64 tile-task kernel.
//
// One persistent CTA walks its packed list of work units. A unit is a 32x32 (or
// 64x64) region of one C tile C_ij; the CTA owns it for the whole task: it runs the
// tile's ascending k-list (the rank-k updates C_ij <- A_ik B_kj + C_ij of the
// paper's Sec. 2.1, multiply and reduction fused as in Sec. 3.2), then applies
// C_ij = alpha*acc + beta*C_ij (Algorithm 1's alpha) and stores.
//
// GB300 has no FP64 tensor-core kind in tcgen05, and its warp-level FP64 MMA
// (mma.sync m8n8k4) measures below its FP64 FMA pipe, so the contraction is a
// register-tiled DFMA loop: (T/4)^2 threads, 4x4 accumulators each, the A and B
// sub-tiles (Tx16 and 16xT) staged through shared memory with the next chunk's
// global loads in flight during the current chunk's FMAs. Irregular tiles are
// read in place from the caller's arena: edges beyond a tile's rows, columns or
// inner size are zero-filled in shared memory, and the FMAs a whole warp would spend
// on them are skipped (see fma_chunk).
//
// Rounding is fixed by construction: each accumulator element takes
// acc = fma(a, b, acc) over k blocks in ascending order and, inside a block,
// ascending kk; the epilogue rounds alpha*acc and beta*C separately before
// adding. The result bits therefore do not depend on the schedule, the CTA count
// or the unit order.
//
// Split k (Sec. 3.2, Fig. 2): when the planner cuts a region's k-list into pieces, each
// piece is a unit that sums its positions from zero and stores the partial sum; the
// reduction kernel adds the partials in piece order and applies the epilogue.
#include <cstdint>

#include <nvtx3/nvToolsExt.h>

#include "bsmm_internal.h"

namespace bsmm {

namespace {

__device__ __forceinline__ int64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (int64_t)t;
}

constexpr int BK = kF64BK;
constexpr int PAD = 2;

// FMAs of one staged chunk for the register-tile rows x < XM and columns y < YM that some
// lane of this warp needs, over the chunk's kv valid inner indices. XM, YM and kv are the
// same for every lane of a warp, so the rows, columns and inner tail a ragged sub-tile does
// not have cost no instructions; each accumulator still takes its FMAs in ascending kk.
template <int XM, int YM, int BK_, int TX, int LDA, int LDB>
__device__ __forceinline__ void fma_chunk(double (&acc)[4][4], const double (*sA)[LDA], const double (*sB)[LDB], int ty,
                                          int tx, int kv) {
  auto step = [&](int kk) {
    double av[XM], bv[YM];
#pragma unroll
    for (int x = 0; x < XM; x++) av[x] = sA[kk][ty + TX * x];
#pragma unroll
    for (int y = 0; y < YM; y++) bv[y] = sB[kk][tx + TX * y];
#pragma unroll
    for (int x = 0; x < XM; x++)
#pragma unroll
      for (int y = 0; y < YM; y++) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
  };
  if (kv == BK_) {
#pragma unroll
    for (int kk = 0; kk < BK_; kk++) step(kk);
  } else {
#pragma unroll 4
    for (int kk = 0; kk < kv; kk++) step(kk);
  }
}

template <int XM, int BK_, int TX, int LDA, int LDB>
__device__ __forceinline__ void fma_chunk_y(double (&acc)[4][4], const double (*sA)[LDA], const double (*sB)[LDB],
                                            int ty, int tx, int kv, int ym) {
  switch (ym) {
    case 4: fma_chunk<XM, 4, BK_, TX, LDA, LDB>(acc, sA, sB, ty, tx, kv); break;
    case 3: fma_chunk<XM, 3, BK_, TX, LDA, LDB>(acc, sA, sB, ty, tx, kv); break;
    case 2: fma_chunk<XM, 2, BK_, TX, LDA, LDB>(acc, sA, sB, ty, tx, kv); break;
    case 1: fma_chunk<XM, 1, BK_, TX, LDA, LDB>(acc, sA, sB, ty, tx, kv); break;
    default: break;
  }
}

struct ChunkIter {
  int64_t t, t_end;  // position in the tile's k-list
  int kk0, qk;
  int k;
};

// T x T sub-tiles (T = 64 or 32): (T/4)^2 threads, each with a 4 x 4 register tile at
// rows ty + (T/4)x and columns tx + (T/4)y. The smaller edge wastes less on ragged tiles.
template <int T>
__global__ void __launch_bounds__((T / 4) * (T / 4), 4096 / (T * T) * 2 > 8 ? 8 : 4096 / (T * T) * 2)
    fp64_tile_kernel(const __grid_constant__ Fp64Args a) {
  constexpr int BM = T, BN = T, TX = T / 4, NT = TX * TX;
  constexpr int A_PER_T = BM * BK / NT;
  constexpr int B_PER_T = BK * BN / NT;
  __shared__ double sA[BK][BM + PAD];  // transposed: [kk][row]
  __shared__ double sB[BK][BN + PAD];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int cta = blockIdx.x;
  const int beg = a.sched_ptr[cta], end = a.sched_ptr[cta + 1];

  for (int idx = beg; idx < end; idx++) {
    // batch: the schedule lists batch-wide unit ids, each of one product
    int u = a.sched_units[idx];
    const Fp64Args& P = a.prods ? a.prods[a.unit_prod[u]] : a;
    if (a.prods) u = a.unit_local[u];
    const Fp64Unit un = P.units[u];
    const int64_t t_unit = a.timings && tid == 0 ? gtimer() : 0;
    if (a.timings && tid == 0) a.timings[2 * (int64_t)u] = t_unit;
    const int i = un.i, j = un.j;
    const int ri = P.r[i], cj = P.c[j];
    const int rows = min(BM, ri - un.r0), cols = min(BN, cj - un.c0);
    const int64_t tile = (int64_t)i * P.N + j;

    double acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; x++)
#pragma unroll
      for (int y = 0; y < 4; y++) acc[x][y] = 0.0;

    ChunkIter it;  // the unit's positions in the tile's k-list (a piece of it under split k)
    it.t = un.t0;
    it.t_end = un.t1;
    it.kk0 = 0;
    it.k = it.t < it.t_end ? P.klist[it.t] : 0;
    it.qk = it.t < it.t_end ? P.q[it.k] : 0;
    // skip empty inner blocks
    while (it.t < it.t_end && it.qk == 0) {
      it.t++;
      if (it.t < it.t_end) {
        it.k = P.klist[it.t];
        it.qk = P.q[it.k];
      }
    }

    double ra[A_PER_T], rb[B_PER_T];
    auto load_chunk = [&](const ChunkIter& c) {
      // offsets of A_ik and B_kj; transposed storage indexes the tables (k,i) / (j,k)
      // and keeps every tile transposed (q_k x r_i, c_j x q_k)
      const int64_t ao = P.transa ? P.a_off[(int64_t)c.k * P.M + i] : P.a_off[(int64_t)i * P.K + c.k];
      const int64_t bo = P.transb ? P.b_off[(int64_t)j * P.K + c.k] : P.b_off[(int64_t)c.k * P.N + j];
      if (P.debug && tid == 0 && (ao < 0 || bo < 0)) atomicOr(a.err, kErrBadOffset);
      const double* At = P.A + (ao < 0 ? 0 : ao);
      const double* Bt = P.B + (bo < 0 ? 0 : bo);
      if (!P.transa) {
#pragma unroll
        for (int m = 0; m < A_PER_T; m++) {  // consecutive threads along k
          const int e = tid + NT * m;
          const int row = e / BK, kc = e % BK;
          const bool ok = ao >= 0 && row < rows && c.kk0 + kc < c.qk;
          ra[m] = ok ? __ldg(At + (int64_t)(un.r0 + row) * c.qk + c.kk0 + kc) : 0.0;
        }
      } else {
#pragma unroll
        for (int m = 0; m < A_PER_T; m++) {  // consecutive threads along the tile's rows
          const int e = tid + NT * m;
          const int row = e % BM, kc = e / BM;
          const bool ok = ao >= 0 && row < rows && c.kk0 + kc < c.qk;
          ra[m] = ok ? __ldg(At + (int64_t)(c.kk0 + kc) * ri + un.r0 + row) : 0.0;
        }
      }
      if (!P.transb) {
#pragma unroll
        for (int m = 0; m < B_PER_T; m++) {  // consecutive threads along the tile's columns
          const int e = tid + NT * m;
          const int kr = e / BN, cc = e % BN;
          const bool ok = bo >= 0 && cc < cols && c.kk0 + kr < c.qk;
          rb[m] = ok ? __ldg(Bt + (int64_t)(c.kk0 + kr) * cj + un.c0 + cc) : 0.0;
        }
      } else {
#pragma unroll
        for (int m = 0; m < B_PER_T; m++) {  // consecutive threads along k
          const int e = tid + NT * m;
          const int kr = e % BK, cc = e / BK;
          const bool ok = bo >= 0 && cc < cols && c.kk0 + kr < c.qk;
          rb[m] = ok ? __ldg(Bt + (int64_t)(un.c0 + cc) * c.qk + c.kk0 + kr) : 0.0;
        }
      }
    };
    auto advance = [&](ChunkIter& c) {
      c.kk0 += BK;
      while (c.t < c.t_end && c.kk0 >= c.qk) {
        c.t++;
        c.kk0 = 0;
        if (c.t < c.t_end) {
          c.k = P.klist[c.t];
          c.qk = P.q[c.k];
        }
      }
    };

    // register-tile rows and columns some lane of this warp needs: warp w holds ty in
    // [w*32/TX, (w+1)*32/TX), rows ty + TX*x, and every tx, columns tx + TX*y
    const int wty = (tid / 32) * (32 / TX);
    const int xm = rows > wty ? min(4, (rows - wty + TX - 1) / TX) : 0;
    const int ym = min(4, (cols + TX - 1) / TX);
    bool have = it.t < it.t_end;
    if (have) load_chunk(it);
    while (have) {
      const int kv = min(BK, it.qk - it.kk0);  // valid inner indices of the chunk being staged
      // staged as sA[kk][row], sB[kk][col] whichever order the loads took
      if (!P.transa) {
#pragma unroll
        for (int m = 0; m < A_PER_T; m++) {
          const int e = tid + NT * m;
          sA[e % BK][e / BK] = ra[m];
        }
      } else {
#pragma unroll
        for (int m = 0; m < A_PER_T; m++) {
          const int e = tid + NT * m;
          sA[e / BM][e % BM] = ra[m];
        }
      }
      if (!P.transb) {
#pragma unroll
        for (int m = 0; m < B_PER_T; m++) {
          const int e = tid + NT * m;
          sB[e / BN][e % BN] = rb[m];
        }
      } else {
#pragma unroll
        for (int m = 0; m < B_PER_T; m++) {
          const int e = tid + NT * m;
          sB[e % BK][e / BK] = rb[m];
        }
      }
      __syncthreads();
      advance(it);
      have = it.t < it.t_end;
      if (have) load_chunk(it);  // next chunk's loads overlap this chunk's FMAs
      switch (xm) {
        case 4: fma_chunk_y<4, BK, TX, BM + PAD, BN + PAD>(acc, sA, sB, ty, tx, kv, ym); break;
        case 3: fma_chunk_y<3, BK, TX, BM + PAD, BN + PAD>(acc, sA, sB, ty, tx, kv, ym); break;
        case 2: fma_chunk_y<2, BK, TX, BM + PAD, BN + PAD>(acc, sA, sB, ty, tx, kv, ym); break;
        case 1: fma_chunk_y<1, BK, TX, BM + PAD, BN + PAD>(acc, sA, sB, ty, tx, kv, ym); break;
        default: break;
      }
      __syncthreads();
    }

    // epilogue: C_ij = alpha*acc + beta*C_ij on the valid part of the region; a piece of a
    // split k-list stores its partial sum for the reduction instead
    const int64_t co = P.c_off[tile];
    if (un.slot >= 0) {
      double* dst = P.part + (int64_t)un.slot * (BM * BN);
#pragma unroll
      for (int x = 0; x < 4; x++) {
        const int row = ty + TX * x;
        if (row >= rows) continue;
#pragma unroll
        for (int y = 0; y < 4; y++) {
          const int col = tx + TX * y;
          if (col < cols) dst[row * BN + col] = acc[x][y];
        }
      }
    } else if (co < 0) {
      if (tid == 0) atomicOr(a.err, kErrBadOffset);
    } else {
      double* Ct = P.C + co + (int64_t)un.r0 * cj + un.c0;
#pragma unroll
      for (int x = 0; x < 4; x++) {
        const int row = ty + TX * x;
        if (row >= rows) continue;
#pragma unroll
        for (int y = 0; y < 4; y++) {
          const int col = tx + TX * y;
          if (col >= cols) continue;
          double* dst = Ct + (int64_t)row * cj + col;
          double v = __dmul_rn(P.alpha, acc[x][y]);
          if (P.beta != 0.0) v = __dadd_rn(v, __dmul_rn(P.beta, *dst));
          *dst = v;
        }
      }
    }
    if (a.timings) {
      __syncthreads();
      if (tid == 0) {
        a.timings[2 * (int64_t)u + 1] = gtimer() - t_unit;  // the unit's time
        a.unit_cta[u] = cta;
      }
    }
  }
}

// Split k: the reduction task of a region whose k-list was cut into pieces (Sec. 3.2,
// Fig. 2). The pieces' partial sums are added in piece order, each addition rounded to
// FP64, then C = alpha*sum + beta*C as in the tile kernel. One CTA per region.
__global__ void __launch_bounds__(256) fp64_reduce_kernel(const __grid_constant__ Fp64Args a) {
  const Fp64Red rd = a.red[blockIdx.x];
  const int T = a.tile;
  const int ri = a.r[rd.i], cj = a.c[rd.j];
  const int rows = min(T, ri - rd.r0), cols = min(T, cj - rd.c0);
  const int64_t tile = (int64_t)rd.i * a.N + rd.j;
  const int64_t co = a.c_off[tile];
  if (co < 0) {
    if (threadIdx.x == 0) atomicOr(a.err, kErrBadOffset);
    return;
  }
  double* Ct = a.C + co + (int64_t)rd.r0 * cj + rd.c0;
  const int64_t stride = (int64_t)T * T;
  const double* src = a.part + (int64_t)rd.slot0 * stride;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    const int row = e / T, col = e % T;
    if (row >= rows || col >= cols) continue;
    double v = src[e];
    for (int p = 1; p < rd.n; p++) v = __dadd_rn(v, src[p * stride + e]);
    double* dst = Ct + (int64_t)row * cj + col;
    double out = __dmul_rn(a.alpha, v);
    if (a.beta != 0.0) out = __dadd_rn(out, __dmul_rn(a.beta, *dst));
    *dst = out;
  }
}

// ---------------------------------------------------------------- rate diagnostics
// Arithmetic paths of the SM, each kept busy on every SM: DFMA (16 independent fused
// multiply-add chains per thread, so issue and not latency sets the rate), the FP64
// tensor-core instruction mma.sync m8n8k4 (4 independent accumulators per warp; 512 flops
// per instruction) and the INT8 one, mma.sync m16n8k32 s8 x s8 -> s32 (4 accumulators per
// warp; 8192 operations per instruction; sm_103a has no INT8 kind of tcgen05.mma, so this
// is the only INT8 tensor path). Every thread stores its accumulators' sum, so nothing is
// eliminated.
constexpr int kRateThreads = 256;
constexpr int kRateBlocksPerSm = 8;

__global__ void __launch_bounds__(kRateThreads) fp64_dfma_rate_kernel(double* out, int iters) {
  double x[16], b[16], c[16];  // every chain its own multiplier and addend
#pragma unroll
  for (int u = 0; u < 16; u++) {
    x[u] = (threadIdx.x + u) * 0x1p-20;
    b[u] = 1.0 + (u + 1) * 0x1p-40;
    c[u] = (u + 1) * 0x1p-60;
  }
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 16; u++) x[u] = fma(x[u], b[u], c[u]);
  }
  double sum = 0.0;
#pragma unroll
  for (int u = 0; u < 16; u++) sum += x[u];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

__global__ void __launch_bounds__(kRateThreads) fp64_dmma_rate_kernel(double* out, int iters) {
  const double a = 1.0 + threadIdx.x * 0x1p-30, b = 1.0 - 0x1p-40;
  double d[4][2];
#pragma unroll
  for (int u = 0; u < 4; u++) d[u][0] = d[u][1] = u * 0x1p-50;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 4; u++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(d[u][0]), "+d"(d[u][1])
                   : "d"(a), "d"(b));
  }
  double sum = 0.0;
#pragma unroll
  for (int u = 0; u < 4; u++) sum += d[u][0] + d[u][1];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

__global__ void __launch_bounds__(kRateThreads) imma_rate_kernel(double* out, int iters) {
  const uint32_t a = 0x01020304u + threadIdx.x, b = 0x05060708u;
  int32_t d[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) d[u][v] = u + v;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 4; u++)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+r"(d[u][0]), "+r"(d[u][1]), "+r"(d[u][2]), "+r"(d[u][3])
          : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
  }
  double sum = 0.0;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) sum += d[u][v];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

}  // namespace

cudaError_t unit_rates(double* rates, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * kRateBlocksPerSm;
  double* out = nullptr;
  e = cudaMalloc(&out, sizeof(double) * (size_t)blocks * kRateThreads);
  if (e != cudaSuccess) return e;
  constexpr int kReps = 3;  // timed passes of each kernel; the fastest counts
  cudaEvent_t ev[3 * kReps + 1] = {};
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  const int it_fma = 8192, it_mma = 2048, it_imma = 8192;
  if (e == cudaSuccess) {
    // one untimed pass of each (clocks up, code loaded), then the timed passes
    fp64_dfma_rate_kernel<<<blocks, kRateThreads, 0, st>>>(out, it_fma / 4);
    fp64_dmma_rate_kernel<<<blocks, kRateThreads, 0, st>>>(out, it_mma / 4);
    imma_rate_kernel<<<blocks, kRateThreads, 0, st>>>(out, it_imma / 4);
    cudaEventRecord(ev[0], st);
    for (int r = 0; r < kReps; r++) {
      fp64_dfma_rate_kernel<<<blocks, kRateThreads, 0, st>>>(out, it_fma);
      cudaEventRecord(ev[3 * r + 1], st);
      fp64_dmma_rate_kernel<<<blocks, kRateThreads, 0, st>>>(out, it_mma);
      cudaEventRecord(ev[3 * r + 2], st);
      imma_rate_kernel<<<blocks, kRateThreads, 0, st>>>(out, it_imma);
      cudaEventRecord(ev[3 * r + 3], st);
    }
    e = cudaGetLastError();
  }
  float best[3] = {0.0f, 0.0f, 0.0f};
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[3 * kReps]);
  for (int i = 0; i < 3 * kReps && e == cudaSuccess; i++) {
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
    if (best[i % 3] == 0.0f || t < best[i % 3]) best[i % 3] = t;
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double threads = (double)blocks * kRateThreads, warps = threads / 32.0;
  rates[0] = threads * 16.0 * it_fma * 2.0 / (best[0] * 1e-3) / 1e12;
  rates[1] = warps * 4.0 * it_mma * 512.0 / (best[1] * 1e-3) / 1e12;
  rates[2] = warps * 4.0 * it_imma * 8192.0 / (best[2] * 1e-3) / 1e12;
  return cudaSuccess;
}

int fp64_ctas_per_sm(int tile) {
  int n = 0;
  const cudaError_t e = tile == 32
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fp64_tile_kernel<32>, 64, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fp64_tile_kernel<64>, 256, 0);
  if (e != cudaSuccess || n < 1) n = 1;
  return n;
}

// One product's launch (a batch launches its products' reductions itself).
cudaError_t launch_fp64(const Fp64Args& a, int ctas, cudaStream_t st, cudaEvent_t* ev, int* nk) {
  if (ev) cudaEventRecord(ev[0], st);
  nvtxRangePushA("bsmm fp64: tile tasks");  // (a timeline tool's name for the phase)
  if (a.tile == 32)
    fp64_tile_kernel<32><<<ctas, 64, 0, st>>>(a);
  else
    fp64_tile_kernel<64><<<ctas, 256, 0, st>>>(a);
  nvtxRangePop();
  if (ev) cudaEventRecord(ev[1], st);
  int k = 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !a.prods && a.n_red > 0) {
    e = launch_fp64_reduce(a, st);
    if (ev) cudaEventRecord(ev[++k], st);
  }
  if (nk) *nk = k;
  return e;
}

cudaError_t launch_fp64_reduce(const Fp64Args& a, cudaStream_t st) {
  if (a.n_red <= 0) return cudaSuccess;
  fp64_reduce_kernel<<<a.n_red, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bsmm
