// Allocation-free split-precision tile task.
//
// Some callers cannot allocate device memory at the point where they need the
// product: code running while a memory pool is locked or a CUDA graph is being
// built around it, allocators that forbid cudaMalloc on their hot path, or hosts
// whose device memory is fully reserved up front. For them, bsmm_split_tile_noalloc
// runs one dense tile task C = alpha*A*B + beta*C with the split-precision method
// of bsmm_execute (same exponents, slices, tensor-core contraction and exact
// recombination, so the same bits) using only the caller's A, B and C and a
// file-scope device array below as its scratch: the packed slices, the exponent
// tables and the small task tables. It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// Limits (checked before any launch; BSMM_ERR_INVALID otherwise): 0 <= m, n <= 256,
// 0 <= k <= 512, 1 <= nslices <= 6. k = 512 is within the exact FP32 accumulation depth
// of every slice count (split_max_depth(s) >= 512 for s <= 6), so no inner depth is
// refused beyond that. k = 0 gives C = beta*C (alpha times an empty sum).
// The scratch array is kNoallocScratchBytes (about 3.2 MB); every GPU that loads the
// library holds it until the process exits.
//
// Set-up: every call, with the target device current, looks up the array's device
// address on that device with cudaGetSymbolAddress (the host-side name of the array is
// not a device address); the first call on a device loads the library's module there
// and should come before any stream capture. Every call reuses the same array and
// leaves the last call's contents in it (the set-up kernel rewrites every entry the
// product reads and clears the error word), so calls that overlap on the GPU -- on
// different streams, or from several host threads -- race and must be serialised by
// the caller. The call reads the error word back from the array on `stream` and
// returns once the product is complete.
#include <cstddef>
#include <cstdint>
#include <cstring>

#include "bsmm_internal.h"

namespace bsmm {

namespace {

constexpr int kNaMaxM = 256, kNaMaxN = 256, kNaMaxK = 512;
constexpr int kNaRB = (kNaMaxM + kSplitBM - 1) / kSplitBM;  // 2 row blocks
constexpr int kNaCB = kNaMaxN / 32;                          // 8 column blocks
constexpr int kNaKC = kNaMaxK / kSplitKC;                    // 16 chunks
constexpr size_t kNaApk = (size_t)kNaRB * kNaKC * kSplitMaxS * kSplitBM * kSplitKC * 2;
constexpr size_t kNaBpk = (size_t)kNaCB * kNaKC * kSplitMaxS * 32 * kSplitKC * 2;
constexpr int kNaColLd = kNaMaxN + 64 + 64;
constexpr int kNaUnits = kNaRB * kNaCB;

// layout of the scratch array (byte offsets, each 256-byte aligned)
struct NaLayout {
  static constexpr size_t apk = 0;
  static constexpr size_t bpk = apk + kNaApk;
  static constexpr size_t tables = bpk + kNaBpk;
};

// task tables of a 1 x 1 x 1 tiling, written on the device by noalloc_setup_kernel
struct NaTables {
  int32_t r[1], c[1], q[1];
  int64_t ro[2], co[2];
  int32_t row_tile[kNaMaxM], col_tile[kNaMaxN];
  uint8_t cs[4], am[4], bm[4];
  uint64_t presA[kNaRB], presB[kNaCB];
  int64_t apk_off[kNaRB], bpk_off[kNaCB];
  alignas(16) int16_t rowexp[kNaMaxM + 64];
  alignas(16) int16_t colexp[kNaColLd + 64];
  alignas(16) int32_t emaxr[kNaMaxM];
  alignas(16) int32_t emaxc[kNaColLd + 64];
  int32_t eA[1], eB[1], eAmax[1], eBmax[1];
  int32_t a_tiles[1], b_tiles[1];
  int32_t a_blocks[kNaRB], b_blocks[kNaCB];
  SplitUnit units[kNaUnits];
  int32_t sched_ptr[kNaUnits + 1], sched_units[kNaUnits];
  int64_t a_off[1], b_off[1], c_off[1];
  int32_t err[4];
};

constexpr size_t kNoallocScratchBytes = NaLayout::tables + ((sizeof(NaTables) + 255) / 256) * 256;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocScratchBytes];

__global__ void noalloc_setup_kernel(uint8_t* base, int m, int n, int k, int s, int RB, int CB, int nkc) {
  NaTables* t = reinterpret_cast<NaTables*>(base + NaLayout::tables);
  const int tid = threadIdx.x;
  for (int i = tid; i < kNaMaxM; i += blockDim.x) t->row_tile[i] = 0;
  for (int i = tid; i < kNaMaxN; i += blockDim.x) t->col_tile[i] = 0;
  for (int i = tid; i < kNaMaxM + 64; i += blockDim.x) t->rowexp[i] = 0;
  for (int i = tid; i < kNaColLd + 64; i += blockDim.x) t->colexp[i] = 0;
  for (int i = tid; i < kNaMaxM; i += blockDim.x) t->emaxr[i] = 0;
  for (int i = tid; i < kNaColLd + 64; i += blockDim.x) t->emaxc[i] = 0;
  if (tid == 0) {
    t->r[0] = m;
    t->c[0] = n;
    t->q[0] = k;
    t->ro[0] = 0;
    t->ro[1] = m;
    t->co[0] = 0;
    t->co[1] = n;
    t->cs[0] = t->am[0] = t->bm[0] = 1;
    const int64_t achunk = (int64_t)s * kSplitBM * kSplitKC * 2;
    const int64_t bchunk = (int64_t)s * 32 * kSplitKC * 2;
    for (int rb = 0; rb < RB; rb++) {
      t->presA[rb] = k > 0 ? 1ull : 0ull;  // an empty inner block holds no stored tile
      t->apk_off[rb] = rb * nkc * achunk;
      t->a_blocks[rb] = rb;  // rb * K + kt with K = 1, kt = 0
    }
    for (int cb = 0; cb < CB; cb++) {
      t->presB[cb] = 1ull;
      t->bpk_off[cb] = cb * nkc * bchunk;
      t->b_blocks[cb] = cb;  // kt * CB + cb with kt = 0
    }
    t->a_tiles[0] = 0;
    t->b_tiles[0] = 0;
    int u = 0;
    for (int rb = 0; rb < RB; rb++)
      for (int cb = 0; cb < CB; cb++) {
        t->units[u] = SplitUnit{rb, cb, 0, 1, -1, k > 0 ? 1 : 0};  // the one inner block, whole
        t->sched_ptr[u] = u;
        t->sched_units[u] = u;
        u++;
      }
    t->sched_ptr[u] = u;
    t->a_off[0] = t->b_off[0] = t->c_off[0] = 0;
    t->err[0] = 0;
  }
}

}  // namespace

}  // namespace bsmm

using namespace bsmm;

extern "C" bsmm_status bsmm_split_tile_noalloc(int32_t m, int32_t n, int32_t k, int32_t nslices, double alpha,
                                               const double* A, const double* B, double beta, double* C,
                                               void* stream) {
  if (m < 0 || n < 0 || k < 0 || m > kNaMaxM || n > kNaMaxN || k > kNaMaxK || nslices < 1 ||
      nslices > kSplitMaxS)
    return set_error("bsmm_split_tile_noalloc: sizes must satisfy 0 <= m, n <= 256, 0 <= k <= 512 and "
                     "nslices in 1..6"),
           BSMM_ERR_INVALID;
  if (m == 0 || n == 0) return BSMM_OK;
  if (!C || (k > 0 && (!A || !B))) return set_error("bsmm_split_tile_noalloc: NULL operand"), BSMM_ERR_INVALID;
  if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 15)
    return set_error("bsmm_split_tile_noalloc: operands must be 16-byte aligned"), BSMM_ERR_INVALID;

  // the array's address on the current device (the host-side symbol is only a handle)
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return set_error(std::string("bsmm_split_tile_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e)),
           BSMM_ERR_CUDA;
  uint8_t* base = (uint8_t*)p;
  cudaStream_t st = (cudaStream_t)stream;
  const int s = nslices;
  const int RB = (m + kSplitBM - 1) / kSplitBM;
  const int CB = (n + 31) / 32;
  const int nkc = (k + kSplitKC - 1) / kSplitKC;
  noalloc_setup_kernel<<<1, 256, 0, st>>>(base, m, n, k, s, RB, CB, nkc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(std::string("noalloc setup: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;

  NaTables* t = reinterpret_cast<NaTables*>(base + NaLayout::tables);
  SplitArgs a{};
  a.M = a.N = a.K = 1;
  a.s = s;
  a.tn = 32;
  a.stages = split_stages(s, 32);
  a.fp16 = 0;
  a.Mtot = m;
  a.Ntot = n;
  a.RB = RB;
  a.CB = CB;
  a.kwords = 1;
  a.r = t->r;
  a.c = t->c;
  a.q = t->q;
  a.ro = t->ro;
  a.co = t->co;
  a.row_tile = t->row_tile;
  a.col_tile = t->col_tile;
  a.cs = t->cs;
  a.am = t->am;
  a.bm = t->bm;
  a.presA = t->presA;
  a.presB = t->presB;
  a.presBg = t->presB;  // clusters of one CTA: a column-block group is one column block
  a.cl = 1;
  a.sw = 0;  // the kernel form without store warps
  a.epi_walk = 0;  // one short k list: the MMA warps' descriptors
  a.deep = 0;      // k <= 512: within the exact depth of every slice count
  a.kdepth = split_max_depth(nslices);
  a.CBG = CB;
  a.apk_off = t->apk_off;
  a.bpk_off = t->bpk_off;
  a.apk = base + NaLayout::apk;
  a.bpk = base + NaLayout::bpk;
  a.rowexp = t->rowexp;
  a.colexp = t->colexp;
  a.colexp_ld = kNaColLd;
  a.emaxr = t->emaxr;
  a.emaxc = t->emaxc;
  a.eA = t->eA;
  a.eB = t->eB;
  a.eAmax = t->eAmax;
  a.eBmax = t->eBmax;
  a.a_tiles = t->a_tiles;
  a.b_tiles = t->b_tiles;
  a.n_a_tiles = k > 0 ? 1 : 0;
  a.n_b_tiles = k > 0 ? 1 : 0;
  a.a_blocks = t->a_blocks;
  a.b_blocks = t->b_blocks;
  a.n_a_blocks = k > 0 ? RB : 0;
  a.n_b_blocks = k > 0 ? CB : 0;
  a.units = t->units;
  a.sched_ptr = t->sched_ptr;
  a.sched_units = t->sched_units;
  a.alpha = alpha;
  a.beta = beta;
  a.A = A;
  a.a_off = t->a_off;
  a.B = B;
  a.b_off = t->b_off;
  a.C = C;
  a.c_off = t->c_off;
  a.timings = nullptr;
  a.unit_cta = nullptr;
  a.err = t->err;
  a.debug = 0;
  a.part = nullptr;  // no split k: one inner block
  a.red = nullptr;
  a.n_red = 0;
  e = launch_split(a, RB * CB, st, nullptr, nullptr);
  if (e != cudaSuccess) return set_error(std::string("noalloc launch: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  // the device error word, read back from the array itself (no buffer of the caller's)
  int32_t w = 0;
  e = cudaMemcpyFromSymbolAsync(&w, g_noalloc_scratch, sizeof(int32_t), NaLayout::tables + offsetof(NaTables, err),
                                cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(std::string("noalloc status: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  if (w & kErrTimeout) return set_error("bsmm_split_tile_noalloc: a kernel wait timed out"), BSMM_ERR_TIMEOUT;
  if (w & kErrNonFinite)
    return set_error("bsmm_split_tile_noalloc: non-finite input element"), BSMM_ERR_DEVICE;
  if (w) return set_error("bsmm_split_tile_noalloc: device error word set"), BSMM_ERR_DEVICE;
  return BSMM_OK;
}
