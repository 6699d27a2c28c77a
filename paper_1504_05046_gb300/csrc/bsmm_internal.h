// Internal declarations shared by the planner, the C ABI and the kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bsmm.h"

namespace bsmm {

// Device error word bits (set by kernels with atomicOr, read by bsmm_status_device).
enum : int32_t {
  kErrTimeout = 1,     // a bounded wait ran out
  kErrBadOffset = 2,   // debug check: a C tile of S_C without a C offset, or a bad A/B offset
  kErrNonFinite = 4,   // split modes: a non-finite input element
};

// Split-mode geometry.
constexpr int kSplitBM = 128;      // rows of one work unit (tcgen05 M)
constexpr int kSplitKC = 32;       // inner elements per staged chunk (64-byte swizzled rows)
constexpr int kSplitBeta = 7;      // bits per slice
constexpr int kSplitMaxS = 6;      // slices per operand
constexpr int kSplitEpiWarps = 8;  // epilogue warps (2 per TMEM lane quadrant)
constexpr int kSplitGuard = 55;    // guard bits of the 128-bit accumulator below the largest scale
constexpr double kEpiWalkBlocks = 32.0;  // mean k blocks per unit from which the epilogue walks
constexpr int kSplitMaxK = 8192;   // inner blocks per product
constexpr int64_t kSplitMaxInner = int64_t(1) << 22;  // inner elements per product (128-bit sums' headroom)

// FP64-mode geometry.
constexpr int kF64BK = 16;  // inner depth of one staged chunk (FP64 path)

// Deepest inner range (elements) over which every diagonal sum of slice products stays an
// integer of magnitude <= 2^24 (exact in the FP32 tensor-core accumulator); a deeper inner
// block is accumulated in several groups.
int split_max_depth(int s);
int split_tile_n(int s);          // work-unit width (32 or 64)
int split_stages(int s, int tn);  // smem ring depth
size_t split_smem_bytes(int s, int tn, int stages);
constexpr size_t kMaxSmemPerCta = 227 * 1024;  // opt-in dynamic shared memory of one CTA
constexpr size_t kSplitBarBytes = 512;          // mbarriers, TMEM slot, flags and group descriptors after the ring
constexpr int16_t kNonUniform = 0x7FFF;         // scale-class sentinel (offsets are <= 0)
constexpr int32_t kZeroLine = -(1 << 20);       // exponent of an all-zero row or column
int split_max_depth(int s);
constexpr int kSplitDefaultCluster = 1;  // groups of one: no CTA idles on a neighbour's empty column block
// Largest number of groups of `cl` contraction CTAs that can be resident at once (the
// kernel form with store warps when sw is set).
int split_max_clusters(int s, int cl, int stages, bool sw);

// Device arrays owned by a plan.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  bool borrowed = false;  // memory of another plan: not freed with this one
};

// Work units. A unit covers a region of C over a range of its k-list: the whole list,
// or one piece of it when the planner splits k (Sec. 3.2, Fig. 2: multiply tasks on
// parts of the k-list, then a reduction task). A piece writes its partial sum to the
// plan's partial workspace at `slot` instead of finishing the region; a reduction unit
// then adds the region's partials in slot order and applies the epilogue.
struct Fp64Unit {  // one sub-tile of one C tile, k-list positions [t0, t1)
  int32_t i, j, r0, c0;
  int64_t t0, t1;
  int32_t slot;  // -1: the unit finishes its region
  int32_t pad;
};

struct SplitUnit {  // one (128-row block, group of cl TN-column blocks), inner blocks [k0, k1)
  int32_t rb, cb;
  int32_t k0, k1;
  int32_t slot;  // -1: the unit finishes its region; else the partial-sum slot of this piece
  int32_t own;   // bit r: the group's r-th column block has a B tile at some k of [k0, k1)
                 // where the row block has an A tile (that CTA's list is not empty)
};

struct Fp64Red {  // a region whose k-list was split: partial slots [slot0, slot0 + n)
  int32_t i, j, r0, c0, slot0, n;
};

struct SplitRed {  // a (row block, column-block group) whose k-list was split
  int32_t rb, cb, slot0, n;
};

// Arguments of the FP64 tile-task kernel.
struct Fp64Args {
  const int32_t* r;
  const int32_t* c;
  const int32_t* q;
  int32_t M, N, K;
  const int64_t* kptr;     // CSR over M*N tiles
  const int32_t* klist;    // ascending k per tile
  const uint8_t* cs;       // S_C, M*N
  const Fp64Unit* units;
  const int32_t* sched_ptr;
  const int32_t* sched_units;
  double alpha, beta;
  const double* A;
  const int64_t* a_off;
  const double* B;
  const int64_t* b_off;
  double* C;
  const int64_t* c_off;
  int64_t* timings;        // 2 per unit or null
  int32_t* unit_cta;       // per unit or null
  int32_t* err;
  int32_t debug;
  int32_t tile;            // sub-tile edge of the units (64 or 32)
  int32_t transa, transb;  // transposed operand storage (bsmm_options)
  double* part;            // split k: tile x tile partial sums per slot (row-major)
  const Fp64Red* red;      // split k: the regions to reduce
  int32_t n_red;
  // batch: per-product arguments in device memory; the schedule then lists batch-wide
  // unit ids, each mapped to (product, unit of that product)
  const Fp64Args* prods;
  const int32_t* unit_prod;
  const int32_t* unit_local;
};

// Arguments of the split-mode kernels.
struct SplitArgs {
  int32_t M, N, K, s, tn, stages, fp16;
  int32_t cl, CBG;          // CTAs per column-block group; groups (units are (rb, group))
  int32_t sw;               // the contraction kernel's form: 1 = with C store warps
  int32_t deep;             // 1: some inner block is deeper than kdepth (the kernel's DEEP form)
  int32_t epi_walk;         // 1: the epilogue finds the accumulation groups on its own k list
                            // (long lists); 0: it takes them from the MMA warps' descriptors
  int64_t Mtot, Ntot;
  int32_t RB, CB, kwords;
  const int32_t* r;
  const int32_t* c;
  const int32_t* q;
  const int64_t* ro;        // row prefix offsets (M+1)
  const int64_t* co;        // col prefix offsets (N+1)
  const int32_t* row_tile;  // Mtot
  const int32_t* col_tile;  // Ntot
  const uint8_t* cs;        // S_C
  const uint8_t* am;        // A tile mask (M x K)
  const uint8_t* bm;        // B tile mask (K x N)
  const uint64_t* presA;    // RB x kwords
  const uint64_t* presB;    // CB x kwords
  const uint64_t* presBg;   // CBG x kwords: union over the cl column blocks of a group
  const int64_t* apk_off;   // RB x K byte offsets into apk (-1 absent)
  const int64_t* bpk_off;   // K x CB byte offsets into bpk (-1 absent)
  uint8_t* apk;
  uint8_t* bpk;
  int16_t* rowexp;          // K x Mtot: e_A(i,k) - Emax_A(i) per row (0 for absent tiles)
  int16_t* colexp;          // K x colexp_ld: e_B(k,j) - Emax_B(j) per column
  int64_t colexp_ld;        // row stride of colexp (Ntot rounded up to 64)
  // Scale classes for merging k blocks into one TMEM accumulation: urow[k*RB+rb] is the
  // common rowexp of the present rows of row block rb at k block k, ucol[k*CB+cb] the
  // common colexp of the present columns of column block cb (kNonUniform when they
  // differ); null: every k block is drained on its own.
  int16_t* urow;
  int16_t* ucol;
  // the row's and the column's part of a merged group's binary position (Mtot; padded like
  // a colexp row): the largest Emax of the row block (column block) minus the line's Emax
  int16_t* rowadj;
  int16_t* coladj;
  // every row's and column's largest exponent (Emax_A of the row, Emax_B of the column;
  // Mtot, and padded like a colexp row), the parts of the accumulator unit 2^L
  int32_t* emaxr;
  int32_t* emaxc;
  int32_t kdepth;           // deepest exact FP32 accumulation (inner elements) for s slices
  int32_t transa, transb;   // transposed operand storage (bsmm_options)
  // per-row / per-column scaling (split_scale = 1): exponents of every row of every A tile
  // (K x Mtot) and column of every B tile (K x Ntot; kZeroLine for an all-zero line), and
  // the row / column maxima that set the accumulator unit (Mtot, Ntot)
  int32_t rowscale;
  int32_t* eArow;
  int32_t* eBcol;
  int32_t* eAmaxr;
  int32_t* eBmaxc;
  int32_t* eAmax;           // M: largest exponent of the stored A tiles of a row block
  int32_t* eBmax;           // N
  int32_t* eA;              // M x K
  int32_t* eB;              // K x N
  const int32_t* a_tiles;   // present A tiles (i*K+k), count n_a_tiles
  const int32_t* b_tiles;   // present B tiles (k*N+j)
  int32_t n_a_tiles, n_b_tiles;
  const int32_t* a_blocks;  // present (rb*K+kt)
  const int32_t* b_blocks;  // present (kt*CB+cb)
  int32_t n_a_blocks, n_b_blocks;
  const SplitUnit* units;
  const int32_t* sched_ptr;
  const int32_t* sched_units;
  double alpha, beta;
  const double* A;
  const int64_t* a_off;
  const double* B;
  const int64_t* b_off;
  double* C;
  const int64_t* c_off;
  int64_t* timings;
  int32_t* unit_cta;
  int32_t* err;
  int32_t debug;
  // float32 elements (bsmm_options.elem): A, B and C are the float arrays below instead
  // of the double ones; offsets count float elements
  int32_t f32;
  // complex elements: A, B, C are interleaved (re, im) double arenas and offsets count
  // complex elements; the plan's inner and column tilings are doubled (the real product
  // [Ar, -Ai] x [[Br, Bi], [Bi, -Br]]), so the tiles' complex sizes are half of q and c
  int32_t cplx;
  const float* Af;
  const float* Bf;
  float* Cf;
  // split k: exact 128-bit partial sums, per slot and cluster rank a TN x 128 array
  // (column-major: element (row, col) at col * 128 + row), and the regions to reduce
  uint4* part;
  const SplitRed* red;
  int32_t n_red;
  // batch (see Fp64Args)
  const SplitArgs* prods;
  const int32_t* unit_prod;
  const int32_t* unit_local;
};

// ev: null, or kMaxEvents events; ev[0] is recorded before the first kernel and
// ev[i+1] after kernel i. *nk receives the number of kernels launched.
constexpr int kMaxEvents = 8;
constexpr int kProfileRing = 64;  // executes whose per-kernel times a plan keeps
cudaError_t launch_fp64(const Fp64Args& a, int ctas, cudaStream_t st, cudaEvent_t* ev, int* nk);
cudaError_t launch_split(const SplitArgs& a, int ctas, cudaStream_t st, cudaEvent_t* ev, int* nk);
// the two halves of launch_split: per-product exponents, scales and slices; the
// persistent contraction over the schedule in `a` (clusters of a.cl CTAs)
cudaError_t launch_split_prep(const SplitArgs& a, cudaStream_t st, cudaEvent_t* ev, int* k);
int split_prep_kernels(const SplitArgs& a);  // how many kernels launch_split_prep launches
cudaError_t launch_split_mma(const SplitArgs& a, int clusters, cudaStream_t st);
// split k: the reductions of the regions whose k-list was split (no launch when none)
cudaError_t launch_split_reduce(const SplitArgs& a, cudaStream_t st);
// a kernel whose bounded waits can never be satisfied (see bsmm_selftest_wait)
cudaError_t launch_wait_selftest(int32_t* err, int64_t limit_ns, cudaStream_t st);
cudaError_t launch_fp64_reduce(const Fp64Args& a, cudaStream_t st);

// Longest-processing-time packing of n units with `cost` onto `bins` persistent CTAs
// (or clusters); natural = round robin in unit order. CSR output.
void lpt_pack(const std::vector<double>& cost, int bins, bool natural, std::vector<int32_t>& ptr,
              std::vector<int32_t>& units, const std::vector<int64_t>* segments = nullptr);
void wave_segments(int64_t u0, int64_t u1, int bins, std::vector<int64_t>& seg);
// Kernel arguments of one product (device pointers from the caller).
void fill_fp64_args(bsmm_plan_s* p, Fp64Args& a, double alpha, const double* A, const int64_t* a_off,
                    const double* B, const int64_t* b_off, double beta, double* C, const int64_t* c_off);
// (A, B, C are double arrays, or float arrays for a plan with float32 elements)
void fill_split_args(bsmm_plan_s* p, SplitArgs& a, double alpha, const void* A, const int64_t* a_off,
                     const void* B, const int64_t* b_off, double beta, void* C, const int64_t* c_off);
int default_bins(const bsmm_plan_s* p);
// Persistent CTAs (FP64) or clusters (split modes) of the machine, capped by max_ctas but
// not by the unit count.
int machine_bins(const bsmm_plan_s* p);
// Split k: pieces per unit from the units' costs, k-list lengths and the bin count.
std::vector<int32_t> choose_pieces(const std::vector<double>& cost, const std::vector<int64_t>& len, int bins,
                                   double overhead, int ksplit);
int fp64_ctas_per_sm(int tile);
// measured rates of this GPU: rates[0] DFMA, rates[1] FP64 mma.sync (TFLOP/s), rates[2]
// INT8 mma.sync (TOP/s); synchronises `st`
cudaError_t unit_rates(double* rates, cudaStream_t st);

void set_error(const std::string& msg);
// waits for the plan's host-buffer products and frees their staging slots, streams, events
void host_release(bsmm_plan_s* p);

// bsmm_plan with an optional donor: a split plan of the same structure and slice count
// whose slice workspace the new plan shares instead of allocating its own (the packed
// layout does not depend on the cluster size or the ring depth).
bsmm_status plan_build(bsmm_plan_t* out, int32_t M, const int32_t* row_sizes, int32_t N, const int32_t* col_sizes,
                       int32_t K, const int32_t* inner_sizes, const uint8_t* a_mask, const uint8_t* b_mask,
                       const uint8_t* c_mask, const bsmm_options* opt, const bsmm_plan_s* donor);

}  // namespace bsmm

// The plan object behind bsmm_plan_t.
struct bsmm_plan_s {
  int32_t M = 0, N = 0, K = 0;
  std::vector<int32_t> r, c, q;
  std::vector<int64_t> ro, co, qo;
  std::vector<uint8_t> am, bm, cs;
  int64_t n_ctiles = 0, n_triples = 0;
  double useful_flops = 0.0;
  bsmm_options opt{};
  int device = 0, sms = 0;

  // work units (one kind per mode)
  std::vector<bsmm::Fp64Unit> f64_units;
  int f64_tile = 64;           // FP64 sub-tile edge (64 or 32)
  std::vector<bsmm::SplitUnit> sp_units;
  std::vector<int64_t> kptr;   // FP64: CSR over M*N tiles
  std::vector<int32_t> klist;
  int64_t n_units = 0;
  // split k: regions cut into pieces and their partial slots
  std::vector<bsmm::Fp64Red> f64_red;
  std::vector<bsmm::SplitRed> sp_red;
  std::vector<int32_t> unit_pieces;  // per unit: pieces of its region (1: not split)
  int64_t n_slots = 0;
  std::vector<double> flop_cost, cost;
  std::vector<float> features;  // n_units x BSMM_NFEATURES
  int ctas = 0;
  std::vector<int32_t> sched_ptr, sched_units;

  // split geometry
  int s = 0, tn = 0, stages = 0, RB = 0, CB = 0, kwords = 0, cl = 1, CBG = 0;
  int sw = 0;                // contraction kernel with C store warps
  int epi_walk = 0;          // the epilogue walks the k lists itself (SplitArgs::epi_walk)
  int deep = 0;              // some inner block is deeper than the exact FP32 depth
  int64_t Mtot = 0, Ntot = 0, colexp_ld = 0;
  int64_t apk_bytes = 0, bpk_bytes = 0;

  // device memory
  bsmm::DevBuf d_r, d_c, d_q, d_ro, d_co, d_kptr, d_klist, d_cs, d_units, d_sched_ptr, d_sched_units;
  bsmm::DevBuf d_row_tile, d_col_tile, d_presA, d_presB, d_presBg, d_apk_off, d_bpk_off, d_apk, d_bpk;
  bsmm::DevBuf d_eArow, d_eBcol, d_eAmaxr, d_eBmaxc;
  bsmm::DevBuf d_rowadj, d_coladj, d_emaxr, d_emaxc;
  bsmm::DevBuf d_am, d_bm, d_rowexp, d_colexp, d_urow, d_ucol, d_eA, d_eB, d_eAmax, d_eBmax, d_a_tiles, d_b_tiles, d_a_blocks, d_b_blocks;
  bsmm::DevBuf d_err, d_timings, d_unit_cta, d_part, d_red;
  int32_t n_a_tiles = 0, n_b_tiles = 0, n_a_blocks = 0, n_b_blocks = 0;

  // per-kernel profiling events (profile option): a ring of event sets, one set per
  // execute; bsmm_plan_kernel_ms averages the sets recorded since its previous call
  cudaEvent_t ev[bsmm::kProfileRing][bsmm::kMaxEvents] = {};
  int ev_counts[bsmm::kProfileRing] = {};
  int ev_next = 0;     // the set the next execute records into
  int ev_pending = 0;  // sets recorded since the last bsmm_plan_kernel_ms (at most the ring)
  int ev_last = -1;    // the set of the last execute

  // a plan whose slice workspace (d_apk, d_bpk) this one shares, or null
  const bsmm_plan_s* donor = nullptr;
  int32_t cost_source = BSMM_COSTS_FLOPS;  // where `cost` came from (bsmm_cost_source)
  uint64_t uid = 0;  // unique over the process's plans (never reused, unlike an address)

  // Host-buffer executes: two device staging slots (grown on demand), so that the copies
  // of one product run while the product before it computes (several iterations in
  // flight, Sec. 3.2). Slot i % 2 takes the i-th product; its events mark where that
  // product's copies in, contraction and copy out end.
  struct HostSlot {
    bsmm::DevBuf A, B, C, aoff, boff, coff;
    cudaEvent_t in = nullptr, run = nullptr, out = nullptr;
    bool used = false;
  } hs[2];
  cudaStream_t h2d = nullptr, d2h = nullptr;  // copy streams (created on first use)
  cudaEvent_t last_run = nullptr;             // the last host product's kernels (workspace order)
  int64_t host_count = 0;                     // host-buffer products enqueued so far
};
