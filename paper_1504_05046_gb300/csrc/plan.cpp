// Host planner and C ABI of the block-sparse product.
//
// The planner turns the three tilings and two tile masks into the data-driven
// task set of the paper's task-based SUMMA (Sec. 3.2): the C tile set S_C (the
// boolean product of the masks), one task per C tile region with its ascending
// k order (the rank-k updates of Sec. 2.1, each owned by one CTA so that the
// multiply and the reduction into C are fused, Sec. 3.2 last paragraphs), the
// useful flop count, and a packing of the tasks onto persistent CTAs
// (longest-processing-time first onto the least-loaded CTA) that replaces the
// paper's process grid and task queue on one GPU. Where the grid would idle, a
// region's k-list is cut into pieces with a reduction task (split k, Sec. 3.2, Fig. 2).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>

#include "bsmm_internal.h"

using namespace bsmm;

namespace bsmm {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int split_max_depth(int s) {
  // |S_d| <= q * 2^(2*beta-2) * max(4, d+1) with d <= s+1 (slice bounds |N_1| <= 2^beta,
  // |N_t| <= 2^(beta-1)); require that to be <= 2^24.
  const double per = std::ldexp(1.0, 2 * kSplitBeta - 2) * std::max(4, s + 2);
  return (int)std::floor(std::ldexp(1.0, 24) / per);
}

// 32 columns per unit: 16 per epilogue thread keeps the 128-bit accumulators in registers,
// and two TMEM buffers of s*32 columns fit the 512 columns for every s <= 6.
int split_tile_n(int) { return 32; }

static size_t stage_bytes(int s, int tn) {
  return (size_t)s * (kSplitBM * kSplitKC * 2) + (size_t)s * (tn * kSplitKC * 2);
}

// the deepest ring (at most 8 stages) that fits one CTA's shared memory
int split_stages(int s, int tn) {
  int st = 8;
  while (st > 2 && split_smem_bytes(s, tn, st) > kMaxSmemPerCta) st--;
  return st;
}

size_t split_smem_bytes(int s, int tn, int stages) {
  return 1024 /*alignment slack*/ + (size_t)stages * stage_bytes(s, tn) + kSplitBarBytes +
         (size_t)kSplitBM * (tn + 1) * sizeof(double) /*C staging*/;
}

// Longest processing time first: units by descending cost (ties keep unit order), each
// to the least-loaded bin (ties to the lowest bin). A bin then runs its units in unit
// order: the bins' loads are set by the assignment alone, and walking every list in
// the planner's raster order keeps the units that run at the same time close in the
// index space, so their A and B panels are shared through L2.
void lpt_pack(const std::vector<double>& cost, int bins, bool natural, std::vector<int32_t>& ptr,
              std::vector<int32_t>& units, const std::vector<int64_t>* segments) {
  const int64_t n = (int64_t)cost.size();
  std::vector<std::vector<int32_t>> lists(bins);
  if (natural) {
    for (int64_t u = 0; u < n; u++) lists[u % bins].push_back((int32_t)u);
  } else {
    // segments (the products of a batch) are packed one after the other, the bins
    // carrying their loads over, so every bin runs its share of segment 0, then of
    // segment 1, ...: the bins move through the segments together and the panels they
    // read at any time belong to one or two products (shared in L2)
    std::vector<int64_t> seg = segments ? *segments : std::vector<int64_t>{0, n};
    using E = std::pair<double, int>;  // (load, bin), smallest first
    std::priority_queue<E, std::vector<E>, std::greater<E>> heap;
    for (int t = 0; t < bins; t++) heap.push({0.0, t});
    for (size_t g = 0; g + 1 < seg.size(); g++) {
      std::vector<int64_t> order(seg[g + 1] - seg[g]);
      std::iota(order.begin(), order.end(), seg[g]);
      std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
      for (int64_t u : order) {
        E e = heap.top();
        heap.pop();
        lists[e.second].push_back((int32_t)u);
        heap.push({e.first + cost[u], e.second});
      }
    }
    for (auto& l : lists) std::sort(l.begin(), l.end());
  }
  ptr.assign(bins + 1, 0);
  units.clear();
  units.reserve(n);
  for (int t = 0; t < bins; t++) {
    ptr[t] = (int32_t)units.size();
    for (int32_t u : lists[t]) units.push_back(u);
  }
  ptr[bins] = (int32_t)units.size();
}

// Units [u0, u1) in waves of `bins` consecutive units (segment starts, then u1): packed
// wave by wave, every bin's i-th unit comes from wave i, so the bins walk the raster
// order together and the units that run at the same time share their panels in L2
// (one LPT pass over all units would let costlier bins fall behind in unit order).
// With fewer than kWaveMinUnits units per bin the range stays one segment: one LPT pass
// over few units balances the bins much better than wave-by-wave packing, and the waves'
// locality gain needs many units per bin to show.
constexpr int64_t kWaveMinUnits = 16;
void wave_segments(int64_t u0, int64_t u1, int bins, std::vector<int64_t>& seg) {
  if (seg.empty() || seg.back() != u0) seg.push_back(u0);
  if (u1 - u0 >= kWaveMinUnits * bins)
    for (int64_t u = u0 + bins; u < u1; u += bins) seg.push_back(u);
  if (u1 > u0) seg.push_back(u1);
}

// FP64: persistent CTAs; split modes: persistent groups of p->cl CTAs.
int machine_bins(const bsmm_plan_s* p) {
  int64_t c;
  if (p->opt.mode == BSMM_FP64)
    c = (int64_t)p->sms * std::max(1, fp64_ctas_per_sm(p->f64_tile));
  else
    c = std::max(1, split_max_clusters(p->s, p->cl, p->stages, p->sw != 0));
  if (p->opt.max_ctas > 0) c = std::min<int64_t>(c, p->opt.max_ctas);
  return (int)std::max<int64_t>(1, c);
}

int default_bins(const bsmm_plan_s* p) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(machine_bins(p), std::max<int64_t>(1, p->n_units)));
}

// Split k (Sec. 3.2, Fig. 2). The paper cuts the dependency between the rank-k updates
// of one C tile by running each update as a multiply task into a temporary and adding
// the temporaries in a separate task. Here a region's k-list is cut into a few
// consecutive pieces only when that lets the persistent grid fill: a piece costs its
// share of the region's work plus a fixed overhead (pipeline start and drain, the
// partial sum's store and its reduction), and the longest-processing-time packing of
// the pieces is simulated for several granularities.
static double lpt_makespan(const std::vector<double>& cost, const std::vector<int32_t>& n, int bins, double overhead) {
  std::vector<double> pc;
  for (size_t u = 0; u < cost.size(); u++)
    for (int32_t k = 0; k < n[u]; k++) pc.push_back(cost[u] / n[u] + (n[u] > 1 ? overhead : 0.0));
  std::sort(pc.begin(), pc.end(), std::greater<double>());
  std::priority_queue<double, std::vector<double>, std::greater<double>> heap;
  for (int b = 0; b < bins; b++) heap.push(0.0);
  double mk = 0.0;
  for (double c : pc) {
    double l = heap.top() + c;
    heap.pop();
    mk = std::max(mk, l);
    heap.push(l);
  }
  return mk;
}

// Pieces per unit. Forced (ksplit >= 2): min(ksplit, len) for every unit. Automatic
// (ksplit == 0): target piece costs total / (bins * g) for g in kGran give every unit
// clamp(ceil(cost / target), 1, len) pieces; the candidate with the shortest simulated
// makespan is taken if it is at least 10% shorter than the unsplit one.
std::vector<int32_t> choose_pieces(const std::vector<double>& cost, const std::vector<int64_t>& len, int bins,
                                   double overhead, int ksplit) {
  const size_t n = cost.size();
  std::vector<int32_t> one(n, 1);
  if (ksplit == 1 || n == 0) return one;
  if (ksplit >= 2) {
    for (size_t u = 0; u < n; u++) one[u] = (int32_t)std::max<int64_t>(1, std::min<int64_t>(ksplit, len[u]));
    return one;
  }
  constexpr int kGran[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
  double total = 0.0, mx = 0.0;
  for (size_t u = 0; u < n; u++) {
    total += cost[u];
    mx = std::max(mx, cost[u]);
  }
  const double avg = total / std::max(1, bins);
  if (mx <= avg / kGran[sizeof(kGran) / sizeof(kGran[0]) - 1]) return one;  // no candidate cuts a unit
  double best = 0.9 * lpt_makespan(cost, one, bins, overhead);
  std::vector<int32_t> pick = one;
  for (int g : kGran) {
    const double target = avg / g;
    std::vector<int32_t> nn(n, 1);
    bool any = false;
    for (size_t u = 0; u < n; u++) {
      const int64_t k = std::min<int64_t>(std::max<int64_t>(1, (int64_t)std::ceil(cost[u] / target)),
                                          std::max<int64_t>(1, len[u]));
      nn[u] = (int32_t)std::min<int64_t>(k, 1 << 20);
      any |= nn[u] > 1;
    }
    if (!any) continue;
    const double mk = lpt_makespan(cost, nn, bins, overhead);
    if (mk < best) {
      best = mk;
      pick = nn;
    }
  }
  return pick;
}

}  // namespace bsmm

namespace {

#define CUDA_TRY(x)                                                              \
  do {                                                                           \
    cudaError_t e_ = (x);                                                        \
    if (e_ != cudaSuccess) {                                                     \
      set_error(std::string(#x) + ": " + cudaGetErrorString(e_));                \
      return BSMM_ERR_CUDA;                                                      \
    }                                                                            \
  } while (0)

bsmm_status dev_alloc(DevBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return BSMM_OK;
  if (b.p) {
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BSMM_ERR_NOMEM : BSMM_ERR_CUDA;
  }
  b.bytes = bytes;
  return BSMM_OK;
}

template <class T>
bsmm_status upload(DevBuf& b, const std::vector<T>& v) {
  bsmm_status st = dev_alloc(b, sizeof(T) * v.size());
  if (st != BSMM_OK) return st;
  if (!v.empty()) CUDA_TRY(cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return BSMM_OK;
}

void dev_free(DevBuf& b) {
  if (b.p && !b.borrowed) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  b.borrowed = false;
}

inline int log2i_ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

inline float lg(double x) { return (float)std::log2(1.0 + x); }

void pack_lpt(bsmm_plan_s* p) {
  std::vector<int64_t> seg;
  wave_segments(0, (int64_t)p->cost.size(), p->ctas, seg);
  lpt_pack(p->cost, p->ctas, p->opt.schedule == BSMM_SCHED_NATURAL, p->sched_ptr, p->sched_units, &seg);
}

int default_ctas(const bsmm_plan_s* p) { return default_bins(p); }

bsmm_status upload_schedule(bsmm_plan_s* p) {
  bsmm_status st;
  if ((st = upload(p->d_sched_ptr, p->sched_ptr)) != BSMM_OK) return st;
  if ((st = upload(p->d_sched_units, p->sched_units)) != BSMM_OK) return st;
  return BSMM_OK;
}

// ------------------------------------------------------------------------------------
// FP64 mode: units are 64x64 sub-tiles of the C tiles of S_C; each runs the tile's
// ascending k-list.
// ------------------------------------------------------------------------------------
// Cost charged per piece when simulating a split k-list, in useful flops: about 3 us of
// one FP64 CTA (pipeline start, the partial's store and its share of the reduction).
constexpr double kF64PieceOverhead = 4096.0;

bsmm_status plan_fp64(bsmm_plan_s* p) {
  const int M = p->M, N = p->N;
  // Sub-tile edge: 32 by default. The kernel skips the register-tile rows, columns and
  // inner steps a ragged sub-tile lacks, so padding costs little at either edge; 32-wide
  // units are four times as many, which balances the persistent CTAs better, and measured
  // as fast or faster than 64 on every workload shape here (64 stays an option).
  p->f64_tile = p->opt.fp64_tile ? p->opt.fp64_tile : 32;
  const int T = p->f64_tile;
  // regions (sub-tiles of the C tiles of S_C), each with its tile's k-list
  std::vector<Fp64Unit> base;
  std::vector<double> bcost;
  std::vector<int64_t> blen;
  for (int i = 0; i < M; i++)
    for (int j = 0; j < N; j++) {
      const int64_t t = (int64_t)i * N + j;
      if (!p->cs[t]) continue;
      const int ri = p->r[i], cj = p->c[j];
      if (ri == 0 || cj == 0) continue;
      int64_t kq = 0;
      for (int64_t e = p->kptr[t]; e < p->kptr[t + 1]; e++) kq += p->q[p->klist[e]];
      for (int r0 = 0; r0 < ri; r0 += T)
        for (int c0 = 0; c0 < cj; c0 += T) {
          const int rows = std::min(T, ri - r0), cols = std::min(T, cj - c0);
          base.push_back({i, j, r0, c0, p->kptr[t], p->kptr[t + 1], -1, 0});
          bcost.push_back(std::max(2.0 * rows * cols * (double)kq, 1.0));
          blen.push_back(p->kptr[t + 1] - p->kptr[t]);
        }
    }
  // automatic cuts change FP64 rounding, so FP64 takes them only when asked (ksplit = -1)
  const int ks = p->opt.ksplit == 0 ? 1 : p->opt.ksplit == -1 ? 0 : p->opt.ksplit;
  const std::vector<int32_t> np = choose_pieces(bcost, blen, machine_bins(p), kF64PieceOverhead, ks);
  std::vector<int32_t> slot0(base.size(), -1);
  int32_t maxp = 1;
  p->n_slots = 0;
  for (size_t u = 0; u < base.size(); u++) {
    maxp = std::max(maxp, np[u]);
    if (np[u] < 2) continue;
    slot0[u] = (int32_t)p->n_slots;
    p->f64_red.push_back({base[u].i, base[u].j, base[u].r0, base[u].c0, slot0[u], np[u]});
    p->n_slots += np[u];
  }
  // units piece by piece (every region's piece 0, then every piece 1, ...): the pieces
  // that run at the same time then read the same part of the k range
  for (int32_t pc = 0; pc < maxp; pc++)
    for (size_t u = 0; u < base.size(); u++) {
      const int32_t n = np[u];
      if (pc >= n) continue;
      Fp64Unit un = base[u];
      const int64_t L = un.t1 - un.t0;
      if (n > 1) {
        un.t1 = base[u].t0 + (int64_t)(pc + 1) * L / n;
        un.t0 = base[u].t0 + (int64_t)pc * L / n;
        un.slot = slot0[u] + pc;
      }
      const int rows = std::min(T, p->r[un.i] - un.r0), cols = std::min(T, p->c[un.j] - un.c0);
      int64_t kq = 0, kg = 0;
      for (int64_t e = un.t0; e < un.t1; e++) {
        const int qk = p->q[p->klist[e]];
        kq += qk;
        kg += log2i_ceil_div(qk, kF64BK);
      }
      const int64_t nk = un.t1 - un.t0;
      p->f64_units.push_back(un);
      p->unit_pieces.push_back(n);
      const double fl = 2.0 * rows * cols * (double)kq;
      p->flop_cost.push_back(std::max(fl, 1.0));
      float f[BSMM_NFEATURES] = {lg(rows), lg(cols), lg((double)nk), lg((double)kq), lg((double)kg),
                                 lg(fl), (float)(fl / std::max(1.0, 2.0 * T * T * kF64BK * (double)kg)),
                                 0.0f, 0.0f, 0.0f, 0.0f, lg((double)kg)};
      p->features.insert(p->features.end(), f, f + BSMM_NFEATURES);
    }
  p->n_units = (int64_t)p->f64_units.size();
  return BSMM_OK;
}

// ------------------------------------------------------------------------------------
// Split modes: units are (128-row block) x (tn-column block) of the global row and
// column index spaces; a unit's k order is the ascending set of inner blocks for which
// both its packed A row block and packed B column block are present.
// ------------------------------------------------------------------------------------
// Cost charged per piece when simulating a split k-list, in useful flops: about 4 us of
// one cluster (pipeline start and drain, the 128-bit partial's store and its reduction).
constexpr double kSplitPieceOverhead = 4.0e6;

// The column-block group size for bsmm_options.cluster = -1. The CTAs of a group take the
// same row block at the same time, one column block each, and read its A panel once from
// DRAM between them; a CTA whose column block carries less tensor-core work waits for its
// partners. So: the largest of 4 and 2 for which, summed over the groups that hold a C
// tile, the CTAs' work (32-deep chunks of the k blocks where both the row block's A panel
// and the CTA's own B column block are present, on column blocks that hold a C tile) is
// at least 99.5% of the group count times its slowest CTA's; else 1.
int choose_cluster(const bsmm_plan_s* p, const std::vector<uint64_t>& presA, const std::vector<uint64_t>& presB,
                   const std::vector<int32_t>& row_tile) {
  const int RB = p->RB, CB = p->CB, KW = p->kwords, tn = p->tn, N = p->N;
  if (RB == 0 || CB < 2) return 1;
  // C tile present in (row block, column block), and the pair's chunk count
  std::vector<uint8_t> has((size_t)RB * CB, 0);
  for (int rb = 0; rb < RB; rb++) {
    const int64_t m0 = (int64_t)rb * kSplitBM, m1 = std::min<int64_t>(p->Mtot, m0 + kSplitBM);
    for (int i = row_tile[m0]; i < p->M && p->ro[i] < m1; i++) {
      if (p->ro[i + 1] <= m0) continue;
      for (int j = 0; j < N; j++) {
        if (!p->cs[(int64_t)i * N + j] || p->c[j] == 0) continue;
        for (int64_t cb = p->co[j] / tn; cb <= (p->co[j + 1] - 1) / tn; cb++) has[(size_t)rb * CB + cb] = 1;
      }
    }
  }
  std::vector<double> w((size_t)RB * CB, 0.0);
  for (int rb = 0; rb < RB; rb++)
    for (int cb = 0; cb < CB; cb++) {
      if (!has[(size_t)rb * CB + cb]) continue;
      double chunks = 0.0;
      for (int wd = 0; wd < KW; wd++) {
        uint64_t bits = presA[(size_t)rb * KW + wd] & presB[(size_t)cb * KW + wd];
        while (bits) {
          chunks += (double)((p->q[wd * 64 + __builtin_ctzll(bits)] + kSplitKC - 1) / kSplitKC);
          bits &= bits - 1;
        }
      }
      w[(size_t)rb * CB + cb] = chunks;
    }
  for (int cl : {4, 2}) {
    double sum = 0.0, worst = 0.0;
    for (int rb = 0; rb < RB; rb++)
      for (int g = 0; g * cl < CB; g++) {
        double s = 0.0, mx = 0.0;
        bool any = false;
        for (int r = 0; r < cl; r++) {
          const int cb = g * cl + r;
          if (cb >= CB) continue;  // a CTA past the last column block idles
          any = any || has[(size_t)rb * CB + cb];
          s += w[(size_t)rb * CB + cb];
          mx = std::max(mx, w[(size_t)rb * CB + cb]);
        }
        if (!any) continue;
        sum += s;
        worst += cl * mx;
      }
    if (worst > 0.0 && sum >= 0.995 * worst) return cl;
  }
  return 1;
}

bsmm_status plan_split(bsmm_plan_s* p) {
  const int M = p->M, N = p->N, K = p->K;
  const int s = p->s, tn = p->tn;
  const int64_t Mtot = p->Mtot, Ntot = p->Ntot;
  p->RB = (int)((Mtot + kSplitBM - 1) / kSplitBM);
  p->CB = (int)((Ntot + tn - 1) / tn);
  p->kwords = std::max(1, (K + 63) / 64);
  const int RB = p->RB, CB = p->CB, KW = p->kwords;
  const int maxd = split_max_depth(s);
  if (K > kSplitMaxK) {
    set_error("split modes take at most " + std::to_string(kSplitMaxK) + " inner blocks");
    return BSMM_ERR_UNSUPPORTED;
  }
  // an inner block deeper than the exact FP32 depth is accumulated in several groups (the
  // kernel's DEEP form, with store warps); the 128-bit sums stay below 2^127 while the
  // whole inner dimension is at most 2^22 elements (every slice-pair term of one inner
  // element is below 2^(7(s+1)+56) units of 2^L)
  {
    int64_t depth = 0;
    p->deep = 0;
    for (int k = 0; k < K; k++) {
      depth += p->q[k];
      if (p->q[k] > maxd) p->deep = 1;
    }
    if (depth > kSplitMaxInner) {
      set_error("split modes take an inner dimension of at most " + std::to_string(kSplitMaxInner) + " elements");
      return BSMM_ERR_UNSUPPORTED;
    }
    if (p->deep && p->opt.store_warps == 1) {
      set_error("an inner block deeper than " + std::to_string(maxd) +
                " elements needs the kernel form with store warps (store_warps 0 or 2)");
      return BSMM_ERR_UNSUPPORTED;
    }
  }

  std::vector<int32_t> row_tile(std::max<int64_t>(Mtot, 1), 0), col_tile(std::max<int64_t>(Ntot, 1), 0);
  for (int i = 0; i < M; i++)
    for (int64_t m = p->ro[i]; m < p->ro[i + 1]; m++) row_tile[m] = i;
  for (int j = 0; j < N; j++)
    for (int64_t n = p->co[j]; n < p->co[j + 1]; n++) col_tile[n] = j;

  std::vector<uint64_t> presA((size_t)RB * KW, 0), presB((size_t)CB * KW, 0);
  std::vector<int32_t> a_tiles, b_tiles;
  for (int i = 0; i < M; i++)
    for (int k = 0; k < K; k++) {
      if (!p->am[(int64_t)i * K + k] || p->r[i] == 0 || p->q[k] == 0) continue;
      a_tiles.push_back(i * K + k);
      for (int64_t rb = p->ro[i] / kSplitBM; rb <= (p->ro[i + 1] - 1) / kSplitBM; rb++)
        presA[rb * KW + k / 64] |= 1ull << (k % 64);
    }
  for (int k = 0; k < K; k++)
    for (int j = 0; j < N; j++) {
      if (!p->bm[(int64_t)k * N + j] || p->c[j] == 0 || p->q[k] == 0) continue;
      b_tiles.push_back(k * N + j);
      for (int64_t cb = p->co[j] / tn; cb <= (p->co[j + 1] - 1) / tn; cb++)
        presB[cb * KW + k / 64] |= 1ull << (k % 64);
    }
  const int64_t a_chunk_bytes = (int64_t)s * kSplitBM * kSplitKC * 2;
  const int64_t b_chunk_bytes = (int64_t)s * tn * kSplitKC * 2;
  std::vector<int64_t> apk_off((size_t)RB * K, -1), bpk_off((size_t)K * CB, -1);
  std::vector<int32_t> a_blocks, b_blocks;
  int64_t cur = 0;
  for (int rb = 0; rb < RB; rb++)
    for (int k = 0; k < K; k++)
      if (presA[(size_t)rb * KW + k / 64] >> (k % 64) & 1) {
        apk_off[(size_t)rb * K + k] = cur;
        a_blocks.push_back(rb * K + k);
        cur += (int64_t)log2i_ceil_div(p->q[k], kSplitKC) * a_chunk_bytes;
      }
  p->apk_bytes = cur;
  cur = 0;
  for (int k = 0; k < K; k++)
    for (int cb = 0; cb < CB; cb++)
      if (presB[(size_t)cb * KW + k / 64] >> (k % 64) & 1) {
        bpk_off[(size_t)k * CB + cb] = cur;
        b_blocks.push_back(k * CB + cb);
        cur += (int64_t)log2i_ceil_div(p->q[k], kSplitKC) * b_chunk_bytes;
      }
  p->bpk_bytes = cur;

  // per C tile: sum over its k-list of 2*q_k (useful flops per element)
  std::vector<double> w((size_t)M * N, 0.0);
  for (int64_t t = 0; t < (int64_t)M * N; t++)
    for (int64_t e = p->kptr[t]; e < p->kptr[t + 1]; e++) w[t] += 2.0 * p->q[p->klist[e]];

  if (p->opt.cluster == -1) p->cl = choose_cluster(p, presA, presB, row_tile);

  // A work unit is one group's task: a 128-row block times CL consecutive column blocks
  // (CL * tn columns), one column block per CTA of the group; the CL CTAs read the same
  // A panel at about the same time, so L2 serves it once from DRAM.
  const int CL = p->cl;
  const int CBG = (CB + CL - 1) / CL;
  p->CBG = CBG;
  std::vector<uint64_t> presBg((size_t)CBG * KW, 0);
  for (int cb = 0; cb < CB; cb++)
    for (int wd = 0; wd < KW; wd++) presBg[(size_t)(cb / CL) * KW + wd] |= presB[(size_t)cb * KW + wd];
  std::vector<uint8_t> umark((size_t)RB * CBG, 0);
  for (int i = 0; i < M; i++)
    for (int j = 0; j < N; j++) {
      if (!p->cs[(int64_t)i * N + j] || p->r[i] == 0 || p->c[j] == 0) continue;
      for (int64_t rb = p->ro[i] / kSplitBM; rb <= (p->ro[i + 1] - 1) / kSplitBM; rb++)
        for (int64_t cb = p->co[j] / tn; cb <= (p->co[j + 1] - 1) / tn; cb++) umark[rb * CBG + cb / CL] = 1;
    }
  // Units are numbered in bands of kRasterRows row blocks, column group by column group
  // inside a band: the persistent CTAs, which take units in this order when costs tie,
  // then work concurrently on a few A row panels and a few B column panels at a time,
  // so both stay in L2 while the CTAs stream through k.
  constexpr int kRasterRows = 8;
  std::vector<SplitUnit> base;
  std::vector<double> bcost;
  std::vector<int64_t> blen, bk_ptr{0};
  std::vector<int32_t> bk;  // each region's k-list (CSR)
  for (int rb0 = 0; rb0 < RB; rb0 += kRasterRows)
    for (int cb = 0; cb < CBG; cb++)  // cb indexes column-block groups here
      for (int rb = rb0; rb < std::min(RB, rb0 + kRasterRows); rb++) {
        if (!umark[(size_t)rb * CBG + cb]) continue;
        base.push_back({rb, cb, 0, K, -1, 0});
        for (int wd = 0; wd < KW; wd++) {
          uint64_t bits = presA[(size_t)rb * KW + wd] & presBg[(size_t)cb * KW + wd];
          while (bits) {
            bk.push_back(wd * 64 + __builtin_ctzll(bits));
            bits &= bits - 1;
          }
        }
        bk_ptr.push_back((int64_t)bk.size());
        blen.push_back(bk_ptr.back() - bk_ptr[bk_ptr.size() - 2]);
        bcost.push_back(0.0);  // set below
      }
  // useful flops of a region over inner blocks [k0, k1): its C tiles' overlap with the
  // region times 2 q_k summed over their k-lists within the range
  auto region_flops = [&](int rb, int cb, int k0, int k1, int& nrt, int& nct) {
    const int64_t m0 = (int64_t)rb * kSplitBM, m1 = std::min<int64_t>(Mtot, m0 + kSplitBM);
    const int64_t n0 = (int64_t)cb * CL * tn, n1 = std::min<int64_t>(Ntot, n0 + (int64_t)CL * tn);
    const bool whole = k0 == 0 && k1 == K;
    double fl = 0.0;
    nrt = 0;
    nct = 0;
    for (int i = row_tile[m0]; i < M && p->ro[i] < m1; i++) {
      const int64_t ov_r = std::min(m1, p->ro[i + 1]) - std::max(m0, p->ro[i]);
      if (ov_r <= 0) continue;
      nrt++;
      for (int j = col_tile[n0]; j < N && p->co[j] < n1; j++) {
        const int64_t ov_c = std::min(n1, p->co[j + 1]) - std::max(n0, p->co[j]);
        if (ov_c <= 0) continue;
        const int64_t t = (int64_t)i * N + j;
        double wt = w[t];
        if (!whole) {
          wt = 0.0;
          const int32_t* b = p->klist.data() + p->kptr[t];
          const int32_t* e = p->klist.data() + p->kptr[t + 1];
          for (const int32_t* x = std::lower_bound(b, e, k0); x != e && *x < k1; x++) wt += 2.0 * p->q[*x];
        }
        fl += (double)ov_r * (double)ov_c * wt;
      }
    }
    for (int j = col_tile[n0]; j < N && p->co[j] < n1; j++)
      if (std::min(n1, p->co[j + 1]) - std::max(n0, p->co[j]) > 0) nct++;
    return fl;
  };
  for (size_t u = 0; u < base.size(); u++) {
    int nrt, nct;
    bcost[u] = std::max(region_flops(base[u].rb, base[u].cb, 0, K, nrt, nct), 1.0);
  }
  // the contraction kernel's form: with C store warps unless the options say otherwise
  p->sw = p->opt.store_warps == 1 ? 0 : 1;
  // how the epilogue learns the accumulation groups (forms with store warps, 3 to 6
  // slices): on units of long k lists it walks the list itself, ahead of the MMA warps
  // (the dense product: 3.5% faster); on short ones it takes the MMA warps' descriptors,
  // which spares the walk's table loads on its critical path (banded: 8% faster)
  {
    double blocks = 0.0;
    for (size_t u = 0; u < base.size(); u++) blocks += (double)blen[u];
    p->epi_walk = !base.empty() && blocks >= kEpiWalkBlocks * (double)base.size() ? 1 : 0;
  }
  const std::vector<int32_t> np =
      choose_pieces(bcost, blen, machine_bins(p), kSplitPieceOverhead, p->opt.ksplit == -1 ? 0 : p->opt.ksplit);
  std::vector<int32_t> slot0(base.size(), -1);
  int32_t maxp = 1;
  p->n_slots = 0;
  for (size_t u = 0; u < base.size(); u++) {
    maxp = std::max(maxp, np[u]);
    if (np[u] < 2) continue;
    slot0[u] = (int32_t)p->n_slots;
    p->sp_red.push_back({base[u].rb, base[u].cb, slot0[u], np[u]});
    p->n_slots += np[u];
  }
  // units piece by piece (every region's piece 0, then every piece 1, ...), so the pieces
  // that run at the same time read the same part of the k range
  for (int32_t pc = 0; pc < maxp; pc++)
    for (size_t u = 0; u < base.size(); u++) {
      const int32_t n = np[u];
      if (pc >= n) continue;
      SplitUnit un = base[u];
      const int32_t* ks = bk.data() + bk_ptr[u];
      const int64_t L = blen[u];
      int64_t lo = 0, hi = L;
      if (n > 1) {
        lo = (int64_t)pc * L / n;
        hi = (int64_t)(pc + 1) * L / n;
        un.k0 = ks[lo];
        un.k1 = hi < L ? ks[hi] : K;
        un.slot = slot0[u] + pc;
      }
      un.own = 0;
      for (int r = 0; r < CL; r++) {
        const int64_t cbr = (int64_t)un.cb * CL + r;
        if (cbr >= CB) break;
        for (int k = un.k0; k < un.k1; k++)  // presA & presB of the CTA's own column block
          if ((presA[(size_t)un.rb * KW + k / 64] & presB[(size_t)cbr * KW + k / 64]) >> (k % 64) & 1) {
            un.own |= 1 << r;
            break;
          }
      }
      p->sp_units.push_back(un);
      p->unit_pieces.push_back(n);
      const int rb = un.rb, cb = un.cb;
      const int64_t m0 = (int64_t)rb * kSplitBM, m1 = std::min<int64_t>(Mtot, m0 + kSplitBM);
      const int64_t n0 = (int64_t)cb * CL * tn, n1 = std::min<int64_t>(Ntot, n0 + (int64_t)CL * tn);
      int nrt, nct;
      const double fl = region_flops(rb, cb, un.k0, un.k1, nrt, nct);
      // the k-list terms of the group's slowest CTA: each CTA of a group takes the k blocks
      // where its own column block has a B tile, and the group costs what its slowest CTA
      // does (with groups of one: the unit's whole list)
      int64_t kq = 0, kg = 0, kc = 0, nk = 0;
      for (int r = 0; r < CL; r++) {
        const int64_t cbr = (int64_t)cb * CL + r;
        if (cbr >= CB) break;
        int64_t q_r = 0, g_r = 0, c_r = 0, n_r = 0;
        for (int64_t x = lo; x < hi; x++) {
          const int k = ks[x];
          if (!(presB[(size_t)cbr * KW + k / 64] >> (k % 64) & 1)) continue;
          q_r += p->q[k];
          g_r += log2i_ceil_div(p->q[k], 16);
          c_r += log2i_ceil_div(p->q[k], kSplitKC);
          n_r++;
        }
        if (g_r > kg || (g_r == kg && q_r > kq)) kq = q_r, kg = g_r, kc = c_r, nk = n_r;
      }
      p->flop_cost.push_back(std::max(fl, 1.0));
      const double padded = 2.0 * kSplitBM * tn * CL * 16.0 * (double)kg;
      float f[BSMM_NFEATURES] = {lg((double)(m1 - m0)), lg((double)(n1 - n0)), lg((double)nk), lg((double)kq),
                                 lg((double)kg), lg(fl), (float)(padded > 0 ? fl / padded : 0.0),
                                 1.0f, (float)s / 6.0f, lg(nrt), lg(nct), lg((double)kc)};
      p->features.insert(p->features.end(), f, f + BSMM_NFEATURES);
    }
  p->n_units = (int64_t)p->sp_units.size();

  bsmm_status st;
  std::vector<int64_t> ro(p->ro), co(p->co);
  if ((st = upload(p->d_ro, ro)) != BSMM_OK) return st;
  if ((st = upload(p->d_co, co)) != BSMM_OK) return st;
  if ((st = upload(p->d_row_tile, row_tile)) != BSMM_OK) return st;
  if ((st = upload(p->d_col_tile, col_tile)) != BSMM_OK) return st;
  if ((st = upload(p->d_presA, presA)) != BSMM_OK) return st;
  if ((st = upload(p->d_presB, presB)) != BSMM_OK) return st;
  if ((st = upload(p->d_presBg, presBg)) != BSMM_OK) return st;
  if ((st = upload(p->d_apk_off, apk_off)) != BSMM_OK) return st;
  if ((st = upload(p->d_bpk_off, bpk_off)) != BSMM_OK) return st;
  if ((st = upload(p->d_a_tiles, a_tiles)) != BSMM_OK) return st;
  if ((st = upload(p->d_b_tiles, b_tiles)) != BSMM_OK) return st;
  if ((st = upload(p->d_a_blocks, a_blocks)) != BSMM_OK) return st;
  if ((st = upload(p->d_b_blocks, b_blocks)) != BSMM_OK) return st;
  if ((st = upload(p->d_units, p->sp_units)) != BSMM_OK) return st;
  if ((st = upload(p->d_red, p->sp_red)) != BSMM_OK) return st;
  if ((st = dev_alloc(p->d_part, (size_t)p->n_slots * CL * kSplitBM * tn * 16)) != BSMM_OK) return st;
  if ((st = upload(p->d_am, p->am)) != BSMM_OK) return st;
  if ((st = upload(p->d_bm, p->bm)) != BSMM_OK) return st;
  p->n_a_tiles = (int32_t)a_tiles.size();
  p->n_b_tiles = (int32_t)b_tiles.size();
  p->n_a_blocks = (int32_t)a_blocks.size();
  p->n_b_blocks = (int32_t)b_blocks.size();
  const bsmm_plan_s* d = p->donor;
  if (d && d->opt.mode != BSMM_FP64 && d->s == p->s && d->apk_bytes == p->apk_bytes && d->bpk_bytes == p->bpk_bytes &&
      d->d_apk.p && d->d_bpk.p) {
    p->d_apk = d->d_apk;
    p->d_bpk = d->d_bpk;
    p->d_apk.borrowed = p->d_bpk.borrowed = true;
  } else {
    p->donor = nullptr;
    if ((st = dev_alloc(p->d_apk, (size_t)p->apk_bytes)) != BSMM_OK) return st;
    if ((st = dev_alloc(p->d_bpk, (size_t)p->bpk_bytes)) != BSMM_OK) return st;
  }
  if ((st = dev_alloc(p->d_eA, sizeof(int32_t) * std::max<int64_t>(1, (int64_t)M * K))) != BSMM_OK) return st;
  if ((st = dev_alloc(p->d_eB, sizeof(int32_t) * std::max<int64_t>(1, (int64_t)K * N))) != BSMM_OK) return st;
  if ((st = dev_alloc(p->d_eAmax, sizeof(int32_t) * std::max(1, M))) != BSMM_OK) return st;
  if ((st = dev_alloc(p->d_eBmax, sizeof(int32_t) * std::max(1, N))) != BSMM_OK) return st;
  if ((st = dev_alloc(p->d_rowexp, sizeof(int16_t) * std::max<int64_t>(1, (int64_t)K * Mtot))) != BSMM_OK) return st;
  p->colexp_ld = (Ntot + 63) / 64 * 64 + 64;  // padded rows: aligned 16-byte loads past the last column
  if ((st = dev_alloc(p->d_colexp, sizeof(int16_t) * ((int64_t)K * p->colexp_ld + 64))) != BSMM_OK) return st;
  if (p->opt.split_scale) {
    if ((st = dev_alloc(p->d_eArow, sizeof(int32_t) * std::max<int64_t>(1, (int64_t)K * Mtot))) != BSMM_OK) return st;
    if ((st = dev_alloc(p->d_eBcol, sizeof(int32_t) * std::max<int64_t>(1, (int64_t)K * Ntot))) != BSMM_OK) return st;
    if ((st = dev_alloc(p->d_eAmaxr, sizeof(int32_t) * std::max<int64_t>(1, Mtot))) != BSMM_OK) return st;
    if ((st = dev_alloc(p->d_eBmaxc, sizeof(int32_t) * std::max<int64_t>(1, Ntot))) != BSMM_OK) return st;
  }
  if ((st = dev_alloc(p->d_urow, sizeof(int16_t) * std::max<int64_t>(1, (int64_t)K * p->RB))) != BSMM_OK) return st;
  if ((st = dev_alloc(p->d_ucol, sizeof(int16_t) * std::max<int64_t>(1, (int64_t)K * p->CB))) != BSMM_OK) return st;
  if ((st = dev_alloc(p->d_rowadj, sizeof(int16_t) * std::max<int64_t>(1, Mtot))) != BSMM_OK) return st;
  if ((st = dev_alloc(p->d_coladj, sizeof(int16_t) * (p->colexp_ld + 64))) != BSMM_OK) return st;
  CUDA_TRY(cudaMemset(p->d_coladj.p, 0, p->d_coladj.bytes));  // padding columns read as 0
  if ((st = dev_alloc(p->d_emaxr, sizeof(int32_t) * std::max<int64_t>(1, Mtot))) != BSMM_OK) return st;
  if ((st = dev_alloc(p->d_emaxc, sizeof(int32_t) * (p->colexp_ld + 64))) != BSMM_OK) return st;
  CUDA_TRY(cudaMemset(p->d_emaxc.p, 0, p->d_emaxc.bytes));
  // exponents of absent tiles stay 0 (their slices are zero, so the scale is never used)
  CUDA_TRY(cudaMemset(p->d_rowexp.p, 0, p->d_rowexp.bytes));
  CUDA_TRY(cudaMemset(p->d_colexp.p, 0, p->d_colexp.bytes));
  return BSMM_OK;
}

bsmm_status validate_options(const bsmm_options& o) {
  if (o.mode < 0 || o.mode > 2) return set_error("unknown mode"), BSMM_ERR_INVALID;
  if (o.mode != BSMM_FP64 && (o.nslices < 1 || o.nslices > kSplitMaxS))
    return set_error("nslices must be in 1..6"), BSMM_ERR_INVALID;
  if (o.schedule < 0 || o.schedule > 2) return set_error("unknown schedule"), BSMM_ERR_INVALID;
  if (o.max_ctas < 0) return set_error("max_ctas < 0"), BSMM_ERR_INVALID;
  if (o.profile < 0 || o.profile > 1) return set_error("profile must be 0 or 1"), BSMM_ERR_INVALID;
  if (o.cluster != -1 && o.cluster != 0 && o.cluster != 1 && o.cluster != 2 && o.cluster != 4)
    return set_error("cluster must be -1, 0, 1, 2 or 4"), BSMM_ERR_INVALID;
  if (o.fp64_tile != 0 && o.fp64_tile != 32 && o.fp64_tile != 64)
    return set_error("fp64_tile must be 0, 32 or 64"), BSMM_ERR_INVALID;
  if (o.stages != 0 && (o.stages < 2 || o.stages > 8)) return set_error("stages must be 0 or 2..8"), BSMM_ERR_INVALID;
  if (o.mode != BSMM_FP64 && o.stages && split_smem_bytes(o.nslices, split_tile_n(o.nslices), o.stages) > kMaxSmemPerCta)
    return set_error("stages: the ring does not fit the shared memory of one CTA"), BSMM_ERR_UNSUPPORTED;
  if ((o.transa != 0 && o.transa != 1) || (o.transb != 0 && o.transb != 1))
    return set_error("transa and transb must be 0 or 1"), BSMM_ERR_INVALID;
  if (o.split_scale != 0 && o.split_scale != 1) return set_error("split_scale must be 0 or 1"), BSMM_ERR_INVALID;
  if (o.ksplit < -1 || o.ksplit > 65536) return set_error("ksplit must be in -1..65536"), BSMM_ERR_INVALID;
  if (o.store_warps < 0 || o.store_warps > 2) return set_error("store_warps must be 0, 1 or 2"), BSMM_ERR_INVALID;
  if (o.elem != BSMM_F64 && o.elem != BSMM_F32 && o.elem != BSMM_C128)
    return set_error("unknown element type"), BSMM_ERR_INVALID;
  if (o.elem != BSMM_F64 && o.mode == BSMM_FP64)
    return set_error("float32 and complex elements take a split mode"), BSMM_ERR_UNSUPPORTED;
  return BSMM_OK;
}

}  // namespace

// ======================================================================================
// C ABI
// ======================================================================================
namespace bsmm {

void host_release(bsmm_plan_s* p) {
  for (auto& h : p->hs) {
    if (h.used && h.out) cudaEventSynchronize(h.out);
    for (DevBuf* b : {&h.A, &h.B, &h.C, &h.aoff, &h.boff, &h.coff}) dev_free(*b);
    for (cudaEvent_t* ev : {&h.in, &h.run, &h.out})
      if (*ev) {
        cudaEventDestroy(*ev);
        *ev = nullptr;
      }
    h.used = false;
  }
  if (p->last_run) cudaEventDestroy(p->last_run);
  if (p->h2d) cudaStreamDestroy(p->h2d);
  if (p->d2h) cudaStreamDestroy(p->d2h);
  p->last_run = nullptr;
  p->h2d = p->d2h = nullptr;
}

}  // namespace bsmm

extern "C" {

void bsmm_options_default(bsmm_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->mode = BSMM_FP64;
  opt->nslices = 6;
  opt->schedule = BSMM_SCHED_FLOPS;
}

const char* bsmm_last_error(void) { return g_last_error.c_str(); }

void bsmm_destroy(bsmm_plan_t p) {
  if (!p) return;
  DevBuf* bufs[] = {&p->d_r, &p->d_c, &p->d_q, &p->d_ro, &p->d_co, &p->d_kptr, &p->d_klist, &p->d_cs,
                    &p->d_units, &p->d_sched_ptr, &p->d_sched_units, &p->d_row_tile, &p->d_col_tile,
                    &p->d_presA, &p->d_presB, &p->d_presBg, &p->d_apk_off, &p->d_bpk_off, &p->d_apk, &p->d_bpk,
                    &p->d_eArow, &p->d_eBcol, &p->d_eAmaxr, &p->d_eBmaxc,
                    &p->d_am, &p->d_bm, &p->d_rowexp, &p->d_colexp, &p->d_urow, &p->d_ucol, &p->d_rowadj, &p->d_coladj, &p->d_emaxr, &p->d_emaxc, &p->d_eA, &p->d_eB, &p->d_eAmax, &p->d_eBmax, &p->d_a_tiles, &p->d_b_tiles,
                    &p->d_a_blocks, &p->d_b_blocks, &p->d_err, &p->d_timings, &p->d_unit_cta, &p->d_part, &p->d_red};
  host_release(p);
  for (DevBuf* b : bufs) dev_free(*b);
  for (auto& set : p->ev)
    for (cudaEvent_t& e : set)
      if (e) cudaEventDestroy(e);
  delete p;
}

}  // extern "C"

namespace bsmm {

bsmm_status plan_build(bsmm_plan_t* out, int32_t M, const int32_t* row_sizes, int32_t N, const int32_t* col_sizes,
                       int32_t K, const int32_t* inner_sizes, const uint8_t* a_mask, const uint8_t* b_mask,
                       const uint8_t* c_mask, const bsmm_options* opt, const bsmm_plan_s* donor) {
  if (!out) return set_error("out is NULL"), BSMM_ERR_INVALID;
  *out = nullptr;
  if (M < 0 || N < 0 || K < 0) return set_error("negative block count"), BSMM_ERR_INVALID;
  if ((M && !row_sizes) || (N && !col_sizes) || (K && !inner_sizes))
    return set_error("NULL tiling"), BSMM_ERR_INVALID;
  if (((int64_t)M * K && !a_mask) || ((int64_t)K * N && !b_mask))
    return set_error("NULL mask"), BSMM_ERR_INVALID;
  bsmm_options o;
  if (opt)
    o = *opt;
  else
    bsmm_options_default(&o);
  bsmm_status st = validate_options(o);
  if (st != BSMM_OK) return st;
  for (int i = 0; i < M; i++)
    if (row_sizes[i] < 0) return set_error("negative row block size"), BSMM_ERR_INVALID;
  for (int j = 0; j < N; j++)
    if (col_sizes[j] < 0) return set_error("negative column block size"), BSMM_ERR_INVALID;
  for (int k = 0; k < K; k++)
    if (inner_sizes[k] < 0) return set_error("negative inner block size"), BSMM_ERR_INVALID;

  bsmm_plan_s* p = new (std::nothrow) bsmm_plan_s();
  if (!p) return set_error("out of host memory"), BSMM_ERR_NOMEM;
  p->M = M;
  p->N = N;
  p->K = K;
  p->opt = o;
  const std::string model_path = o.model_path ? o.model_path : "";
  p->opt.model_path = nullptr;  // the caller's string is read here only
  p->donor = donor;
  static std::atomic<uint64_t> next_uid{1};
  p->uid = next_uid++;
  p->r.assign(row_sizes, row_sizes + M);
  p->c.assign(col_sizes, col_sizes + N);
  p->q.assign(inner_sizes, inner_sizes + K);
  if (o.elem == BSMM_C128) {
    // complex elements run as the real product [Ar, -Ai] x [[Br, Bi], [Bi, -Br]]: every
    // inner and column block holds twice as many real lines
    for (int32_t& x : p->q) x *= 2;
    for (int32_t& x : p->c) x *= 2;
  }
  p->ro.assign(M + 1, 0);
  p->co.assign(N + 1, 0);
  p->qo.assign(K + 1, 0);
  for (int i = 0; i < M; i++) p->ro[i + 1] = p->ro[i] + p->r[i];
  for (int j = 0; j < N; j++) p->co[j + 1] = p->co[j] + p->c[j];
  for (int k = 0; k < K; k++) p->qo[k + 1] = p->qo[k] + p->q[k];
  p->Mtot = p->ro[M];
  p->Ntot = p->co[N];
  p->am.resize((size_t)M * K);
  p->bm.resize((size_t)K * N);
  // masks in the (i,k) / (k,j) orientation the planner works in (transposed inputs are
  // read transposed; the kernels index the caller's offset tables accordingly)
  for (int i = 0; i < M; i++)
    for (int k = 0; k < K; k++)
      p->am[(int64_t)i * K + k] = (o.transa ? a_mask[(int64_t)k * M + i] : a_mask[(int64_t)i * K + k]) ? 1 : 0;
  for (int k = 0; k < K; k++)
    for (int j = 0; j < N; j++)
      p->bm[(int64_t)k * N + j] = (o.transb ? b_mask[(int64_t)j * K + k] : b_mask[(int64_t)k * N + j]) ? 1 : 0;

  // S_C = boolean product of the masks (bitset rows), united with the C mask;
  // per C tile the ascending k-list; the useful flop count.
  const int KW = std::max(1, (K + 63) / 64);
  std::vector<uint64_t> arow((size_t)M * KW, 0), bcol((size_t)N * KW, 0);
  for (int i = 0; i < M; i++)
    for (int k = 0; k < K; k++)
      if (p->am[(int64_t)i * K + k]) arow[(size_t)i * KW + k / 64] |= 1ull << (k % 64);
  for (int k = 0; k < K; k++)
    for (int j = 0; j < N; j++)
      if (p->bm[(int64_t)k * N + j]) bcol[(size_t)j * KW + k / 64] |= 1ull << (k % 64);
  p->cs.assign((size_t)M * N, 0);
  p->kptr.assign((size_t)M * N + 1, 0);
  p->klist.clear();
  double flops = 0.0;
  for (int i = 0; i < M; i++)
    for (int j = 0; j < N; j++) {
      const int64_t t = (int64_t)i * N + j;
      p->kptr[t] = (int64_t)p->klist.size();
      for (int wd = 0; wd < KW; wd++) {
        uint64_t bits = arow[(size_t)i * KW + wd] & bcol[(size_t)j * KW + wd];
        while (bits) {
          const int k = wd * 64 + __builtin_ctzll(bits);
          bits &= bits - 1;
          p->klist.push_back(k);
          flops += 2.0 * (double)p->r[i] * (double)p->c[j] * (double)p->q[k];
        }
      }
      const bool any = (int64_t)p->klist.size() > p->kptr[t];
      p->cs[t] = (any || (c_mask && c_mask[t])) ? 1 : 0;
      p->n_ctiles += p->cs[t];
    }
  p->kptr[(size_t)M * N] = (int64_t)p->klist.size();
  p->n_triples = (int64_t)p->klist.size();
  p->useful_flops = flops;

  cudaError_t ce = cudaGetDevice(&p->device);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
  if (ce != cudaSuccess) {
    set_error(std::string("no CUDA device: ") + cudaGetErrorString(ce));
    delete p;
    return BSMM_ERR_CUDA;
  }

  if (o.mode == BSMM_FP64) {
    st = plan_fp64(p);
  } else {
    p->s = o.nslices;
    p->cl = o.cluster > 0 ? o.cluster : kSplitDefaultCluster;  // -1: chosen in plan_split
    p->tn = split_tile_n(p->s);
    p->stages = o.stages ? o.stages : split_stages(p->s, p->tn);
    st = plan_split(p);
  }
  if (st != BSMM_OK) {
    bsmm_destroy(p);
    return st;
  }
  p->donor = nullptr;  // only planning reads it
  p->cost = p->flop_cost;
  p->ctas = default_ctas(p);
  pack_lpt(p);

  std::vector<int32_t> r(p->r), c(p->c), q(p->q);
  std::vector<int32_t> klist(p->klist);
  if (klist.empty()) klist.push_back(0);
  if ((st = upload(p->d_r, r)) != BSMM_OK || (st = upload(p->d_c, c)) != BSMM_OK ||
      (st = upload(p->d_q, q)) != BSMM_OK || (st = upload(p->d_kptr, p->kptr)) != BSMM_OK ||
      (st = upload(p->d_klist, klist)) != BSMM_OK || (st = upload(p->d_cs, p->cs)) != BSMM_OK ||
      (st = upload_schedule(p)) != BSMM_OK) {
    bsmm_destroy(p);
    return st;
  }
  if (o.mode == BSMM_FP64 &&
      ((st = upload(p->d_units, p->f64_units)) != BSMM_OK || (st = upload(p->d_red, p->f64_red)) != BSMM_OK ||
       (st = dev_alloc(p->d_part, sizeof(double) * (size_t)p->n_slots * p->f64_tile * p->f64_tile)) != BSMM_OK)) {
    bsmm_destroy(p);
    return st;
  }
  if ((st = dev_alloc(p->d_err, sizeof(int32_t))) != BSMM_OK) {
    bsmm_destroy(p);
    return st;
  }
  if (cudaMemset(p->d_err.p, 0, sizeof(int32_t)) != cudaSuccess) {
    set_error("cudaMemset of the error word failed");
    bsmm_destroy(p);
    return BSMM_ERR_CUDA;
  }
  if (o.record_timings) {
    if ((st = dev_alloc(p->d_timings, sizeof(int64_t) * 2 * std::max<int64_t>(1, p->n_units))) != BSMM_OK ||
        (st = dev_alloc(p->d_unit_cta, sizeof(int32_t) * std::max<int64_t>(1, p->n_units))) != BSMM_OK) {
      bsmm_destroy(p);
      return st;
    }
  }
  // the learned costs of a cost-model file; a file that cannot be used leaves the
  // flop-count costs (the fallback) and the plan is still built
  if (!model_path.empty() && o.schedule != BSMM_SCHED_NATURAL && p->n_units > 0) {
    const std::string keep = g_last_error;
    bsmm_mlp_t mlp = nullptr;
    if (bsmm_mlp_load(&mlp, model_path.c_str()) == BSMM_OK) {
      if (bsmm_plan_predict_costs(p, mlp, nullptr) == BSMM_OK) {
        p->cost_source = BSMM_COSTS_MODEL;
      } else {  // back to the flop-count packing
        p->cost = p->flop_cost;
        p->opt.schedule = o.schedule;
        pack_lpt(p);
        if ((st = upload_schedule(p)) != BSMM_OK) {
          bsmm_mlp_destroy(mlp);
          bsmm_destroy(p);
          return st;
        }
      }
      bsmm_mlp_destroy(mlp);
    }
    if (p->cost_source != BSMM_COSTS_MODEL) g_last_error = keep;  // the fallback is not an error
  }
  *out = p;
  return BSMM_OK;
}

}  // namespace bsmm

extern "C" {

bsmm_status bsmm_plan(bsmm_plan_t* out, int32_t M, const int32_t* row_sizes, int32_t N,
                      const int32_t* col_sizes, int32_t K, const int32_t* inner_sizes,
                      const uint8_t* a_mask, const uint8_t* b_mask, const uint8_t* c_mask,
                      const bsmm_options* opt) {
  return plan_build(out, M, row_sizes, N, col_sizes, K, inner_sizes, a_mask, b_mask, c_mask, opt, nullptr);
}

bsmm_status bsmm_plan_query(bsmm_plan_t p, int64_t* n_ctiles, int64_t* n_triples, double* useful_flops,
                            uint8_t* c_mask_out, int64_t* n_units) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  if (n_ctiles) *n_ctiles = p->n_ctiles;
  if (n_triples) *n_triples = p->n_triples;
  if (useful_flops) *useful_flops = p->useful_flops;
  if (c_mask_out && !p->cs.empty()) std::memcpy(c_mask_out, p->cs.data(), p->cs.size());
  if (n_units) *n_units = p->n_units;
  return BSMM_OK;
}

bsmm_status bsmm_schedule_lpt(int64_t n, const double* cost, int32_t bins, int32_t* ptr, int32_t* units,
                              double* makespan) {
  if (n < 0 || bins < 1 || (n > 0 && (!cost || !units)) || !ptr)
    return set_error("schedule_lpt: NULL array, n < 0 or bins < 1"), BSMM_ERR_INVALID;
  std::vector<double> c(cost, cost + n);
  for (double x : c)
    if (!(x > 0.0) || !std::isfinite(x)) return set_error("schedule_lpt: costs must be finite and > 0"), BSMM_ERR_INVALID;
  std::vector<int32_t> p_, u_;
  lpt_pack(c, bins, false, p_, u_);
  std::copy(p_.begin(), p_.end(), ptr);
  std::copy(u_.begin(), u_.end(), units);
  if (makespan) {
    double mk = 0.0;
    for (int b = 0; b < bins; b++) {
      double l = 0.0;
      for (int32_t x = p_[b]; x < p_[b + 1]; x++) l += c[u_[x]];
      mk = std::max(mk, l);
    }
    *makespan = mk;
  }
  return BSMM_OK;
}

bsmm_status bsmm_schedule_pieces(int64_t n, const double* cost, const int64_t* len, int32_t bins, double overhead,
                                 int32_t ksplit, int32_t* pieces) {
  if (n < 0 || bins < 1 || (n > 0 && (!cost || !len || !pieces)))
    return set_error("schedule_pieces: NULL array, n < 0 or bins < 1"), BSMM_ERR_INVALID;
  if (ksplit < 0 || ksplit > 65536 || !(overhead >= 0.0)) return set_error("schedule_pieces: bad ksplit or overhead"), BSMM_ERR_INVALID;
  std::vector<double> c(cost, cost + n);
  std::vector<int64_t> l(len, len + n);
  for (int64_t i = 0; i < n; i++)
    if (!(c[i] > 0.0) || !std::isfinite(c[i]) || l[i] < 0)
      return set_error("schedule_pieces: costs must be finite and > 0, lengths >= 0"), BSMM_ERR_INVALID;
  const std::vector<int32_t> np = choose_pieces(c, l, bins, overhead, ksplit);
  std::copy(np.begin(), np.end(), pieces);
  return BSMM_OK;
}

bsmm_status bsmm_plan_ksplit(bsmm_plan_t p, int64_t* n_regions, int64_t* n_pieces, int32_t* pieces) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  if (n_regions) *n_regions = (int64_t)(p->opt.mode == BSMM_FP64 ? p->f64_red.size() : p->sp_red.size());
  if (n_pieces) *n_pieces = p->n_slots;
  if (pieces && !p->unit_pieces.empty())
    std::memcpy(pieces, p->unit_pieces.data(), sizeof(int32_t) * p->unit_pieces.size());
  return BSMM_OK;
}

bsmm_status bsmm_plan_features(bsmm_plan_t p, float* features, double* flop_costs) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  if (features && !p->features.empty())
    std::memcpy(features, p->features.data(), sizeof(float) * p->features.size());
  if (flop_costs && !p->flop_cost.empty())
    std::memcpy(flop_costs, p->flop_cost.data(), sizeof(double) * p->flop_cost.size());
  return BSMM_OK;
}

bsmm_status bsmm_plan_set_costs(bsmm_plan_t p, const double* costs) {
  if (!p || !costs) return set_error("NULL argument"), BSMM_ERR_INVALID;
  for (int64_t u = 0; u < p->n_units; u++)
    if (!(costs[u] > 0.0) || !std::isfinite(costs[u])) return set_error("costs must be finite and > 0"), BSMM_ERR_INVALID;
  p->cost.assign(costs, costs + p->n_units);
  p->opt.schedule = BSMM_SCHED_COSTS;
  p->cost_source = BSMM_COSTS_GIVEN;
  pack_lpt(p);
  return upload_schedule(p);
}

bsmm_status bsmm_plan_cost_source(bsmm_plan_t p, int32_t* source) {
  if (!p || !source) return set_error("NULL argument"), BSMM_ERR_INVALID;
  *source = p->cost_source;
  return BSMM_OK;
}

bsmm_status bsmm_plan_form(bsmm_plan_t p, int32_t* cluster, int32_t* store_warps, int32_t* epi_walk,
                           int32_t* stages, int32_t* ctas) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  const bool split = p->opt.mode != BSMM_FP64;
  if (cluster) *cluster = split ? p->cl : 1;
  if (store_warps) *store_warps = split ? p->sw : 0;
  if (epi_walk) *epi_walk = split && p->sw && p->s >= 3 ? p->epi_walk : 0;
  if (stages) *stages = split ? p->stages : 0;
  if (ctas) *ctas = p->ctas;
  return BSMM_OK;
}

bsmm_status bsmm_plan_set_ctas(bsmm_plan_t p, int32_t ctas) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  if (ctas < 0 || ctas > 65535) return set_error("ctas out of range"), BSMM_ERR_INVALID;
  p->ctas = ctas == 0 ? default_ctas(p) : (int)std::min<int64_t>(ctas, std::max<int64_t>(1, p->n_units));
  pack_lpt(p);
  return upload_schedule(p);
}

}  // extern "C"
