// Many independent block-sparse products in few persistent launches.
//
// The paper schedules the tasks of one product over a process grid (Sec. 3.2); a
// batch is the same idea across products: the work units of many products form one
// task set, packed longest-processing-time first onto the persistent CTAs (FP64) or
// clusters (split modes) of one contraction launch, so short products fill the gaps
// left by long ones instead of each paying a launch and a tail. Each unit reads its
// product's arguments from a device table. In the split modes the products are cut
// into waves whose slice workspaces fit in half of L2: a wave issues its products'
// exponent and slicing kernels and then its contraction launch, which finds the slices
// still in L2 (a product larger than that is a wave of its own). FP64 is one wave.
// Products whose plans split a k-list (bsmm_options.ksplit) get their reduction kernels
// after the contraction launch of their wave.
// Consecutive waves of a split batch go to two streams in turn (the caller's and one of
// the batch's, forked from and joined back into the caller's), as the paper lets the
// stages of independent products overlap (Sec. 1: no global synchronisation between
// multiplications): a wave's slicing kernels and contraction start on the SMs that the
// previous wave's contraction frees during its last units, instead of after its last
// CTA. Waves share no buffer, so nothing orders them but the stream they run on.
// bsmm_batch_execute issues kernels and stream events only, so a stream capture of it
// records a CUDA graph that replays the whole batch with one graph launch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>

#include "bsmm_internal.h"

using namespace bsmm;

struct bsmm_batch_s {
  std::vector<bsmm_plan_t> plans;
  int mode = 0, s = 0, cl = 1, stages = 0;
  int sw = 0;  // split modes: the contraction launches use the kernel form with store warps
  int64_t n_units = 0;
  double useful_flops = 0.0;
  std::vector<int32_t> unit_prod, unit_local;
  std::vector<int64_t> prod_begin;  // first batch-wide unit of each product (+ total)
  std::vector<double> cost;
  int bins = 0;  // persistent CTAs (FP64) or clusters (split) of a full launch
  // Waves: consecutive products whose slice workspace fits in half of L2 run their
  // slicing kernels and then one contraction launch, so the contraction reads slices
  // the slicing kernels just left in L2; a product larger than that is a wave of its
  // own. FP64 has no slice workspace: one wave. wave_prod[w] is the first product of
  // wave w (+ count), wave_bins[w] its grid, wave_ptr[w] the start of its schedule in
  // sched_ptr (wave_bins[w] + 1 entries, absolute positions in sched_units).
  std::vector<int32_t> wave_prod, wave_bins;
  std::vector<int64_t> wave_ptr;
  std::vector<int32_t> sched_ptr, sched_units;
  std::vector<Fp64Args> fargs;
  std::vector<SplitArgs> sargs;
  bool args_set = false;
  int32_t launches = 0;  // kernels the last bsmm_batch_execute launched
  DevBuf d_prods, d_unit_prod, d_unit_local, d_sched_ptr, d_sched_units, d_err;
  std::vector<bsmm_plan_t> owned;  // plans made by bsmm_batch_autotune, destroyed with the batch
  cudaStream_t side = nullptr;     // split modes with two or more waves: the second stream
  cudaEvent_t fork = nullptr, join = nullptr;
};

namespace {

bsmm_status dalloc(DevBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return BSMM_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    b.p = nullptr;
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BSMM_ERR_NOMEM : BSMM_ERR_CUDA;
  }
  b.bytes = bytes ? bytes : 16;
  return BSMM_OK;
}

template <class T>
bsmm_status put(DevBuf& b, const std::vector<T>& v) {
  bsmm_status st = dalloc(b, sizeof(T) * v.size());
  if (st != BSMM_OK) return st;
  if (!v.empty() && cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error("batch table upload failed"), BSMM_ERR_CUDA;
  return BSMM_OK;
}

bsmm_status repack(bsmm_batch_s* b) {
  b->sched_ptr.clear();
  b->sched_units.clear();
  b->wave_ptr.clear();
  for (size_t w = 0; w + 1 < b->wave_prod.size(); w++) {
    const int64_t u0 = b->prod_begin[b->wave_prod[w]], u1 = b->prod_begin[b->wave_prod[w + 1]];
    std::vector<double> cost(b->cost.begin() + u0, b->cost.begin() + u1);
    std::vector<int64_t> seg;  // product by product, each in waves of one unit per bin
    for (int32_t p = b->wave_prod[w]; p < b->wave_prod[w + 1]; p++)
      wave_segments(b->prod_begin[p] - u0, b->prod_begin[p + 1] - u0, b->wave_bins[w], seg);
    if (seg.empty()) seg.push_back(0);
    std::vector<int32_t> ptr, units;
    lpt_pack(cost, b->wave_bins[w], false, ptr, units, &seg);
    b->wave_ptr.push_back((int64_t)b->sched_ptr.size());
    const int32_t base = (int32_t)b->sched_units.size();
    for (int32_t x : ptr) b->sched_ptr.push_back(base + x);
    for (int32_t u : units) b->sched_units.push_back((int32_t)(u0 + u));
  }
  bsmm_status st;
  if ((st = put(b->d_sched_ptr, b->sched_ptr)) != BSMM_OK) return st;
  return put(b->d_sched_units, b->sched_units);
}

void free_batch(bsmm_batch_s* b) {
  if (b->side) cudaStreamSynchronize(b->side);
  for (DevBuf* d : {&b->d_prods, &b->d_unit_prod, &b->d_unit_local, &b->d_sched_ptr, &b->d_sched_units, &b->d_err})
    if (d->p) cudaFree(d->p);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->side) cudaStreamDestroy(b->side);
  for (bsmm_plan_t p : b->owned) bsmm_destroy(p);
  delete b;
}

// The caller's per-product arguments, as stored by bsmm_batch_set_args.
struct BatchArgs {
  std::vector<double> alpha, beta;
  std::vector<const void*> A, B;
  std::vector<const int64_t*> ao, bo, co;
  std::vector<void*> C;
  explicit BatchArgs(const bsmm_batch_s* b) {
    const size_t n = b->plans.size();
    alpha.resize(n), beta.resize(n), A.resize(n), B.resize(n), ao.resize(n), bo.resize(n), co.resize(n), C.resize(n);
    for (size_t i = 0; i < n; i++) {
      if (b->mode == BSMM_FP64) {
        const Fp64Args& a = b->fargs[i];
        alpha[i] = a.alpha, beta[i] = a.beta, A[i] = a.A, B[i] = a.B, ao[i] = a.a_off, bo[i] = a.b_off;
        co[i] = a.c_off, C[i] = a.C;
      } else {
        const SplitArgs& a = b->sargs[i];
        alpha[i] = a.alpha, beta[i] = a.beta, ao[i] = a.a_off, bo[i] = a.b_off, co[i] = a.c_off;
        A[i] = a.f32 ? (const void*)a.Af : (const void*)a.A;
        B[i] = a.f32 ? (const void*)a.Bf : (const void*)a.B;
        C[i] = a.f32 ? (void*)a.Cf : (void*)a.C;
      }
    }
  }
  bsmm_status set(bsmm_batch_t b, const std::vector<void*>& Cs) const;
};

// Plans of every product of `src` under options `o` (sharing the slice workspace of the
// batch's own plans); on failure none is left.
bsmm_status replan(const bsmm_batch_s* src, const bsmm_tune_point& t, std::vector<bsmm_plan_t>& out) {
  out.clear();
  for (const bsmm_plan_s* p : src->plans) {
    bsmm_options o = p->opt;
    o.profile = 0;
    o.record_timings = 0;
    if (o.schedule == BSMM_SCHED_COSTS) o.schedule = BSMM_SCHED_FLOPS;
    if (o.mode == BSMM_FP64) {
      o.fp64_tile = t.fp64_tile;
    } else {
      o.cluster = t.cluster;
      o.stages = t.stages;
      o.store_warps = t.store_warps;
    }
    bsmm_plan_t np = nullptr;
    const bsmm_status st = plan_build(&np, p->M, p->r.data(), p->N, p->c.data(), p->K, p->q.data(), p->am.data(),
                                      p->bm.data(), p->cs.data(), &o, p);
    if (st != BSMM_OK) {
      for (bsmm_plan_t q : out) bsmm_destroy(q);
      out.clear();
      return st;
    }
    out.push_back(np);
  }
  return BSMM_OK;
}

}  // namespace

namespace {

// The batch takes its products re-planned under candidate t, with the arguments already
// set (the previous tables, and the plans of an earlier tuning, are released; the plans
// given to bsmm_batch_create keep owning the slice workspace the new plans share).
bsmm_status adopt(bsmm_batch_s* b, const bsmm_tune_point& t) {
  const BatchArgs args(b);
  std::vector<bsmm_plan_t> plans;
  bsmm_status s = replan(b, t, plans);
  bsmm_batch_t nb = nullptr;
  if (s == BSMM_OK) s = bsmm_batch_create(&nb, (int32_t)plans.size(), plans.data());
  if (s == BSMM_OK) s = args.set(nb, args.C);
  if (s != BSMM_OK) {
    if (nb) bsmm_batch_destroy(nb);
    for (bsmm_plan_t q : plans) bsmm_destroy(q);
    return s;
  }
  nb->owned = plans;
  std::swap(*b, *nb);
  free_batch(nb);
  return BSMM_OK;
}

// The tuning cache: a JSON file, one entry per line, keyed by GPU, mode and slice count.
//   {"format": "bsmm-tune", "version": 1, "entries": [
//    {"key": "<gpu>|<mode>|s=<n>", "cluster": c, "stages": t, "fp64_tile": f, "store_warps": w,
//     "ms_x1000": the candidate's median time in microseconds},
//    ...
//   ]}
constexpr int kTuneCacheVersion = 1;

struct TuneEntry {
  std::string key;
  bsmm_tune_point t{};
  double ms = 0.0;
};

bool json_int(const std::string& line, const char* name, long long& v) {
  const std::string pat = std::string("\"") + name + "\": ";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return false;
  char* end = nullptr;
  v = std::strtoll(line.c_str() + at + pat.size(), &end, 10);
  return end != line.c_str() + at + pat.size();
}

// the entries of a cache file of this version (none for a missing, foreign or older file)
std::vector<TuneEntry> read_tune_cache(const char* path) {
  std::vector<TuneEntry> out;
  FILE* f = std::fopen(path, "r");
  if (!f) return out;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0 && text.size() < (1u << 22)) text.append(buf, n);
  std::fclose(f);
  long long ver = 0;
  if (text.find("\"format\": \"bsmm-tune\"") == std::string::npos || !json_int(text, "version", ver) ||
      ver != kTuneCacheVersion)
    return out;
  size_t pos = 0;
  while (pos < text.size()) {
    size_t eol = text.find('\n', pos);
    if (eol == std::string::npos) eol = text.size();
    const std::string line = text.substr(pos, eol - pos);
    pos = eol + 1;
    const size_t k = line.find("\"key\": \"");
    if (k == std::string::npos) continue;
    const size_t k0 = k + 8, k1 = line.find('"', k0);
    if (k1 == std::string::npos) continue;
    TuneEntry e;
    e.key = line.substr(k0, k1 - k0);
    long long cl = 0, st = 0, ft = 0, sw = 0, ms = 0;
    if (!json_int(line, "cluster", cl) || !json_int(line, "stages", st) || !json_int(line, "fp64_tile", ft) ||
        !json_int(line, "store_warps", sw))
      continue;
    json_int(line, "ms_x1000", ms);
    e.t = {(int32_t)cl, (int32_t)st, (int32_t)ft, (int32_t)sw};
    e.ms = ms / 1000.0;
    out.push_back(e);
  }
  return out;
}

bool write_tune_cache(const char* path, const std::vector<TuneEntry>& entries) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  std::fprintf(f, "{\"format\": \"bsmm-tune\", \"version\": %d, \"entries\": [\n", kTuneCacheVersion);
  for (size_t i = 0; i < entries.size(); i++) {
    const TuneEntry& e = entries[i];
    std::fprintf(f,
                 " {\"key\": \"%s\", \"cluster\": %d, \"stages\": %d, \"fp64_tile\": %d, \"store_warps\": %d, "
                 "\"ms_x1000\": %lld}%s\n",
                 e.key.c_str(), e.t.cluster, e.t.stages, e.t.fp64_tile, e.t.store_warps,
                 (long long)std::llround(e.ms * 1000.0), i + 1 < entries.size() ? "," : "");
  }
  std::fprintf(f, "]}\n");
  const bool ok = std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

bsmm_status bsmm_batch_create(bsmm_batch_t* out, int32_t count, const bsmm_plan_t* plans) {
  if (!out) return set_error("out is NULL"), BSMM_ERR_INVALID;
  *out = nullptr;
  if (count <= 0 || !plans) return set_error("a batch needs at least one plan"), BSMM_ERR_INVALID;
  for (int32_t i = 0; i < count; i++)
    if (!plans[i]) return set_error("NULL plan in batch"), BSMM_ERR_INVALID;
  const bsmm_plan_s* p0 = plans[0];
  for (int32_t i = 1; i < count; i++) {
    const bsmm_plan_s* p = plans[i];
    if (p->opt.mode != p0->opt.mode || p->s != p0->s || p->cl != p0->cl || p->stages != p0->stages)
      return set_error("all plans of a batch need the same mode, slice count and cluster size"), BSMM_ERR_INVALID;
    if (p->opt.mode == BSMM_FP64 && p->f64_tile != p0->f64_tile)
      return set_error("all FP64 plans of a batch need the same sub-tile edge (set bsmm_options.fp64_tile)"),
             BSMM_ERR_INVALID;
    if (p->device != p0->device) return set_error("all plans of a batch need the same device"), BSMM_ERR_INVALID;
  }
  bsmm_batch_s* b = new (std::nothrow) bsmm_batch_s();
  if (!b) return set_error("out of host memory"), BSMM_ERR_NOMEM;
  b->plans.assign(plans, plans + count);
  b->mode = p0->opt.mode;
  b->s = p0->s;
  b->cl = p0->cl;
  b->stages = p0->stages;
  for (int32_t i = 0; i < count; i++) {
    const bsmm_plan_s* p = plans[i];
    b->prod_begin.push_back((int64_t)b->unit_prod.size());
    for (int64_t u = 0; u < p->n_units; u++) {
      b->unit_prod.push_back(i);
      b->unit_local.push_back((int32_t)u);
      b->cost.push_back(p->cost[u]);
    }
    b->useful_flops += p->useful_flops;
  }
  b->n_units = (int64_t)b->unit_prod.size();
  b->prod_begin.push_back(b->n_units);
  // the kernel form of the batch's contraction launches: without store warps only when
  // every plan asks for that
  {
    bool none = true;
    for (int32_t i = 0; i < count; i++) none = none && plans[i]->opt.store_warps == 1;
    b->sw = none ? 0 : 1;
  }
  // one product's default bin count describes the machine (CTAs or clusters)
  bsmm_plan_s tmp_view = bsmm_plan_s();
  tmp_view.opt = p0->opt;
  tmp_view.opt.max_ctas = 0;
  tmp_view.sms = p0->sms;
  tmp_view.s = p0->s;
  tmp_view.cl = p0->cl;
  tmp_view.stages = p0->stages;
  tmp_view.sw = b->sw;
  tmp_view.n_units = std::max<int64_t>(1, b->n_units);
  b->bins = default_bins(&tmp_view);
  // waves (see bsmm_batch_s)
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, p0->device) != cudaSuccess || l2 <= 0) l2 = 64 << 20;
  const int64_t budget = (int64_t)l2 / 2;
  b->wave_prod.push_back(0);
  int64_t used = 0;
  for (int32_t i = 0; i < count; i++) {
    const int64_t ws = b->mode == BSMM_FP64 ? 0 : plans[i]->apk_bytes + plans[i]->bpk_bytes;
    if (i > b->wave_prod.back() && used + ws > budget) {
      b->wave_prod.push_back(i);
      used = 0;
    }
    used += ws;
  }
  b->wave_prod.push_back(count);
  for (size_t w = 0; w + 1 < b->wave_prod.size(); w++) {
    const int64_t nu = b->prod_begin[b->wave_prod[w + 1]] - b->prod_begin[b->wave_prod[w]];
    b->wave_bins.push_back((int32_t)std::max<int64_t>(1, std::min<int64_t>(b->bins, nu)));
  }
  bsmm_status st;
  if ((st = put(b->d_unit_prod, b->unit_prod)) != BSMM_OK || (st = put(b->d_unit_local, b->unit_local)) != BSMM_OK ||
      (st = repack(b)) != BSMM_OK || (st = dalloc(b->d_err, sizeof(int32_t))) != BSMM_OK) {
    free_batch(b);
    return st;
  }
  if (cudaMemset(b->d_err.p, 0, sizeof(int32_t)) != cudaSuccess) {
    free_batch(b);
    return set_error("cudaMemset failed"), BSMM_ERR_CUDA;
  }
  if (b->mode != BSMM_FP64 && b->wave_bins.size() >= 2) {
    cudaError_t e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      free_batch(b);
      return set_error(std::string("batch stream: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
    }
  }
  *out = b;
  return BSMM_OK;
}

bsmm_status bsmm_batch_set_args(bsmm_batch_t b, const double* alpha, const void* const* A,
                                const int64_t* const* a_off, const void* const* B, const int64_t* const* b_off,
                                const double* beta, void* const* C, const int64_t* const* c_off) {
  if (!b || !alpha || !beta || !A || !a_off || !B || !b_off || !C || !c_off)
    return set_error("NULL argument array"), BSMM_ERR_INVALID;
  const size_t n = b->plans.size();
  if (b->mode == BSMM_FP64) {
    b->fargs.assign(n, Fp64Args{});
    for (size_t i = 0; i < n; i++) {
      fill_fp64_args(b->plans[i], b->fargs[i], alpha[i], (const double*)A[i], a_off[i], (const double*)B[i], b_off[i],
                     beta[i], (double*)C[i], c_off[i]);
      b->fargs[i].timings = nullptr;
      b->fargs[i].unit_cta = nullptr;
    }
    bsmm_status st = put(b->d_prods, b->fargs);
    if (st != BSMM_OK) return st;
  } else {
    b->sargs.assign(n, SplitArgs{});
    for (size_t i = 0; i < n; i++) {
      // float32 elements take alpha and beta in float32, as bsmm_execute_f32 does
      const bool f32 = b->plans[i]->opt.elem == BSMM_F32;
      fill_split_args(b->plans[i], b->sargs[i], f32 ? (double)(float)alpha[i] : alpha[i], A[i], a_off[i], B[i],
                      b_off[i], f32 ? (double)(float)beta[i] : beta[i], C[i], c_off[i]);
      b->sargs[i].timings = nullptr;
      b->sargs[i].unit_cta = nullptr;
    }
    bsmm_status st = put(b->d_prods, b->sargs);
    if (st != BSMM_OK) return st;
  }
  b->args_set = true;
  return BSMM_OK;
}

bsmm_status bsmm_batch_execute(bsmm_batch_t b, void* stream) {
  if (!b) return set_error("batch is NULL"), BSMM_ERR_INVALID;
  if (!b->args_set) return set_error("bsmm_batch_set_args has not been called"), BSMM_ERR_INVALID;
  if (b->n_units == 0) return BSMM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  int32_t n = 0;
  if (b->side) {  // the second stream starts after everything the caller enqueued before
    e = cudaEventRecord(b->fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
  }
  int32_t nw = 0;  // waves with units so far
  for (size_t w = 0; w + 1 < b->wave_prod.size() && e == cudaSuccess; w++) {
    if (b->prod_begin[b->wave_prod[w + 1]] == b->prod_begin[b->wave_prod[w]]) continue;  // no units
    const cudaStream_t ws = b->side && (nw++ & 1) ? b->side : st;
    const int32_t* sp = (const int32_t*)b->d_sched_ptr.p + b->wave_ptr[w];
    if (b->mode == BSMM_FP64) {
      Fp64Args a = b->fargs[0];
      a.sched_ptr = sp;
      a.sched_units = (const int32_t*)b->d_sched_units.p;
      a.prods = (const Fp64Args*)b->d_prods.p;
      a.unit_prod = (const int32_t*)b->d_unit_prod.p;
      a.unit_local = (const int32_t*)b->d_unit_local.p;
      a.err = (int32_t*)b->d_err.p;
      e = launch_fp64(a, b->wave_bins[w], st, nullptr, nullptr);
      n++;
      // split k: the reductions of the products that cut a k-list
      for (size_t i = 0; i < b->fargs.size() && e == cudaSuccess; i++)
        if (b->fargs[i].n_red > 0) {
          e = launch_fp64_reduce(b->fargs[i], st);
          n++;
        }
    } else {
      for (int32_t i = b->wave_prod[w]; i < b->wave_prod[w + 1] && e == cudaSuccess; i++) {
        int k = 0;
        e = launch_split_prep(b->sargs[i], ws, nullptr, &k);
        n += split_prep_kernels(b->sargs[i]);
      }
      if (e != cudaSuccess) break;
      SplitArgs a = b->sargs[0];
      a.sw = b->sw;
      a.deep = 0;  // the DEEP form when any product of the wave has a deep inner block
      for (int32_t i = b->wave_prod[w]; i < b->wave_prod[w + 1]; i++) a.deep |= b->sargs[i].deep;
      // the epilogue's way of learning the groups (one kernel form per launch): the one
      // most of the wave's units ask for; either gives the same bits
      {
        int64_t walk = 0;
        for (int32_t i = b->wave_prod[w]; i < b->wave_prod[w + 1]; i++)
          if (b->sargs[i].epi_walk) walk += b->prod_begin[i + 1] - b->prod_begin[i];
        a.epi_walk = 2 * walk >= b->prod_begin[b->wave_prod[w + 1]] - b->prod_begin[b->wave_prod[w]] ? 1 : 0;
      }
      a.sched_ptr = sp;
      a.sched_units = (const int32_t*)b->d_sched_units.p;
      a.prods = (const SplitArgs*)b->d_prods.p;
      a.unit_prod = (const int32_t*)b->d_unit_prod.p;
      a.unit_local = (const int32_t*)b->d_unit_local.p;
      a.err = (int32_t*)b->d_err.p;
      e = launch_split_mma(a, b->wave_bins[w], ws);
      n++;
      for (int32_t i = b->wave_prod[w]; i < b->wave_prod[w + 1] && e == cudaSuccess; i++)
        if (b->sargs[i].n_red > 0) {
          e = launch_split_reduce(b->sargs[i], ws);
          n++;
        }
    }
  }
  if (b->side) {  // join: the caller's stream continues after both streams' waves
    const cudaError_t j = cudaEventRecord(b->join, b->side);
    const cudaError_t k = j == cudaSuccess ? cudaStreamWaitEvent(st, b->join, 0) : j;
    if (e == cudaSuccess) e = k;
  }
  if (e != cudaSuccess) return set_error(std::string("batch launch: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  b->launches = n;
  return BSMM_OK;
}

}  // extern "C"

namespace {

// bsmm_execute_batch keeps the batch objects of its last few plan lists: keyed by the
// plans' unique ids (a destroyed plan's id never comes back, so a stale entry never
// matches), with the arguments last uploaded to each.
struct OneCall {
  std::vector<uint64_t> uids;
  bsmm_batch_t batch = nullptr;
  std::vector<double> alpha, beta;
  std::vector<const void*> ptrs;  // A, a_off, B, b_off, C, c_off of every product
  uint64_t used = 0;
};
constexpr size_t kOneCallEntries = 4;
std::mutex g_one_mu;
std::vector<OneCall>* g_one = new std::vector<OneCall>();  // never destroyed: no CUDA call at exit
uint64_t g_one_clock = 0;

}  // namespace

extern "C" {

bsmm_status bsmm_execute_batch(int32_t count, const bsmm_plan_t* plans, const double* alpha, const void* const* A,
                               const int64_t* const* a_off, const void* const* B, const int64_t* const* b_off,
                               const double* beta, void* const* C, const int64_t* const* c_off, void* stream) {
  if (count <= 0 || !plans || !alpha || !beta || !A || !a_off || !B || !b_off || !C || !c_off)
    return set_error("bsmm_execute_batch: NULL argument or count <= 0"), BSMM_ERR_INVALID;
  std::vector<uint64_t> uids(count);
  for (int32_t i = 0; i < count; i++) {
    if (!plans[i]) return set_error("bsmm_execute_batch: NULL plan"), BSMM_ERR_INVALID;
    uids[i] = plans[i]->uid;
  }
  std::lock_guard<std::mutex> lk(g_one_mu);
  std::vector<OneCall>& cache = *g_one;
  OneCall* hit = nullptr;
  for (OneCall& e : cache)
    if (e.uids == uids) hit = &e;
  cudaStream_t st = (cudaStream_t)stream;
  if (!hit) {
    bsmm_batch_t b = nullptr;
    const bsmm_status s = bsmm_batch_create(&b, count, plans);
    if (s != BSMM_OK) return s;
    if (cache.size() >= kOneCallEntries) {  // the least recently used entry makes room
      auto lru = std::min_element(cache.begin(), cache.end(),
                                  [](const OneCall& x, const OneCall& y) { return x.used < y.used; });
      if (cudaStreamSynchronize(st) != cudaSuccess) {
        bsmm_batch_destroy(b);
        return set_error("bsmm_execute_batch: stream synchronisation failed"), BSMM_ERR_CUDA;
      }
      bsmm_batch_destroy(lru->batch);
      cache.erase(lru);
    }
    cache.push_back(OneCall{uids, b, {}, {}, {}, 0});
    hit = &cache.back();
  }
  hit->used = ++g_one_clock;
  std::vector<double> al(alpha, alpha + count), be(beta, beta + count);
  std::vector<const void*> ptrs;
  ptrs.reserve(6 * (size_t)count);
  for (int32_t i = 0; i < count; i++)
    for (const void* x : {(const void*)A[i], (const void*)a_off[i], (const void*)B[i], (const void*)b_off[i],
                          (const void*)C[i], (const void*)c_off[i]})
      ptrs.push_back(x);
  if (al != hit->alpha || be != hit->beta || ptrs != hit->ptrs) {
    // new arguments: the table the previous launch of this batch reads is replaced only
    // after that launch (on this stream) has finished
    if (!hit->ptrs.empty() && cudaStreamSynchronize(st) != cudaSuccess)
      return set_error("bsmm_execute_batch: stream synchronisation failed"), BSMM_ERR_CUDA;
    const bsmm_status s = bsmm_batch_set_args(hit->batch, alpha, A, a_off, B, b_off, beta, C, c_off);
    if (s != BSMM_OK) {
      hit->ptrs.clear();
      return s;
    }
    hit->alpha = al;
    hit->beta = be;
    hit->ptrs = ptrs;
  }
  return bsmm_batch_execute(hit->batch, stream);
}

bsmm_status bsmm_batch_kernels(bsmm_batch_t b, int32_t* kernels) {
  if (!b || !kernels) return set_error("NULL argument"), BSMM_ERR_INVALID;
  *kernels = b->launches;
  return BSMM_OK;
}

bsmm_status bsmm_batch_query(bsmm_batch_t b, int64_t* n_units, double* useful_flops, int32_t* bins) {
  if (!b) return set_error("batch is NULL"), BSMM_ERR_INVALID;
  if (n_units) *n_units = b->n_units;
  if (useful_flops) *useful_flops = b->useful_flops;
  if (bins) *bins = b->bins;
  return BSMM_OK;
}

bsmm_status bsmm_batch_set_costs(bsmm_batch_t b, const double* costs) {
  if (!b || !costs) return set_error("NULL argument"), BSMM_ERR_INVALID;
  for (int64_t u = 0; u < b->n_units; u++)
    if (!(costs[u] > 0.0)) return set_error("costs must be > 0"), BSMM_ERR_INVALID;
  b->cost.assign(costs, costs + b->n_units);
  return repack(b);
}

bsmm_status BatchArgs::set(bsmm_batch_t b, const std::vector<void*>& Cs) const {
  return bsmm_batch_set_args(b, alpha.data(), A.data(), ao.data(), B.data(), bo.data(), beta.data(), Cs.data(),
                             co.data());
}

bsmm_status bsmm_tune_space(int32_t mode, int32_t nslices, bsmm_tune_point* out, int32_t cap, int32_t* count) {
  if (!count) return set_error("count is NULL"), BSMM_ERR_INVALID;
  std::vector<bsmm_tune_point> v;
  if (mode == BSMM_FP64) {
    v.push_back({0, 0, 32, 0});
    v.push_back({0, 0, 64, 0});
  } else if (mode == BSMM_SPLIT_BF16 || mode == BSMM_SPLIT_FP16) {
    if (nslices < 1 || nslices > kSplitMaxS) return set_error("nslices must be in 1..6"), BSMM_ERR_INVALID;
    for (int cl : {1, 2, 4})
      for (int st = 2; st <= 8; st++)
        for (int sw : {1, 2})
          if (split_smem_bytes(nslices, split_tile_n(nslices), st) <= kMaxSmemPerCta) v.push_back({cl, st, 0, sw});
  } else {
    return set_error("unknown mode"), BSMM_ERR_INVALID;
  }
  *count = (int32_t)v.size();
  if (out)
    for (int32_t i = 0; i < std::min<int32_t>(cap, *count); i++) out[i] = v[i];
  return BSMM_OK;
}

bsmm_status bsmm_batch_autotune(bsmm_batch_t b, int32_t n, const bsmm_tune_point* cand, int32_t reps, void* stream,
                                int32_t* chosen, float* ms) {
  if (!b || !cand || n <= 0 || reps < 1) return set_error("batch, candidates and reps >= 1 are required"), BSMM_ERR_INVALID;
  if (!b->args_set) return set_error("bsmm_batch_set_args has not been called"), BSMM_ERR_INVALID;
  for (int32_t c = 0; c < n; c++) {
    const bsmm_tune_point& t = cand[c];
    const bool ok = b->mode == BSMM_FP64
                        ? (t.cluster == 0 && t.stages == 0 && t.store_warps == 0 && (t.fp64_tile == 32 || t.fp64_tile == 64))
                        : (t.fp64_tile == 0 && (t.cluster == 1 || t.cluster == 2 || t.cluster == 4) &&
                           (t.stages == 0 || (t.stages >= 2 && t.stages <= 8)) && t.store_warps >= 0 && t.store_warps <= 2);
    if (!ok) return set_error("candidate " + std::to_string(c) + " does not fit the batch's mode"), BSMM_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const BatchArgs args(b);
  const size_t count = b->plans.size();
  // scratch C per product, as long as the caller's C extent
  std::vector<DevBuf> scratch(count);
  std::vector<void*> scratch_c(count);
  bsmm_status res = BSMM_OK;
  auto cleanup_scratch = [&]() {
    for (DevBuf& d : scratch)
      if (d.p) cudaFree(d.p);
  };
  for (size_t i = 0; i < count && res == BSMM_OK; i++) {
    const bsmm_plan_s* p = b->plans[i];
    std::vector<int64_t> off((size_t)p->M * p->N);
    if (!off.empty() && cudaMemcpy(off.data(), args.co[i], sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
      res = (set_error("reading c_off failed"), BSMM_ERR_CUDA);
      break;
    }
    // the C extent in elements of the plan's type (a complex plan's column tiling counts
    // both parts of each complex column)
    const bool cplx = p->opt.elem == BSMM_C128;
    const size_t es = p->opt.elem == BSMM_F32 ? sizeof(float) : cplx ? 2 * sizeof(double) : sizeof(double);
    int64_t extent = 1;
    for (int ii = 0; ii < p->M; ii++)
      for (int jj = 0; jj < p->N; jj++) {
        const size_t t = (size_t)ii * p->N + jj;
        const int64_t cols = cplx ? p->c[jj] / 2 : p->c[jj];
        if (p->cs[t] && off[t] >= 0) extent = std::max<int64_t>(extent, off[t] + (int64_t)p->r[ii] * cols);
      }
    if ((res = dalloc(scratch[i], es * extent)) != BSMM_OK) break;
    if (cudaMemset(scratch[i].p, 0, es * extent) != cudaSuccess) res = (set_error("cudaMemset failed"), BSMM_ERR_CUDA);
    scratch_c[i] = scratch[i].p;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (res == BSMM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    res = (set_error("cudaEventCreate failed"), BSMM_ERR_CUDA);
  int best = -1;
  float best_ms = std::numeric_limits<float>::infinity();
  for (int32_t c = 0; c < n && res == BSMM_OK; c++) {
    float med = std::numeric_limits<float>::infinity();
    std::vector<bsmm_plan_t> plans;
    bsmm_status s = replan(b, cand[c], plans);
    if (s == BSMM_ERR_UNSUPPORTED) {  // this candidate does not fit (e.g. the ring in shared memory)
      if (ms) ms[c] = med;
      continue;
    }
    if (s != BSMM_OK) {
      res = s;
      break;
    }
    bsmm_batch_t tb = nullptr;
    s = bsmm_batch_create(&tb, (int32_t)count, plans.data());
    if (s == BSMM_OK) s = args.set(tb, scratch_c);
    if (s == BSMM_OK) s = bsmm_batch_execute(tb, stream);  // warm-up
    std::vector<float> t;
    for (int r = 0; r < reps && s == BSMM_OK; r++) {
      cudaEventRecord(e0, st);
      s = bsmm_batch_execute(tb, stream);
      cudaEventRecord(e1, st);
      float x = 0.0f;
      if (s == BSMM_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&x, e0, e1) != cudaSuccess))
        s = (set_error("timing the candidate failed"), BSMM_ERR_CUDA);
      t.push_back(x);
    }
    if (s == BSMM_OK) s = bsmm_batch_status_device(tb, stream);
    if (tb) bsmm_batch_destroy(tb);
    for (bsmm_plan_t q : plans) bsmm_destroy(q);
    if (s != BSMM_OK) {
      res = s;
      break;
    }
    std::sort(t.begin(), t.end());
    med = t[t.size() / 2];
    if (ms) ms[c] = med;
    if (med < best_ms) {
      best_ms = med;
      best = c;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cleanup_scratch();
  if (res != BSMM_OK) return res;
  if (best < 0) return set_error("no candidate fits"), BSMM_ERR_UNSUPPORTED;
  const bsmm_status s = adopt(b, cand[best]);
  if (s != BSMM_OK) return s;
  if (chosen) *chosen = best;
  return BSMM_OK;
}

bsmm_status bsmm_batch_autotune_cached(bsmm_batch_t b, const char* cache_path, int32_t reps, void* stream,
                                       bsmm_tune_point* chosen, int32_t* from_cache) {
  if (!b || !cache_path || !*cache_path || reps < 1)
    return set_error("batch, cache path and reps >= 1 are required"), BSMM_ERR_INVALID;
  if (!b->args_set) return set_error("bsmm_batch_set_args has not been called"), BSMM_ERR_INVALID;
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, b->plans[0]->device) != cudaSuccess)
    return set_error("cudaGetDeviceProperties failed"), BSMM_ERR_CUDA;
  std::string gpu = prop.name;
  for (char& ch : gpu)
    if (ch == '"' || ch == '\\' || ch == '|' || ch == '\n') ch = '_';
  const char* mode = b->mode == BSMM_FP64 ? "fp64" : b->mode == BSMM_SPLIT_FP16 ? "split_fp16" : "split_bf16";
  const std::string key = gpu + "|" + mode + "|s=" + std::to_string(b->mode == BSMM_FP64 ? 0 : b->s);
  std::vector<TuneEntry> entries = read_tune_cache(cache_path);
  int32_t n = 0;
  bsmm_status s = bsmm_tune_space(b->mode, b->mode == BSMM_FP64 ? 6 : b->s, nullptr, 0, &n);
  if (s != BSMM_OK) return s;
  std::vector<bsmm_tune_point> space(n);
  bsmm_tune_space(b->mode, b->mode == BSMM_FP64 ? 6 : b->s, space.data(), n, &n);
  for (const TuneEntry& e : entries) {
    if (e.key != key) continue;
    // a cached choice is used only while it is still one of the library's candidates
    const bool valid = std::any_of(space.begin(), space.end(), [&](const bsmm_tune_point& t) {
      return t.cluster == e.t.cluster && t.stages == e.t.stages && t.fp64_tile == e.t.fp64_tile &&
             t.store_warps == e.t.store_warps;
    });
    if (!valid) break;
    s = adopt(b, e.t);
    if (s != BSMM_OK) return s;
    if (chosen) *chosen = e.t;
    if (from_cache) *from_cache = 1;
    return BSMM_OK;
  }
  std::vector<float> ms(n);
  int32_t best = -1;
  s = bsmm_batch_autotune(b, n, space.data(), reps, stream, &best, ms.data());
  if (s != BSMM_OK) return s;
  entries.erase(std::remove_if(entries.begin(), entries.end(), [&](const TuneEntry& e) { return e.key == key; }),
                entries.end());
  entries.push_back({key, space[best], ms[best]});
  if (!write_tune_cache(cache_path, entries))
    return set_error(std::string("cannot write the tuning cache ") + cache_path), BSMM_ERR_INVALID;
  if (chosen) *chosen = space[best];
  if (from_cache) *from_cache = 0;
  return BSMM_OK;
}

bsmm_status bsmm_batch_status_device(bsmm_batch_t b, void* stream) {
  if (!b) return set_error("batch is NULL"), BSMM_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, b->d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err.p, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(std::string("status: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  if (w & kErrTimeout) return set_error("a kernel wait timed out"), BSMM_ERR_TIMEOUT;
  if (w) return set_error("a kernel check failed"), BSMM_ERR_DEVICE;
  for (bsmm_plan_t p : b->plans) {
    bsmm_status s = bsmm_status_device(p, stream);
    if (s != BSMM_OK) return s;
  }
  return BSMM_OK;
}

void bsmm_batch_destroy(bsmm_batch_t b) {
  if (b) free_batch(b);
}

}  // extern "C"
