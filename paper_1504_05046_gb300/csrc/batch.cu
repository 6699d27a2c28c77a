// Many independent block-sparse products in one persistent launch.
//
// The paper schedules the tasks of one product over a process grid (Sec. 3.2); a
// batch is the same idea across products: the work units of every product form one
// task set, packed longest-processing-time first onto the persistent CTAs (FP64)
// or clusters (split modes) of a single contraction launch, so short products fill
// the gaps left by long ones instead of each paying a launch and a tail. Each unit
// reads its product's arguments from a device table. The per-product preparation
// (exponents and slices, split modes only) is issued as ordinary kernels before the
// contraction. bsmm_batch_execute issues kernels only, so a stream capture of it
// records a CUDA graph that replays the whole batch with one graph launch.
#include <cstring>

#include "bsmm_internal.h"

using namespace bsmm;

struct bsmm_batch_s {
  std::vector<bsmm_plan_t> plans;
  int mode = 0, s = 0, cl = 1, stages = 0;
  int64_t n_units = 0;
  double useful_flops = 0.0;
  std::vector<int32_t> unit_prod, unit_local;
  std::vector<double> cost;
  int bins = 0;
  std::vector<int32_t> sched_ptr, sched_units;
  std::vector<Fp64Args> fargs;
  std::vector<SplitArgs> sargs;
  bool args_set = false;
  DevBuf d_prods, d_unit_prod, d_unit_local, d_sched_ptr, d_sched_units, d_err;
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
  lpt_pack(b->cost, b->bins, false, b->sched_ptr, b->sched_units);
  bsmm_status st;
  if ((st = put(b->d_sched_ptr, b->sched_ptr)) != BSMM_OK) return st;
  return put(b->d_sched_units, b->sched_units);
}

void free_batch(bsmm_batch_s* b) {
  for (DevBuf* d : {&b->d_prods, &b->d_unit_prod, &b->d_unit_local, &b->d_sched_ptr, &b->d_sched_units, &b->d_err})
    if (d->p) cudaFree(d->p);
  delete b;
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
    for (int64_t u = 0; u < p->n_units; u++) {
      b->unit_prod.push_back(i);
      b->unit_local.push_back((int32_t)u);
      b->cost.push_back(p->cost[u]);
    }
    b->useful_flops += p->useful_flops;
  }
  b->n_units = (int64_t)b->unit_prod.size();
  // one product's default bin count describes the machine (CTAs or clusters)
  bsmm_plan_s tmp_view = bsmm_plan_s();
  tmp_view.opt = p0->opt;
  tmp_view.opt.max_ctas = 0;
  tmp_view.sms = p0->sms;
  tmp_view.s = p0->s;
  tmp_view.cl = p0->cl;
  tmp_view.stages = p0->stages;
  tmp_view.n_units = std::max<int64_t>(1, b->n_units);
  b->bins = default_bins(&tmp_view);
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
  *out = b;
  return BSMM_OK;
}

bsmm_status bsmm_batch_set_args(bsmm_batch_t b, const double* alpha, const double* const* A,
                                const int64_t* const* a_off, const double* const* B, const int64_t* const* b_off,
                                const double* beta, double* const* C, const int64_t* const* c_off) {
  if (!b || !alpha || !beta || !A || !a_off || !B || !b_off || !C || !c_off)
    return set_error("NULL argument array"), BSMM_ERR_INVALID;
  const size_t n = b->plans.size();
  if (b->mode == BSMM_FP64) {
    b->fargs.assign(n, Fp64Args{});
    for (size_t i = 0; i < n; i++) {
      fill_fp64_args(b->plans[i], b->fargs[i], alpha[i], A[i], a_off[i], B[i], b_off[i], beta[i], C[i], c_off[i]);
      b->fargs[i].timings = nullptr;
      b->fargs[i].unit_cta = nullptr;
    }
    bsmm_status st = put(b->d_prods, b->fargs);
    if (st != BSMM_OK) return st;
  } else {
    b->sargs.assign(n, SplitArgs{});
    for (size_t i = 0; i < n; i++) {
      fill_split_args(b->plans[i], b->sargs[i], alpha[i], A[i], a_off[i], B[i], b_off[i], beta[i], C[i], c_off[i]);
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
  cudaError_t e;
  if (b->mode == BSMM_FP64) {
    Fp64Args a = b->fargs[0];
    a.sched_ptr = (const int32_t*)b->d_sched_ptr.p;
    a.sched_units = (const int32_t*)b->d_sched_units.p;
    a.prods = (const Fp64Args*)b->d_prods.p;
    a.unit_prod = (const int32_t*)b->d_unit_prod.p;
    a.unit_local = (const int32_t*)b->d_unit_local.p;
    a.err = (int32_t*)b->d_err.p;
    e = launch_fp64(a, b->bins, st, nullptr, nullptr);
  } else {
    for (const SplitArgs& pa : b->sargs) {
      int k = 0;
      e = launch_split_prep(pa, st, nullptr, &k);
      if (e != cudaSuccess) return set_error(std::string("batch prep: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
    }
    SplitArgs a = b->sargs[0];
    a.sched_ptr = (const int32_t*)b->d_sched_ptr.p;
    a.sched_units = (const int32_t*)b->d_sched_units.p;
    a.prods = (const SplitArgs*)b->d_prods.p;
    a.unit_prod = (const int32_t*)b->d_unit_prod.p;
    a.unit_local = (const int32_t*)b->d_unit_local.p;
    a.err = (int32_t*)b->d_err.p;
    e = launch_split_mma(a, b->bins, st);
  }
  if (e != cudaSuccess) return set_error(std::string("batch launch: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
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
