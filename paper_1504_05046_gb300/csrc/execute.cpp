// C ABI: execution entry points, device status, timing records.
#include <algorithm>
#include <cstring>

#include "bsmm_internal.h"

using namespace bsmm;

namespace bsmm {

void fill_fp64_args(bsmm_plan_s* p, Fp64Args& a, double alpha, const double* A, const int64_t* a_off,
                    const double* B, const int64_t* b_off, double beta, double* C, const int64_t* c_off) {
  a.r = (const int32_t*)p->d_r.p;
  a.c = (const int32_t*)p->d_c.p;
  a.q = (const int32_t*)p->d_q.p;
  a.M = p->M;
  a.N = p->N;
  a.K = p->K;
  a.kptr = (const int64_t*)p->d_kptr.p;
  a.klist = (const int32_t*)p->d_klist.p;
  a.cs = (const uint8_t*)p->d_cs.p;
  a.units = (const Fp64Unit*)p->d_units.p;
  a.sched_ptr = (const int32_t*)p->d_sched_ptr.p;
  a.sched_units = (const int32_t*)p->d_sched_units.p;
  a.alpha = alpha;
  a.beta = beta;
  a.A = A;
  a.a_off = a_off;
  a.B = B;
  a.b_off = b_off;
  a.C = C;
  a.c_off = c_off;
  a.timings = p->opt.record_timings ? (int64_t*)p->d_timings.p : nullptr;
  a.unit_cta = p->opt.record_timings ? (int32_t*)p->d_unit_cta.p : nullptr;
  a.err = (int32_t*)p->d_err.p;
  a.debug = p->opt.debug_checks;
  a.tile = p->f64_tile;
  a.transa = p->opt.transa;
  a.transb = p->opt.transb;
  a.part = (double*)p->d_part.p;
  a.red = (const Fp64Red*)p->d_red.p;
  a.n_red = (int32_t)p->f64_red.size();
  a.prods = nullptr;
  a.unit_prod = a.unit_local = nullptr;
}

void fill_split_args(bsmm_plan_s* p, SplitArgs& a, double alpha, const void* A, const int64_t* a_off,
                     const void* B, const int64_t* b_off, double beta, void* C, const int64_t* c_off) {
  a.M = p->M;
  a.N = p->N;
  a.K = p->K;
  a.s = p->s;
  a.tn = p->tn;
  a.stages = p->stages;
  a.fp16 = p->opt.mode == BSMM_SPLIT_FP16;
  a.Mtot = p->Mtot;
  a.Ntot = p->Ntot;
  a.RB = p->RB;
  a.CB = p->CB;
  a.kwords = p->kwords;
  a.r = (const int32_t*)p->d_r.p;
  a.c = (const int32_t*)p->d_c.p;
  a.q = (const int32_t*)p->d_q.p;
  a.ro = (const int64_t*)p->d_ro.p;
  a.co = (const int64_t*)p->d_co.p;
  a.row_tile = (const int32_t*)p->d_row_tile.p;
  a.col_tile = (const int32_t*)p->d_col_tile.p;
  a.cs = (const uint8_t*)p->d_cs.p;
  a.am = (const uint8_t*)p->d_am.p;
  a.bm = (const uint8_t*)p->d_bm.p;
  a.presA = (const uint64_t*)p->d_presA.p;
  a.presB = (const uint64_t*)p->d_presB.p;
  a.presBg = (const uint64_t*)p->d_presBg.p;
  a.cl = p->cl;
  a.CBG = p->CBG;
  a.apk_off = (const int64_t*)p->d_apk_off.p;
  a.bpk_off = (const int64_t*)p->d_bpk_off.p;
  a.apk = (uint8_t*)p->d_apk.p;
  a.bpk = (uint8_t*)p->d_bpk.p;
  a.rowexp = (int16_t*)p->d_rowexp.p;
  a.colexp = (int16_t*)p->d_colexp.p;
  a.colexp_ld = p->colexp_ld;
  a.urow = (int16_t*)p->d_urow.p;
  a.ucol = (int16_t*)p->d_ucol.p;
  a.rowadj = (int16_t*)p->d_rowadj.p;
  a.coladj = (int16_t*)p->d_coladj.p;
  a.emaxr = (int32_t*)p->d_emaxr.p;
  a.emaxc = (int32_t*)p->d_emaxc.p;
  a.kdepth = split_max_depth(p->s);
  a.transa = p->opt.transa;
  a.transb = p->opt.transb;
  a.rowscale = p->opt.split_scale;
  a.eArow = (int32_t*)p->d_eArow.p;
  a.eBcol = (int32_t*)p->d_eBcol.p;
  a.eAmaxr = (int32_t*)p->d_eAmaxr.p;
  a.eBmaxc = (int32_t*)p->d_eBmaxc.p;
  a.eA = (int32_t*)p->d_eA.p;
  a.eB = (int32_t*)p->d_eB.p;
  a.eAmax = (int32_t*)p->d_eAmax.p;
  a.eBmax = (int32_t*)p->d_eBmax.p;
  a.a_tiles = (const int32_t*)p->d_a_tiles.p;
  a.b_tiles = (const int32_t*)p->d_b_tiles.p;
  a.n_a_tiles = p->n_a_tiles;
  a.n_b_tiles = p->n_b_tiles;
  a.a_blocks = (const int32_t*)p->d_a_blocks.p;
  a.b_blocks = (const int32_t*)p->d_b_blocks.p;
  a.n_a_blocks = p->n_a_blocks;
  a.n_b_blocks = p->n_b_blocks;
  a.units = (const SplitUnit*)p->d_units.p;
  a.sched_ptr = (const int32_t*)p->d_sched_ptr.p;
  a.sched_units = (const int32_t*)p->d_sched_units.p;
  a.alpha = alpha;
  a.beta = beta;
  a.sw = p->sw;
  a.epi_walk = p->epi_walk;
  a.deep = p->deep;
  a.f32 = p->opt.elem == BSMM_F32;
  a.cplx = p->opt.elem == BSMM_C128;
  a.A = a.f32 ? nullptr : (const double*)A;
  a.B = a.f32 ? nullptr : (const double*)B;
  a.C = a.f32 ? nullptr : (double*)C;
  a.Af = a.f32 ? (const float*)A : nullptr;
  a.Bf = a.f32 ? (const float*)B : nullptr;
  a.Cf = a.f32 ? (float*)C : nullptr;
  a.a_off = a_off;
  a.b_off = b_off;
  a.c_off = c_off;
  a.timings = p->opt.record_timings ? (int64_t*)p->d_timings.p : nullptr;
  a.unit_cta = p->opt.record_timings ? (int32_t*)p->d_unit_cta.p : nullptr;
  a.err = (int32_t*)p->d_err.p;
  a.debug = p->opt.debug_checks;
  a.part = (uint4*)p->d_part.p;
  a.red = (const SplitRed*)p->d_red.p;
  a.n_red = (int32_t)p->sp_red.size();
  a.prods = nullptr;
  a.unit_prod = a.unit_local = nullptr;
}

}  // namespace bsmm

namespace {

bsmm_status check_ptrs(bsmm_plan_s* p, const void* A, const int64_t* a_off, const void* B,
                       const int64_t* b_off, void* C, const int64_t* c_off) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  if ((int64_t)p->M * p->K && !a_off) return set_error("a_off is NULL"), BSMM_ERR_INVALID;
  if ((int64_t)p->K * p->N && !b_off) return set_error("b_off is NULL"), BSMM_ERR_INVALID;
  if (p->n_ctiles && (!c_off || !C)) return set_error("C or c_off is NULL"), BSMM_ERR_INVALID;
  if (p->n_triples && (!A || !B)) return set_error("A or B is NULL"), BSMM_ERR_INVALID;
  return BSMM_OK;
}

bsmm_status run(bsmm_plan_s* p, double alpha, const void* A, const int64_t* a_off, const void* B,
                const int64_t* b_off, double beta, void* C, const int64_t* c_off, cudaStream_t st) {
  if (p->n_units == 0) return BSMM_OK;
  cudaError_t e;
  cudaEvent_t* ev = nullptr;
  int set = -1;
  if (p->opt.profile) {
    if (!p->ev[0][0])
      for (int r = 0; r < kProfileRing; r++)
        for (int i = 0; i < kMaxEvents; i++)
          if (cudaEventCreate(&p->ev[r][i]) != cudaSuccess) return set_error("cudaEventCreate failed"), BSMM_ERR_CUDA;
    set = p->ev_next;
    ev = p->ev[set];
  }
  int nk = 0;
  // the split kernels take the longest of a group's CTA times with atomicMax
  if (p->opt.record_timings && p->d_timings.p) {
    e = cudaMemsetAsync(p->d_timings.p, 0, p->d_timings.bytes, st);
    if (e != cudaSuccess) return set_error(std::string("timing records: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  }
  if (p->opt.mode == BSMM_FP64) {
    Fp64Args a{};
    fill_fp64_args(p, a, alpha, (const double*)A, a_off, (const double*)B, b_off, beta, (double*)C, c_off);
    e = launch_fp64(a, p->ctas, st, ev, &nk);
  } else {
    SplitArgs a{};
    fill_split_args(p, a, alpha, A, a_off, B, b_off, beta, C, c_off);
    e = launch_split(a, p->ctas, st, ev, &nk);
  }
  if (set >= 0) {
    p->ev_counts[set] = nk;
    p->ev_last = set;
    p->ev_next = (set + 1) % kProfileRing;
    p->ev_pending = std::min(p->ev_pending + 1, kProfileRing);
  }
  if (e != cudaSuccess) {
    set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return BSMM_ERR_CUDA;
  }
  return BSMM_OK;
}

bsmm_status grow(DevBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return BSMM_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BSMM_ERR_NOMEM : BSMM_ERR_CUDA;
  }
  b.bytes = bytes;
  return BSMM_OK;
}


// The host-buffer path (bsmm_execute_host_async): product i uses staging slot i % 2.
//   copy stream in:  [slot's previous contraction done] offsets, A, B; [its copy out done] C
//                    (when beta != 0)                                        -> event in
//   stream:          [in] [slot's previous copy out done] [previous host product's kernels]
//                    the product's kernels                                  -> event run
//   copy stream out: [run] C back to the host                                -> event out
// so the copies of product i + 1 (and the copy out of product i - 1) overlap the
// contraction of product i, and at most two products hold staging memory.
bsmm_status host_setup(bsmm_plan_s* p) {
  if (p->h2d) return BSMM_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->last_run, cudaEventDisableTiming);
  for (auto& h : p->hs) {
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.run, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.out, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    host_release(p);
    return set_error(std::string("host streams: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  }
  return BSMM_OK;
}

bsmm_status enqueue_host(bsmm_plan_s* p, double alpha, const void* A, int64_t a_elems, const int64_t* a_off,
                         const void* B, int64_t b_elems, const int64_t* b_off, double beta, void* C, int64_t c_elems,
                         const int64_t* c_off, cudaStream_t st) {
  bsmm_status s = host_setup(p);
  if (s != BSMM_OK) return s;
  // bytes per element of the plan's element type
  const size_t es = p->opt.elem == BSMM_F32 ? sizeof(float) : p->opt.elem == BSMM_C128 ? 2 * sizeof(double)
                                                                                        : sizeof(double);
  const size_t na = (size_t)p->M * p->K, nb = (size_t)p->K * p->N, nc = (size_t)p->M * p->N;
  bsmm_plan_s::HostSlot& h = p->hs[p->host_count & 1];
  const bool fits = h.A.bytes >= es * a_elems && h.B.bytes >= es * b_elems && h.C.bytes >= es * c_elems &&
                    h.aoff.bytes >= sizeof(int64_t) * na && h.boff.bytes >= sizeof(int64_t) * nb &&
                    h.coff.bytes >= sizeof(int64_t) * nc;
  cudaError_t e = cudaSuccess;
  if (!fits && h.used) e = cudaEventSynchronize(h.out);  // the slot's buffers are about to be replaced
  if (e != cudaSuccess) return set_error(std::string("host slot: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  if ((s = grow(h.A, es * a_elems)) != BSMM_OK) return s;
  if ((s = grow(h.B, es * b_elems)) != BSMM_OK) return s;
  if ((s = grow(h.C, es * c_elems)) != BSMM_OK) return s;
  if ((s = grow(h.aoff, sizeof(int64_t) * na)) != BSMM_OK) return s;
  if ((s = grow(h.boff, sizeof(int64_t) * nb)) != BSMM_OK) return s;
  if ((s = grow(h.coff, sizeof(int64_t) * nc)) != BSMM_OK) return s;
  auto h2d = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes > 0) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, p->h2d);
  };
  if (h.used) e = cudaStreamWaitEvent(p->h2d, h.run, 0);  // the slot's inputs are no longer read
  h2d(h.aoff.p, a_off, sizeof(int64_t) * na);
  h2d(h.boff.p, b_off, sizeof(int64_t) * nb);
  h2d(h.coff.p, c_off, sizeof(int64_t) * nc);
  h2d(h.A.p, A, es * a_elems);
  h2d(h.B.p, B, es * b_elems);
  if (beta != 0.0) {
    if (h.used && e == cudaSuccess) e = cudaStreamWaitEvent(p->h2d, h.out, 0);  // its C went back
    h2d(h.C.p, C, es * c_elems);
  }
  if (e == cudaSuccess) e = cudaEventRecord(h.in, p->h2d);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h.in, 0);
  if (e == cudaSuccess && h.used) e = cudaStreamWaitEvent(st, h.out, 0);  // C is written by this product
  if (e == cudaSuccess && p->host_count > 0) e = cudaStreamWaitEvent(st, p->last_run, 0);  // shared workspaces
  if (e != cudaSuccess) {
    cudaStreamSynchronize(p->h2d);
    return set_error(std::string("H2D: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  }
  const double al = p->opt.elem == BSMM_F32 ? (double)(float)alpha : alpha;
  const double be = p->opt.elem == BSMM_F32 ? (double)(float)beta : beta;
  s = run(p, al, h.A.p, (const int64_t*)h.aoff.p, h.B.p, (const int64_t*)h.boff.p, be, h.C.p,
          (const int64_t*)h.coff.p, st);
  if (s != BSMM_OK) {
    cudaStreamSynchronize(p->h2d);
    cudaStreamSynchronize(st);
    return s;
  }
  e = cudaEventRecord(h.run, st);
  if (e == cudaSuccess) e = cudaEventRecord(p->last_run, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h, h.run, 0);
  if (e == cudaSuccess && c_elems > 0) e = cudaMemcpyAsync(C, h.C.p, es * c_elems, cudaMemcpyDeviceToHost, p->d2h);
  if (e == cudaSuccess) e = cudaEventRecord(h.out, p->d2h);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(p->d2h);
    return set_error(std::string("D2H: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  }
  h.used = true;
  p->host_count++;
  return BSMM_OK;
}

}  // namespace

extern "C" {

bsmm_status bsmm_execute(bsmm_plan_t p, double alpha, const double* A, const int64_t* a_off, const double* B,
                         const int64_t* b_off, double beta, double* C, const int64_t* c_off, void* stream) {
  bsmm_status s = check_ptrs(p, A, a_off, B, b_off, C, c_off);
  if (s != BSMM_OK) return s;
  if (p->opt.elem == BSMM_F32) return set_error("plan has float32 elements: use bsmm_execute_f32"), BSMM_ERR_INVALID;
  return run(p, alpha, A, a_off, B, b_off, beta, C, c_off, (cudaStream_t)stream);
}

bsmm_status bsmm_execute_f32(bsmm_plan_t p, float alpha, const float* A, const int64_t* a_off, const float* B,
                             const int64_t* b_off, float beta, float* C, const int64_t* c_off, void* stream) {
  bsmm_status s = check_ptrs(p, A, a_off, B, b_off, C, c_off);
  if (s != BSMM_OK) return s;
  if (p->opt.elem != BSMM_F32) return set_error("plan has float64 elements: use bsmm_execute"), BSMM_ERR_INVALID;
  return run(p, alpha, A, a_off, B, b_off, beta, C, c_off, (cudaStream_t)stream);
}

bsmm_status bsmm_execute_host_async(bsmm_plan_t p, double alpha, const void* A, int64_t a_elems,
                                    const int64_t* a_off, const void* B, int64_t b_elems, const int64_t* b_off,
                                    double beta, void* C, int64_t c_elems, const int64_t* c_off, void* stream) {
  bsmm_status s = check_ptrs(p, A, a_off, B, b_off, C, c_off);
  if (s != BSMM_OK) return s;
  if (a_elems < 0 || b_elems < 0 || c_elems < 0) return set_error("negative arena length"), BSMM_ERR_INVALID;
  return enqueue_host(p, alpha, A, a_elems, a_off, B, b_elems, b_off, beta, C, c_elems, c_off, (cudaStream_t)stream);
}

bsmm_status bsmm_host_wait(bsmm_plan_t p) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  for (const auto& h : p->hs) {
    if (!h.used) continue;
    const cudaError_t e = cudaEventSynchronize(h.out);
    if (e != cudaSuccess) return set_error(std::string("host wait: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  }
  return BSMM_OK;
}

bsmm_status bsmm_execute_host(bsmm_plan_t p, double alpha, const void* A, int64_t a_elems, const int64_t* a_off,
                              const void* B, int64_t b_elems, const int64_t* b_off, double beta, void* C,
                              int64_t c_elems, const int64_t* c_off, void* stream) {
  bsmm_status s = bsmm_execute_host_async(p, alpha, A, a_elems, a_off, B, b_elems, b_off, beta, C, c_elems, c_off,
                                          stream);
  if (s != BSMM_OK) return s;
  return bsmm_host_wait(p);
}

bsmm_status bsmm_status_device(bsmm_plan_t p, void* stream) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, p->d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err.p, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(std::string("status: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  if (w & kErrTimeout) return set_error("a kernel wait timed out"), BSMM_ERR_TIMEOUT;
  if (w & kErrBadOffset) return set_error("a kernel found a missing or invalid tile offset"), BSMM_ERR_DEVICE;
  if (w & kErrNonFinite) return set_error("non-finite input element in a split mode"), BSMM_ERR_DEVICE;
  return BSMM_OK;
}

bsmm_status bsmm_measure_rates(double* rates, void* stream) {
  if (!rates) return set_error("rates is NULL"), BSMM_ERR_INVALID;
  const cudaError_t e = unit_rates(rates, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(std::string("rates: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  return BSMM_OK;
}

bsmm_status bsmm_selftest_wait(int64_t limit_ns, void* stream) {
  if (limit_ns < 1000000 || limit_ns > 1000000000) return set_error("limit_ns must be in 1e6..1e9"), BSMM_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* d = nullptr;
  int32_t w = 0;
  cudaError_t e = cudaMalloc(&d, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = launch_wait_selftest(d, limit_ns, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&w, d, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return set_error(std::string("self-test: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  if (w & kErrTimeout) return set_error("the self-test's waits ran out (as designed)"), BSMM_ERR_TIMEOUT;
  return BSMM_OK;
}

bsmm_status bsmm_plan_kernel_ms(bsmm_plan_t p, float* ms, int32_t max_n, int32_t* count) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  if (!p->opt.profile || p->ev_last < 0)
    return set_error("plan has no profile events (profile option, one execute)"), BSMM_ERR_INVALID;
  if (max_n < 0 || (max_n > 0 && !ms)) return set_error("ms is NULL"), BSMM_ERR_INVALID;
  // the executes since the previous call (or, when there was none, the last one again)
  const int sets = std::max(1, p->ev_pending);
  const int nk = p->ev_counts[p->ev_last];
  const int n = std::min<int>(nk, max_n);
  const int last = p->ev_last;
  if (cudaEventSynchronize(p->ev[last][p->ev_counts[last]]) != cudaSuccess)
    return set_error("event sync failed"), BSMM_ERR_CUDA;
  std::vector<double> sum(n, 0.0);
  for (int b = 0; b < sets; b++) {
    const int set = (last - b + kProfileRing) % kProfileRing;
    if (p->ev_counts[set] != nk) return set_error("executes with different kernel counts"), BSMM_ERR_INVALID;
    for (int i = 0; i < n; i++) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, p->ev[set][i], p->ev[set][i + 1]) != cudaSuccess)
        return set_error("cudaEventElapsedTime failed"), BSMM_ERR_CUDA;
      sum[i] += t;
    }
  }
  for (int i = 0; i < n; i++) ms[i] = (float)(sum[i] / sets);
  p->ev_pending = 0;
  if (count) *count = nk;
  return BSMM_OK;
}

bsmm_status bsmm_plan_timings(bsmm_plan_t p, int64_t* start_ns, int64_t* end_ns, int32_t* cta) {
  if (!p) return set_error("plan is NULL"), BSMM_ERR_INVALID;
  if (!p->opt.record_timings) return set_error("plan was built without record_timings"), BSMM_ERR_INVALID;
  if (cudaDeviceSynchronize() != cudaSuccess) return set_error("device sync failed"), BSMM_ERR_CUDA;
  std::vector<int64_t> t(2 * p->n_units);
  if (p->n_units) {
    if (cudaMemcpy(t.data(), p->d_timings.p, sizeof(int64_t) * t.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return set_error("timing copy failed"), BSMM_ERR_CUDA;
    if (cta && cudaMemcpy(cta, p->d_unit_cta.p, sizeof(int32_t) * p->n_units, cudaMemcpyDeviceToHost) != cudaSuccess)
      return set_error("timing copy failed"), BSMM_ERR_CUDA;
  }
  // the device records each unit's start and the longest time a CTA spent on it
  for (int64_t u = 0; u < p->n_units; u++) {
    if (start_ns) start_ns[u] = t[2 * u];
    if (end_ns) end_ns[u] = t[2 * u] + t[2 * u + 1];
  }
  return BSMM_OK;
}

}  // extern "C"
