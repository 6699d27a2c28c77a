"""Python binding of the bsmm C ABI (``include/bsmm.h``).

Argument marshalling only: every step of the product (planning, slicing,
contraction, epilogue) runs in the native library ``_build/libbsmm.so``; this
module converts numpy arrays and torch tensors to pointers and status codes to
exceptions. There is no Python or CPU fallback: if the library cannot be built
or loaded, every call raises.

Function names follow the C entry points.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

__all__ = [
    "BsmmError", "lib", "library_path", "BSMM_FP64", "BSMM_SPLIT_BF16", "BSMM_SPLIT_FP16",
    "BSMM_SCHED_FLOPS", "BSMM_SCHED_COSTS", "BSMM_SCHED_NATURAL", "BSMM_NFEATURES", "BSMM_FEATURE_VERSION", "Plan",
    "bsmm_options_default", "bsmm_plan", "bsmm_plan_query", "bsmm_plan_ksplit", "bsmm_plan_features",
    "bsmm_plan_set_costs", "bsmm_plan_set_ctas", "bsmm_execute", "bsmm_execute_f32", "bsmm_execute_host",
    "bsmm_execute_host_async", "bsmm_host_wait", "bsmm_status_device", "BSMM_F64", "BSMM_F32", "BSMM_C128",
    "bsmm_plan_timings", "bsmm_plan_kernel_ms", "bsmm_split_tile_noalloc", "bsmm_selftest_wait", "bsmm_last_error",
    "bsmm_measure_rates", "bsmm_plan_form",
    "bsmm_destroy", "EXPORTED",
]

BSMM_FP64, BSMM_SPLIT_BF16, BSMM_SPLIT_FP16 = 0, 1, 2
BSMM_SCHED_FLOPS, BSMM_SCHED_COSTS, BSMM_SCHED_NATURAL = 0, 1, 2
BSMM_F64, BSMM_F32, BSMM_C128 = 0, 1, 2
BSMM_NFEATURES = 12
BSMM_FEATURE_VERSION = 2  # include/bsmm.h: the meaning of the bsmm_plan_features columns
STATUS = {0: "BSMM_OK", 1: "BSMM_ERR_INVALID", 2: "BSMM_ERR_CUDA", 3: "BSMM_ERR_NOMEM",
          4: "BSMM_ERR_TIMEOUT", 5: "BSMM_ERR_UNSUPPORTED", 6: "BSMM_ERR_DEVICE"}

# every symbol include/bsmm.h declares
EXPORTED = [
    "bsmm_options_default", "bsmm_plan", "bsmm_plan_query", "bsmm_plan_ksplit", "bsmm_plan_features", "bsmm_plan_set_costs",
    "bsmm_plan_set_ctas", "bsmm_execute", "bsmm_execute_f32", "bsmm_execute_host", "bsmm_execute_host_async",
    "bsmm_host_wait", "bsmm_status_device", "bsmm_plan_timings",
    "bsmm_plan_kernel_ms", "bsmm_split_tile_noalloc", "bsmm_batch_create", "bsmm_batch_set_args",
    "bsmm_batch_execute", "bsmm_batch_query", "bsmm_batch_kernels", "bsmm_batch_set_costs", "bsmm_batch_status_device",
    "bsmm_batch_destroy", "bsmm_tune_space", "bsmm_batch_autotune", "bsmm_mlp_create", "bsmm_mlp_num_params", "bsmm_mlp_set_params", "bsmm_mlp_get_params",
    "bsmm_mlp_set_norm", "bsmm_mlp_get_norm", "bsmm_mlp_loss_grad", "bsmm_mlp_fit", "bsmm_mlp_predict",
    "bsmm_plan_predict_costs", "bsmm_mlp_destroy", "bsmm_selftest_wait", "bsmm_schedule_lpt",
    "bsmm_schedule_pieces", "bsmm_measure_rates", "bsmm_mlp_save", "bsmm_mlp_load", "bsmm_plan_cost_source",
    "bsmm_execute_batch", "bsmm_batch_autotune_cached", "bsmm_plan_form", "bsmm_last_error", "bsmm_destroy",
]


class BsmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("nslices", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("max_ctas", ctypes.c_int32), ("debug_checks", ctypes.c_int32),
                ("record_timings", ctypes.c_int32), ("profile", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("fp64_tile", ctypes.c_int32), ("stages", ctypes.c_int32), ("transa", ctypes.c_int32),
                ("transb", ctypes.c_int32), ("split_scale", ctypes.c_int32), ("ksplit", ctypes.c_int32),
                ("elem", ctypes.c_int32), ("store_warps", ctypes.c_int32), ("model_path", ctypes.c_char_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load (building from source first if needed) the native library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.bsmm_options_default.argtypes = [ctypes.POINTER(Options)]
        L.bsmm_options_default.restype = None
        L.bsmm_plan.argtypes = [ctypes.POINTER(P), i32, P, i32, P, i32, P, P, P, P, ctypes.POINTER(Options)]
        L.bsmm_plan_query.argtypes = [P, P, P, P, P, P]
        L.bsmm_plan_features.argtypes = [P, P, P]
        L.bsmm_plan_ksplit.argtypes = [P, P, P, P]
        L.bsmm_plan_set_costs.argtypes = [P, P]
        L.bsmm_plan_set_ctas.argtypes = [P, i32]
        L.bsmm_execute.argtypes = [P, f64, P, P, P, P, f64, P, P, P]
        L.bsmm_execute_f32.argtypes = [P, ctypes.c_float, P, P, P, P, ctypes.c_float, P, P, P]
        L.bsmm_execute_host.argtypes = [P, f64, P, i64, P, P, i64, P, f64, P, i64, P, P]
        L.bsmm_execute_host_async.argtypes = [P, f64, P, i64, P, P, i64, P, f64, P, i64, P, P]
        L.bsmm_host_wait.argtypes = [P]
        L.bsmm_status_device.argtypes = [P, P]
        L.bsmm_plan_timings.argtypes = [P, P, P, P]
        L.bsmm_plan_kernel_ms.argtypes = [P, P, i32, P]
        L.bsmm_split_tile_noalloc.argtypes = [i32, i32, i32, i32, f64, P, P, f64, P, P]
        L.bsmm_measure_rates.argtypes = [P, P]
        L.bsmm_batch_create.argtypes = [ctypes.POINTER(P), i32, P]
        L.bsmm_batch_set_args.argtypes = [P, P, P, P, P, P, P, P, P]
        L.bsmm_batch_execute.argtypes = [P, P]
        L.bsmm_batch_query.argtypes = [P, P, P, P]
        L.bsmm_batch_kernels.argtypes = [P, P]
        L.bsmm_selftest_wait.argtypes = [i64, P]
        L.bsmm_schedule_lpt.argtypes = [i64, P, i32, P, P, P]
        L.bsmm_schedule_pieces.argtypes = [i64, P, P, i32, f64, i32, P]
        L.bsmm_batch_set_costs.argtypes = [P, P]
        L.bsmm_batch_status_device.argtypes = [P, P]
        L.bsmm_batch_destroy.argtypes = [P]
        L.bsmm_batch_destroy.restype = None
        L.bsmm_tune_space.argtypes = [i32, i32, P, i32, P]
        L.bsmm_batch_autotune.argtypes = [P, i32, P, i32, P, P, P]
        L.bsmm_mlp_create.argtypes = [ctypes.POINTER(P), ctypes.c_uint64]
        L.bsmm_mlp_num_params.argtypes = []
        L.bsmm_mlp_set_params.argtypes = [P, P, i64]
        L.bsmm_mlp_get_params.argtypes = [P, P, i64]
        L.bsmm_mlp_set_norm.argtypes = [P, P, P, ctypes.c_float, ctypes.c_float]
        L.bsmm_mlp_get_norm.argtypes = [P, P, P, P, P]
        L.bsmm_mlp_loss_grad.argtypes = [P, P, P, i64, P, P, P]
        L.bsmm_mlp_fit.argtypes = [P, P, P, i64, i32, ctypes.c_float, P, P]
        L.bsmm_mlp_predict.argtypes = [P, P, i64, P, P]
        L.bsmm_plan_predict_costs.argtypes = [P, P, P]
        L.bsmm_mlp_save.argtypes = [P, ctypes.c_char_p]
        L.bsmm_execute_batch.argtypes = [i32, P, P, P, P, P, P, P, P, P, P]
        L.bsmm_batch_autotune_cached.argtypes = [P, ctypes.c_char_p, i32, P, P, P]
        L.bsmm_mlp_load.argtypes = [ctypes.POINTER(P), ctypes.c_char_p]
        L.bsmm_plan_cost_source.argtypes = [P, P]
        L.bsmm_plan_form.argtypes = [P, P, P, P, P, P]
        L.bsmm_mlp_destroy.argtypes = [P]
        L.bsmm_mlp_destroy.restype = None
        L.bsmm_last_error.argtypes = []
        L.bsmm_last_error.restype = ctypes.c_char_p
        L.bsmm_destroy.argtypes = [P]
        L.bsmm_destroy.restype = None
        for name in EXPORTED:
            if name not in ("bsmm_options_default", "bsmm_last_error", "bsmm_destroy", "bsmm_batch_destroy",
                            "bsmm_mlp_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def bsmm_last_error() -> str:
    return lib().bsmm_last_error().decode()


def _check(status: int):
    if status != 0:
        raise BsmmError(status, bsmm_last_error())


def _np(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or a torch tensor (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data if a.size else None
    if hasattr(a, "data_ptr"):
        return a.data_ptr() if a.numel() else None
    if isinstance(a, int):
        return a
    raise TypeError(f"cannot take the address of {type(a)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def bsmm_options_default() -> Options:
    o = Options()
    lib().bsmm_options_default(ctypes.byref(o))
    return o


class Plan:
    """Owns one bsmm_plan_t; destroyed with the object or by bsmm_destroy."""

    def __init__(self, handle: int, M: int, N: int, K: int, mode: int, nslices: int = 6):
        self.handle = handle
        self.M, self.N, self.K, self.mode, self.nslices = M, N, K, mode, nslices

    def __del__(self):
        try:
            bsmm_destroy(self)
        except Exception:
            pass


def bsmm_plan(row_sizes, col_sizes, inner_sizes, a_mask, b_mask, c_mask=None, *, mode: int = BSMM_FP64,
              nslices: int = 6, schedule: int = BSMM_SCHED_FLOPS, max_ctas: int = 0, debug_checks: int = 0,
              record_timings: int = 0, profile: int = 0, cluster: int = 0, fp64_tile: int = 0,
              stages: int = 0, transa: int = 0, transb: int = 0, split_scale: int = 0,
              ksplit: int = 0, elem: int = BSMM_F64, model_path=None, store_warps: int = 0) -> Plan:
    r = _np(row_sizes, np.int32)
    c = _np(col_sizes, np.int32)
    q = _np(inner_sizes, np.int32)
    am = _np(a_mask, np.uint8)
    bm = _np(b_mask, np.uint8)
    cm = None if c_mask is None else _np(c_mask, np.uint8)
    o = bsmm_options_default()
    o.mode, o.nslices, o.schedule, o.max_ctas = mode, nslices, schedule, max_ctas
    o.debug_checks, o.record_timings, o.profile, o.cluster = debug_checks, record_timings, profile, cluster
    o.fp64_tile = fp64_tile
    o.stages = stages
    o.transa = transa
    o.transb = transb
    o.split_scale = split_scale
    o.ksplit = ksplit
    o.elem = elem
    o.store_warps = store_warps
    path = None if model_path is None else os.fsencode(model_path)
    o.model_path = path  # read by bsmm_plan only; `path` keeps the bytes alive until it returns
    h = ctypes.c_void_p()
    _check(lib().bsmm_plan(ctypes.byref(h), len(r), _ptr(r), len(c), _ptr(c), len(q), _ptr(q), _ptr(am),
                           _ptr(bm), _ptr(cm), ctypes.byref(o)))
    return Plan(h.value, len(r), len(c), len(q), mode, nslices)


def bsmm_plan_query(plan: Plan) -> dict:
    nct, ntr, nun = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    fl = ctypes.c_double()
    cs = np.zeros((plan.M, plan.N), np.uint8)
    _check(lib().bsmm_plan_query(plan.handle, ctypes.addressof(nct), ctypes.addressof(ntr), ctypes.addressof(fl),
                                 _ptr(cs), ctypes.addressof(nun)))
    return {"n_ctiles": nct.value, "n_triples": ntr.value, "useful_flops": fl.value, "c_mask": cs,
            "n_units": nun.value}


def bsmm_plan_ksplit(plan: Plan) -> dict:
    """Split k of a plan: regions cut into pieces, their total piece count, and per work
    unit the number of pieces of its region."""
    nr, npc = ctypes.c_int64(), ctypes.c_int64()
    n = bsmm_plan_query(plan)["n_units"]
    pieces = np.zeros(max(n, 1), np.int32)
    _check(lib().bsmm_plan_ksplit(plan.handle, ctypes.addressof(nr), ctypes.addressof(npc), _ptr(pieces)))
    return {"n_regions": nr.value, "n_pieces": npc.value, "pieces": pieces[:n]}


def bsmm_plan_features(plan: Plan):
    n = bsmm_plan_query(plan)["n_units"]
    f = np.zeros((n, BSMM_NFEATURES), np.float32)
    c = np.zeros(n, np.float64)
    _check(lib().bsmm_plan_features(plan.handle, _ptr(f), _ptr(c)))
    return f, c


def bsmm_plan_set_costs(plan: Plan, costs):
    c = _np(costs, np.float64)
    _check(lib().bsmm_plan_set_costs(plan.handle, _ptr(c)))


def bsmm_plan_set_ctas(plan: Plan, ctas: int):
    _check(lib().bsmm_plan_set_ctas(plan.handle, int(ctas)))


def bsmm_execute(plan: Plan, alpha, A, a_off, B, b_off, beta, C, c_off, stream=None):
    """Device tensors (torch, CUDA): A, B, C float64 arenas (complex128 for a plan with
    complex elements; alpha and beta real); a_off, b_off, c_off int64 tables."""
    _check(lib().bsmm_execute(plan.handle, float(alpha), _ptr(A), _ptr(a_off), _ptr(B), _ptr(b_off), float(beta),
                              _ptr(C), _ptr(c_off), _stream(stream)))


def bsmm_execute_f32(plan: Plan, alpha, A, a_off, B, b_off, beta, C, c_off, stream=None):
    """Device tensors for a plan with float32 elements: A, B, C float32 arenas (offsets in
    float elements, multiples of 4); a_off, b_off, c_off int64 tables."""
    _check(lib().bsmm_execute_f32(plan.handle, float(alpha), _ptr(A), _ptr(a_off), _ptr(B), _ptr(b_off),
                                  float(beta), _ptr(C), _ptr(c_off), _stream(stream)))


def bsmm_execute_host(plan: Plan, alpha, A, a_off, B, b_off, beta, C, c_off, stream=None):
    """Host arrays (numpy or CPU tensors, pinned for asynchronous copies); C is updated in place."""
    def n(x):
        return int(x.size if isinstance(x, np.ndarray) else x.numel())
    _check(lib().bsmm_execute_host(plan.handle, float(alpha), _ptr(A), n(A), _ptr(a_off), _ptr(B), n(B),
                                   _ptr(b_off), float(beta), _ptr(C), n(C), _ptr(c_off), _stream(stream)))


# host arrays of the products in flight per plan handle, kept alive until bsmm_host_wait
_in_flight = {}


def bsmm_execute_host_async(plan: Plan, alpha, A, a_off, B, b_off, beta, C, c_off, stream=None):
    """Enqueues one host-buffer product and returns; C holds its result after bsmm_host_wait.
    The arrays are kept referenced until then (and must not be changed meanwhile)."""
    def n(x):
        return int(x.size if isinstance(x, np.ndarray) else x.numel())
    _check(lib().bsmm_execute_host_async(plan.handle, float(alpha), _ptr(A), n(A), _ptr(a_off), _ptr(B), n(B),
                                         _ptr(b_off), float(beta), _ptr(C), n(C), _ptr(c_off), _stream(stream)))
    _in_flight.setdefault(plan.handle, []).append((A, a_off, B, b_off, C, c_off))


def bsmm_host_wait(plan: Plan):
    """Waits until every host product enqueued on the plan has its C on the host."""
    try:
        _check(lib().bsmm_host_wait(plan.handle))
    finally:
        _in_flight.pop(plan.handle, None)


def bsmm_status_device(plan: Plan, stream=None):
    _check(lib().bsmm_status_device(plan.handle, _stream(stream)))


def bsmm_plan_timings(plan: Plan):
    n = bsmm_plan_query(plan)["n_units"]
    s = np.zeros(n, np.int64)
    e = np.zeros(n, np.int64)
    cta = np.zeros(n, np.int32)
    _check(lib().bsmm_plan_timings(plan.handle, _ptr(s), _ptr(e), _ptr(cta)))
    return s, e, cta


def bsmm_plan_kernel_ms(plan: Plan):
    """Per-kernel device milliseconds of the last execute (plan built with profile=1)."""
    ms = (ctypes.c_float * 8)()
    n = ctypes.c_int32()
    _check(lib().bsmm_plan_kernel_ms(plan.handle, ms, 8, ctypes.byref(n)))
    return [float(ms[i]) for i in range(n.value)]


def bsmm_measure_rates(stream=None):
    """Measured rates of the current GPU: {"dfma": TFLOP/s of FP64 fused multiply-adds,
    "dmma": TFLOP/s of the FP64 tensor-core mma.sync, "imma": TOP/s of the INT8 one}."""
    r = (ctypes.c_double * 3)()
    _check(lib().bsmm_measure_rates(r, _stream(stream)))
    return {"dfma": r[0], "dmma": r[1], "imma": r[2]}


def bsmm_split_tile_noalloc(m, n, k, nslices, alpha, A, B, beta, C, stream=None):
    """One dense split-precision tile task with no device allocation (device tensors:
    A m x k, B k x n, C m x n, row-major float64). For callers that cannot allocate
    device memory at the point of the call (an allocator that is locked or forbids
    allocation on their hot path, or device memory reserved up front); see
    include/bsmm.h for the limits and the shared-scratch rules (calls overlapping on
    the GPU race). Returns once the product is complete; raises BsmmError with the
    library's status otherwise."""
    m, n, k = int(m), int(n), int(k)
    for name, t, need in (("A", A, m * k), ("B", B, k * n), ("C", C, m * n)):
        if need == 0 and t is None:
            continue
        if t is None or str(getattr(t, "dtype", "")) != "torch.float64" or not getattr(t, "is_cuda", False) \
                or not t.is_contiguous():
            raise BsmmError(1, f"bsmm_split_tile_noalloc: {name} must be a contiguous float64 "
                                              f"CUDA tensor")
        if t.numel() < need:
            raise BsmmError(1, f"bsmm_split_tile_noalloc: {name} holds {t.numel()} elements, "
                                              f"needs {need}")
    _check(lib().bsmm_split_tile_noalloc(m, n, k, int(nslices), float(alpha), _ptr(A), _ptr(B),
                                         float(beta), _ptr(C), _stream(stream)))


class Batch:
    """Owns one bsmm_batch_t (and keeps its plans alive)."""

    def __init__(self, handle: int, plans):
        self.handle = handle
        self.plans = list(plans)

    def __del__(self):
        try:
            bsmm_batch_destroy(self)
        except Exception:
            pass


def bsmm_execute_batch(plans, alphas, As, a_offs, Bs, b_offs, betas, Cs, c_offs, stream=None):
    """The whole batch in one library call (device tensors per product; see
    include/bsmm.h: the library caches the batch object of the plan list)."""
    n = len(plans)
    keep = list(plans)  # the plans stay referenced for the duration of the call
    ptrs = lambda xs: (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    _check(lib().bsmm_execute_batch(n, (ctypes.c_void_p * n)(*[p.handle for p in keep]),
                                    (ctypes.c_double * n)(*[float(a) for a in alphas]), ptrs(As), ptrs(a_offs),
                                    ptrs(Bs), ptrs(b_offs), (ctypes.c_double * n)(*[float(b) for b in betas]),
                                    ptrs(Cs), ptrs(c_offs), _stream(stream)))


def bsmm_batch_create(plans) -> Batch:
    arr = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    h = ctypes.c_void_p()
    _check(lib().bsmm_batch_create(ctypes.byref(h), len(plans), arr))
    return Batch(h.value, plans)


def bsmm_batch_set_args(batch: Batch, alpha, A, a_off, B, b_off, beta, C, c_off):
    """Per-product lists: alpha, beta floats; A, a_off, B, b_off, C, c_off device tensors."""
    n = len(batch.plans)
    def ptrs(xs):
        return (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    al = (ctypes.c_double * n)(*[float(x) for x in alpha])
    be = (ctypes.c_double * n)(*[float(x) for x in beta])
    batch._keep = (A, a_off, B, b_off, C, c_off)
    _check(lib().bsmm_batch_set_args(batch.handle, al, ptrs(A), ptrs(a_off), ptrs(B), ptrs(b_off), be, ptrs(C),
                                     ptrs(c_off)))


def bsmm_batch_execute(batch: Batch, stream=None):
    _check(lib().bsmm_batch_execute(batch.handle, _stream(stream)))


def bsmm_batch_query(batch: Batch) -> dict:
    nu, fl, bins = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().bsmm_batch_query(batch.handle, ctypes.byref(nu), ctypes.byref(fl), ctypes.byref(bins)))
    return {"n_units": nu.value, "useful_flops": fl.value, "bins": bins.value}


def bsmm_schedule_lpt(cost, bins: int):
    """The planner's longest-processing-time packing on the host: (ptr, units, makespan)."""
    c = _np(cost, np.float64)
    ptr = np.zeros(bins + 1, np.int32)
    units = np.zeros(max(len(c), 1), np.int32)
    mk = ctypes.c_double()
    _check(lib().bsmm_schedule_lpt(len(c), _ptr(c), int(bins), _ptr(ptr), _ptr(units), ctypes.byref(mk)))
    return ptr, units[:len(c)], mk.value


def bsmm_schedule_pieces(cost, length, bins: int, overhead: float, ksplit: int = 0):
    """The planner's split-k choice on the host: pieces per unit."""
    c = _np(cost, np.float64)
    ln = _np(length, np.int64)
    out = np.zeros(max(len(c), 1), np.int32)
    _check(lib().bsmm_schedule_pieces(len(c), _ptr(c), _ptr(ln), int(bins), float(overhead), int(ksplit), _ptr(out)))
    return out[:len(c)]


def bsmm_selftest_wait(limit_ns: int, stream=None):
    """Runs the bounded-wait self-test kernel; raises BsmmError with status BSMM_ERR_TIMEOUT
    (4) when its waits ran out as designed."""
    _check(lib().bsmm_selftest_wait(int(limit_ns), _stream(stream)))


def bsmm_batch_kernels(batch: Batch) -> int:
    """Kernels the batch's most recent bsmm_batch_execute launched."""
    n = ctypes.c_int32()
    _check(lib().bsmm_batch_kernels(batch.handle, ctypes.byref(n)))
    return n.value


def bsmm_batch_set_costs(batch: Batch, costs):
    c = _np(costs, np.float64)
    _check(lib().bsmm_batch_set_costs(batch.handle, _ptr(c)))


def bsmm_batch_status_device(batch: Batch, stream=None):
    _check(lib().bsmm_batch_status_device(batch.handle, _stream(stream)))


def bsmm_batch_destroy(batch: Batch):
    if batch is not None and batch.handle:
        lib().bsmm_batch_destroy(batch.handle)
        batch.handle = None


class TunePoint(ctypes.Structure):
    _fields_ = [("cluster", ctypes.c_int32), ("stages", ctypes.c_int32), ("fp64_tile", ctypes.c_int32),
                ("store_warps", ctypes.c_int32)]


def bsmm_tune_space(mode: int, nslices: int = 6) -> list:
    """The library's candidate list for a mode: dicts with cluster, stages, fp64_tile,
    store_warps."""
    n = ctypes.c_int32()
    _check(lib().bsmm_tune_space(mode, nslices, None, 0, ctypes.byref(n)))
    arr = (TunePoint * max(n.value, 1))()
    _check(lib().bsmm_tune_space(mode, nslices, arr, n.value, ctypes.byref(n)))
    return [{"cluster": t.cluster, "stages": t.stages, "fp64_tile": t.fp64_tile, "store_warps": t.store_warps}
            for t in arr[:n.value]]


def bsmm_batch_autotune(batch: Batch, candidates=None, reps: int = 3, stream=None):
    """Time the batch under each candidate (default: the library's space for its mode)
    and keep the fastest. Returns (chosen candidate dict, list of median ms)."""
    if candidates is None:
        p0 = batch.plans[0]
        candidates = bsmm_tune_space(p0.mode, p0.nslices)
    n = len(candidates)
    arr = (TunePoint * n)(*[TunePoint(c.get("cluster", 0), c.get("stages", 0), c.get("fp64_tile", 0),
                                      c.get("store_warps", 0)) for c in candidates])
    ms = (ctypes.c_float * n)()
    ch = ctypes.c_int32(-1)
    _check(lib().bsmm_batch_autotune(batch.handle, n, arr, reps, _stream(stream), ctypes.byref(ch), ms))
    return candidates[ch.value], list(ms)


def bsmm_batch_autotune_cached(batch: Batch, cache_path, reps: int = 2, stream=None):
    """Tune the batch with a persistent cache file (see include/bsmm.h); returns
    (candidate dict, from_cache)."""
    t = TunePoint()
    fc = ctypes.c_int32()
    _check(lib().bsmm_batch_autotune_cached(batch.handle, os.fsencode(cache_path), int(reps), _stream(stream),
                                            ctypes.byref(t), ctypes.byref(fc)))
    return {"cluster": t.cluster, "stages": t.stages, "fp64_tile": t.fp64_tile,
            "store_warps": t.store_warps}, bool(fc.value)


class Mlp:
    """Owns one bsmm_mlp_t (the learned task-cost model)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        try:
            bsmm_mlp_destroy(self)
        except Exception:
            pass


def bsmm_mlp_create(seed: int = 0) -> Mlp:
    h = ctypes.c_void_p()
    _check(lib().bsmm_mlp_create(ctypes.byref(h), ctypes.c_uint64(seed)))
    return Mlp(h.value)


def bsmm_mlp_num_params() -> int:
    return int(lib().bsmm_mlp_num_params())


def bsmm_mlp_set_params(mlp: Mlp, params):
    p = _np(params, np.float32)
    _check(lib().bsmm_mlp_set_params(mlp.handle, _ptr(p), p.size))


def bsmm_mlp_get_params(mlp: Mlp) -> np.ndarray:
    p = np.zeros(bsmm_mlp_num_params(), np.float32)
    _check(lib().bsmm_mlp_get_params(mlp.handle, _ptr(p), p.size))
    return p


def bsmm_mlp_set_norm(mlp: Mlp, x_mean, x_sd, y_mean: float, y_sd: float):
    m = _np(x_mean, np.float32)
    s = _np(x_sd, np.float32)
    _check(lib().bsmm_mlp_set_norm(mlp.handle, _ptr(m), _ptr(s), float(y_mean), float(y_sd)))


def bsmm_mlp_get_norm(mlp: Mlp):
    m = np.zeros(BSMM_NFEATURES, np.float32)
    s = np.zeros(BSMM_NFEATURES, np.float32)
    ym, ys = ctypes.c_float(), ctypes.c_float()
    _check(lib().bsmm_mlp_get_norm(mlp.handle, _ptr(m), _ptr(s), ctypes.byref(ym), ctypes.byref(ys)))
    return m, s, ym.value, ys.value


def bsmm_mlp_loss_grad(mlp: Mlp, X, t, stream=None):
    """X (n x F) and t (n) float32 device tensors; returns (loss, grad numpy)."""
    g = np.zeros(bsmm_mlp_num_params(), np.float32)
    loss = ctypes.c_float()
    _check(lib().bsmm_mlp_loss_grad(mlp.handle, _ptr(X), _ptr(t), int(t.numel()), ctypes.byref(loss), _ptr(g),
                                    _stream(stream)))
    return loss.value, g


def bsmm_mlp_fit(mlp: Mlp, X, t, steps: int, lr: float, stream=None) -> float:
    loss = ctypes.c_float()
    _check(lib().bsmm_mlp_fit(mlp.handle, _ptr(X), _ptr(t), int(t.numel()), int(steps), float(lr), ctypes.byref(loss),
                              _stream(stream)))
    return loss.value


def bsmm_mlp_predict(mlp: Mlp, X, y, stream=None):
    _check(lib().bsmm_mlp_predict(mlp.handle, _ptr(X), int(y.numel()), _ptr(y), _stream(stream)))


def bsmm_mlp_save(mlp: Mlp, path) -> None:
    """Write the model to a versioned, checksummed cost-model file (see include/bsmm.h)."""
    _check(lib().bsmm_mlp_save(mlp.handle, os.fsencode(path)))


def bsmm_mlp_load(path) -> Mlp:
    """A model read from a cost-model file written by bsmm_mlp_save."""
    h = ctypes.c_void_p()
    _check(lib().bsmm_mlp_load(ctypes.byref(h), os.fsencode(path)))
    return Mlp(h.value)


BSMM_COSTS_FLOPS, BSMM_COSTS_MODEL, BSMM_COSTS_GIVEN = 0, 1, 2


def bsmm_plan_form(plan: Plan) -> dict:
    """The planner's launch choices: cluster, store_warps, epi_walk, stages, ctas."""
    v = [ctypes.c_int32() for _ in range(5)]
    _check(lib().bsmm_plan_form(plan.handle, *[ctypes.byref(x) for x in v]))
    return dict(zip(("cluster", "store_warps", "epi_walk", "stages", "ctas"), (x.value for x in v)))


def bsmm_plan_cost_source(plan: Plan) -> int:
    """Where the plan's unit costs came from: BSMM_COSTS_FLOPS, _MODEL or _GIVEN."""
    v = ctypes.c_int32()
    _check(lib().bsmm_plan_cost_source(plan.handle, ctypes.byref(v)))
    return v.value


def bsmm_plan_predict_costs(plan: Plan, mlp: Mlp, stream=None):
    _check(lib().bsmm_plan_predict_costs(plan.handle, mlp.handle, _stream(stream)))


def bsmm_mlp_destroy(mlp: Mlp):
    if mlp is not None and mlp.handle:
        lib().bsmm_mlp_destroy(mlp.handle)
        mlp.handle = None


def bsmm_destroy(plan: Plan):
    if plan is not None and plan.handle:
        lib().bsmm_destroy(plan.handle)  # waits for the plan's host products first
        _in_flight.pop(plan.handle, None)
        plan.handle = None
