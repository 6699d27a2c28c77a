"""CPU oracle for block-sparse C = alpha*A*B + beta*C.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package; the library (its C ABI and Python
binding) never does, and shares no code with it.

* ``oracle.c``  - the FP64 tile loop (paper Sec. 2.1 rank-k updates, Algorithm 1's
                  alpha), the boolean mask product, k-lists and the flop count.
* ``split.py``  - the split-precision modes (Ozaki-style slicing, per-tile
                  power-of-two scales) in numpy.
* ``mlp.py``    - FP64 forward/backward of the task-cost MLP.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.oracle_structure.argtypes = [ctypes.c_int] * 3 + [P] * 9
        L.oracle_structure.restype = ctypes.c_int
        L.oracle_klists.argtypes = [ctypes.c_int] * 3 + [P] * 4
        L.oracle_klists.restype = ctypes.c_int
        L.oracle_bsmm.argtypes = [ctypes.c_int] * 3 + [P] * 6 + [f64, P, P, P, P, f64, P, P, ctypes.c_int,
                                                                   ctypes.c_int, ctypes.c_int]
        L.oracle_bsmm.restype = ctypes.c_int
        L.oracle_bsmm_tile.argtypes = [ctypes.c_int] * 5 + [P] * 5 + [f64, P, P, P, P, f64, P, P, ctypes.c_int,
                                                                        ctypes.c_int]
        L.oracle_bsmm_tile.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _std(prob):
    """Masks and offset tables in the (i,k) / (k,j) indexing, and the transposed-storage
    bits (1: A tiles stored transposed, 2: B tiles) for the in-tile addressing."""
    ta, tb = bool(getattr(prob, "transa", False)), bool(getattr(prob, "transb", False))
    am = prob.a_mask.T if ta else prob.a_mask
    ao = prob.a_off.T if ta else prob.a_off
    bm = prob.b_mask.T if tb else prob.b_mask
    bo = prob.b_off.T if tb else prob.b_off
    return _c(am, np.uint8), _c(ao, np.int64), _c(bm, np.uint8), _c(bo, np.int64), int(ta) | (int(tb) << 1)


def _common(prob):
    am, _, bm, _, _ = _std(prob)
    return (_c(prob.row_sizes, np.int32), _c(prob.col_sizes, np.int32), _c(prob.inner_sizes, np.int32), am, bm)


def structure(prob, c_mask=None):
    """(c_struct uint8 MxN, number of nonzero triples, useful flops)."""
    r, c, q, am, bm = _common(prob)
    M, N, K = len(r), len(c), len(q)
    out = np.zeros((M, N), np.uint8)
    nt = ctypes.c_int64(0)
    fl = ctypes.c_double(0.0)
    cm = None if c_mask is None else _c(c_mask, np.uint8)
    rc = lib().oracle_structure(M, N, K, _p(r), _p(c), _p(q), _p(am), _p(bm), _p(cm), _p(out),
                                ctypes.byref(nt), ctypes.byref(fl))
    assert rc == 0
    return out, int(nt.value), float(fl.value)


def klists(prob):
    """CSR (ptr over the M*N tiles in row-major order, ascending k)."""
    r, c, q, am, bm = _common(prob)
    M, N, K = len(r), len(c), len(q)
    cnt = int((am.astype(np.int64) @ bm.astype(np.int64)).sum()) if M and N and K else 0
    ptr = np.zeros(M * N + 1, np.int64)
    kl = np.zeros(max(cnt, 1), np.int32)
    rc = lib().oracle_klists(M, N, K, _p(am), _p(bm), _p(ptr), _p(kl))
    assert rc == 0
    return ptr, kl[:cnt]


def bsmm(prob, c_struct, C, c_off, nthreads: int = 0, pieces: int = 1):
    """FP64 product in place on the C arena (float64 numpy array). ``pieces`` > 1: every
    tile's k-list is cut into that many pieces (split k, see oracle.c) whose partial sums
    are added in piece order."""
    r, c, q, am, bm = _common(prob)
    M, N, K = len(r), len(c), len(q)
    A = _c(prob.A, np.float64)
    B = _c(prob.B, np.float64)
    assert C.dtype == np.float64 and C.flags.c_contiguous
    _, ao, _, bo, trans = _std(prob)
    rc = lib().oracle_bsmm(M, N, K, _p(r), _p(c), _p(q), _p(am), _p(bm), _p(_c(c_struct, np.uint8)),
                           float(prob.alpha), _p(A), _p(ao), _p(B), _p(bo), float(prob.beta), _p(C),
                           _p(_c(c_off, np.int64)), int(nthreads), trans, int(pieces))
    assert rc == 0, "oracle_bsmm failed"
    return C


def bsmm_tile(prob, i, j, cin=None, pieces: int = 1):
    """One C tile (r_i x c_j) of the FP64 product; cin = its prior content; ``pieces`` as
    for bsmm."""
    r, c, q, am, bm = _common(prob)
    M, N, K = len(r), len(c), len(q)
    out = np.zeros((int(r[i]), int(c[j])), np.float64)
    cin_a = None if cin is None else _c(cin, np.float64)
    if float(prob.beta) != 0.0:
        assert cin_a is not None
    _, ao, _, bo, trans = _std(prob)
    rc = lib().oracle_bsmm_tile(i, j, M, N, K, _p(r), _p(c), _p(q), _p(am), _p(bm), float(prob.alpha),
                                _p(_c(prob.A, np.float64)), _p(ao), _p(_c(prob.B, np.float64)), _p(bo),
                                float(prob.beta), _p(cin_a), _p(out), trans, int(pieces))
    assert rc == 0
    return out


def num_threads() -> int:
    return int(lib().oracle_num_threads())
