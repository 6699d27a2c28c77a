"""GPU parity of float32 elements in the split modes (bsmm_options.elem = BSMM_F32),
through the C ABI: the split oracle with float32 arenas fixes every bit (exact sum rounded
once to float32, float32 epilogue), so the comparison is bit for bit; the error against
the FP64 oracle on the same (float32) inputs is asserted at float32 accuracy."""
import dataclasses

import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import c_arena, rel_fro, struct_elements

pytestmark = pytest.mark.gpu


def run_f32(prob, s=6, mode=P.BSMM_SPLIT_BF16, c_mask=None, scaling="tile", fill_seed=0, **opt):
    import torch
    from gpu_helpers import to_dev
    cs, _, _ = oracle.structure(prob, c_mask)
    off, C64 = c_arena(prob, cs, rng=np.random.default_rng(fill_seed))
    C0 = C64.astype(np.float32)
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, s, scaling=scaling)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask, c_mask,
                       mode=mode, nslices=s, elem=P.BSMM_F32, split_scale=int(scaling == "rows"),
                       transa=int(prob.transa), transb=int(prob.transb), debug_checks=1, **opt)
    dev = lambda x: to_dev(x if x.size else np.zeros(4, x.dtype))
    C = dev(C0)
    P.bsmm_execute_f32(plan, prob.alpha, dev(prob.A), dev(prob.a_off.astype(np.int64)), dev(prob.B),
                       dev(prob.b_off.astype(np.int64)), prob.beta, C, dev(off.astype(np.int64)))
    torch.cuda.synchronize()
    P.bsmm_status_device(plan)
    got = C.cpu().numpy()[:C0.size]
    g, w = struct_elements(prob, cs, off, got), struct_elements(prob, cs, off, want)
    if not np.array_equal(g, w):
        bad = np.flatnonzero(g != w)
        raise AssertionError(f"{bad.size} of {g.size} differ; first {bad[:4]}: {g[bad[:4]]} vs {w[bad[:4]]}")
    # against FP64 products of the same float32 inputs
    p64 = dataclasses.replace(prob, A=prob.A.astype(np.float64), B=prob.B.astype(np.float64))
    ref = C0.astype(np.float64)
    oracle.bsmm(p64, cs, ref, off)
    return plan, rel_fro(g.astype(np.float64), struct_elements(prob, cs, off, ref))


@pytest.mark.parametrize("s,mode", [(6, P.BSMM_SPLIT_BF16), (4, P.BSMM_SPLIT_FP16), (3, P.BSMM_SPLIT_BF16)])
@pytest.mark.parametrize("seed", range(5))
def test_small_ragged(seed, s, mode):
    prob = G.as_float32(G.random_small(seed, max_blocks=6, max_size=70))
    _, err = run_f32(prob, s, mode)
    assert err <= {6: 1e-6, 4: 1e-6, 3: 1e-5}[s]


def test_nonuniform_dense_clusters_and_accuracy():
    prob = G.as_float32(G.make_problem("nonuniform_dense", 3, 900, lo=64, hi=256))
    for cl in (1, 2, 4):
        _, err = run_f32(prob, 6, cluster=cl)
        assert err <= 1.2e-7, err  # float32 rounding of the result (unit roundoff 6e-8)
    _, err4 = run_f32(prob, 4)
    assert err4 <= 2e-7, err4


def test_alpha_beta_c_mask_row_scaling_transposed_and_split_k():
    prob = G.make_problem("banded_decay_wide", 5, 1200, lo=32, hi=200, band=3)
    prob.alpha, prob.beta = -0.75, 1.5
    cm = (np.random.default_rng(2).random((prob.M, prob.N)) < 0.2).astype(np.uint8)
    p32 = G.as_float32(prob)
    run_f32(p32, 6, P.BSMM_SPLIT_FP16, c_mask=cm)
    run_f32(p32, 6, P.BSMM_SPLIT_BF16, c_mask=cm, scaling="rows")
    run_f32(p32, 6, c_mask=cm, ksplit=3)
    run_f32(G.as_float32(G.transposed_storage(prob, True, True)), 6, c_mask=cm)


def test_thin_automatic_split_k():
    prob = G.as_float32(G.make_problem("thin_dense", 4, 260, k_factor=60))
    plan, _ = run_f32(prob, 6)
    assert P.bsmm_plan_ksplit(plan)["n_regions"] > 0


def _column(vals, b=None):
    one = np.ones(1, np.int32)
    q = np.ones(len(vals), np.int32)
    am, bm = np.ones((1, len(vals)), np.uint8), np.ones((len(vals), 1), np.uint8)
    a_off, at = G.layout_arena(am, one, q)
    b_off, bt = G.layout_arena(bm, q, one)
    A, B = np.zeros(at), np.zeros(bt)
    A[a_off[0, :]] = vals
    B[b_off[:, 0]] = 1.0 if b is None else b
    return G.as_float32(G.Problem("column", one, one, q, am, bm, a_off, b_off, A, B, 1.0, 0.0))


def test_rounded_once_not_through_float64():
    """1 + 2^-24 + 2^-60 rounds to 1 + 2^-23 in float32; through float64 it would be a tie
    that rounds to 1."""
    import torch
    prob = _column([1.0, 2.0 ** -24, 2.0 ** -60])
    run_f32(prob, 6)
    from gpu_helpers import to_dev
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, elem=P.BSMM_F32)
    C = to_dev(np.zeros(4, np.float32))
    P.bsmm_execute_f32(plan, 1.0, to_dev(prob.A), to_dev(prob.a_off), to_dev(prob.B), to_dev(prob.b_off), 0.0, C,
                       to_dev(np.zeros((1, 1), np.int64)))
    torch.cuda.synchronize()
    assert C.cpu().numpy()[0] == np.float32(1.0 + 2.0 ** -23)


def test_subnormal_float32_results():
    prob = G.as_float32(G.random_small(7, max_blocks=4, max_size=20, values="integers"))
    prob.A *= np.float32(2.0 ** -70)
    prob.B *= np.float32(2.0 ** -70)
    prob.alpha, prob.beta = 1.0, 0.0
    run_f32(prob, 6)


def test_errors_are_reported():
    import torch
    from gpu_helpers import to_dev
    prob = G.as_float32(G.random_small(1, max_blocks=3, max_size=30, allow_zero=False))
    with pytest.raises(P.BsmmError):  # float32 elements take a split mode
        P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask, mode=P.BSMM_FP64,
                    elem=P.BSMM_F32)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, elem=P.BSMM_F32)
    cs, _, _ = oracle.structure(prob)
    off, tot = G.layout_arena(cs, prob.row_sizes, prob.col_sizes)
    C = to_dev(np.zeros(max(tot, 4), np.float32))
    args = (to_dev(prob.A), to_dev(prob.a_off), to_dev(prob.B), to_dev(prob.b_off), 0.0, C, to_dev(off))
    with pytest.raises(P.BsmmError):  # the float64 entry point refuses a float32 plan
        P.bsmm_execute(plan, 1.0, *args)
    # a non-finite element is reported by the device status
    bad = prob.A.copy()
    bad[prob.a_off[prob.a_off >= 0][0]] = np.float32(np.inf)
    P.bsmm_execute_f32(plan, 1.0, to_dev(bad), *args[1:])
    torch.cuda.synchronize()
    with pytest.raises(P.BsmmError):
        P.bsmm_status_device(plan)
    # a float32 tile not 16-byte aligned is reported, not loaded with vector loads
    a_off2 = prob.a_off.copy()
    first = np.argwhere(a_off2 >= 0)[0]
    A2 = np.concatenate([np.zeros(2, np.float32), prob.A])
    a_off2[a_off2 >= 0] += 2
    P.bsmm_execute_f32(plan, 1.0, to_dev(A2), to_dev(a_off2), *args[2:])
    torch.cuda.synchronize()
    with pytest.raises(P.BsmmError):
        P.bsmm_status_device(plan)
    del first


def test_deep_inner_blocks():
    """Float32 elements with inner blocks deeper than the exact FP32 depth (700 and 1100
    at 6 slices): the deep kernel form gives the float32 split oracle's bits."""
    rng = np.random.default_rng(41)
    r, q, c = np.array([50, 90], np.int32), np.array([700, 48, 1100], np.int32), np.array([30, 60], np.int32)
    am, bm = np.ones((2, 3), np.uint8), np.ones((3, 2), np.uint8)
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    prob = G.as_float32(G.Problem("f32_deep", r, c, q, am, bm, a_off, b_off, rng.uniform(-1, 1, at),
                                  rng.uniform(-1, 1, bt), 1.5, -0.25))
    _, err = run_f32(prob, 6)
    assert err <= 1.2e-7, err
