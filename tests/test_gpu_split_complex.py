"""GPU parity of complex elements in the split modes (bsmm_options.elem = BSMM_C128),
through the C ABI: the split oracle with complex arenas fixes every bit (each part's exact
sum rounded once), so the comparison is bit for bit; the error against numpy's complex
FP64 product is asserted at the slice count's bar."""
import dataclasses

import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import c_arena, struct_elements

pytestmark = pytest.mark.gpu
BARS = {3: 1e-5, 4: 1e-7, 6: 1e-11}


def _dense(arena, off, rows, cols):
    ro = np.concatenate([[0], np.cumsum(np.asarray(rows, np.int64))])
    co = np.concatenate([[0], np.cumsum(np.asarray(cols, np.int64))])
    out = np.zeros((ro[-1], co[-1]), np.complex128)
    for u in range(len(rows)):
        for v in range(len(cols)):
            if off[u, v] >= 0:
                n = int(rows[u]) * int(cols[v])
                out[ro[u]:ro[u + 1], co[v]:co[v + 1]] = arena[off[u, v]:off[u, v] + n].reshape(rows[u], cols[v])
    return out


def run_c(prob, s=6, mode=P.BSMM_SPLIT_BF16, c_mask=None, trans=(0, 0), **opt):
    """Plan and run a complex product on the GPU (A and/or B supplied as the transposed
    block matrix when trans says so); bit for bit against the split oracle, and the error
    against numpy's complex product of the untransposed operands."""
    import torch
    from gpu_helpers import to_dev
    base = prob
    if any(trans):
        prob = G.transposed_storage(base, bool(trans[0]), bool(trans[1]))
        opt = dict(opt, transa=trans[0], transb=trans[1])
    cs, _, _ = oracle.structure(base, c_mask)
    off, C64 = c_arena(prob, cs, rng=np.random.default_rng(0))
    C0 = (C64 + 1j * np.random.default_rng(1).uniform(-1, 1, C64.size)).astype(np.complex128)
    want = C0.copy()
    # (the oracle reads the transposed storage; row/column scaling when asked)
    OS.bsmm_split(prob, cs, want, off, s, scaling="rows" if opt.get("split_scale") else "tile")
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask, c_mask,
                       mode=mode, nslices=s, elem=P.BSMM_C128, debug_checks=1, **opt)
    prob, tprob = base, prob  # the reference below uses the untransposed operands
    dev = lambda x: to_dev(x if x.size else np.zeros(2, x.dtype))
    C = dev(C0)
    P.bsmm_execute(plan, prob.alpha, dev(tprob.A), dev(tprob.a_off.astype(np.int64)), dev(tprob.B),
                   dev(tprob.b_off.astype(np.int64)), prob.beta, C, dev(off.astype(np.int64)))
    torch.cuda.synchronize()
    P.bsmm_status_device(plan)
    got = C.cpu().numpy()[:C0.size]
    g, w = struct_elements(prob, cs, off, got), struct_elements(prob, cs, off, want)
    if not np.array_equal(g, w):
        bad = np.flatnonzero(g != w)
        raise AssertionError(f"{bad.size} of {g.size} differ; first {bad[:4]}: {g[bad[:4]]} vs {w[bad[:4]]}")
    # against numpy's complex FP64 product
    Pd = _dense(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes) @ \
        _dense(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes)
    ref = C0.copy()
    ro = np.concatenate([[0], np.cumsum(prob.row_sizes.astype(np.int64))])
    co = np.concatenate([[0], np.cumsum(prob.col_sizes.astype(np.int64))])
    for i in range(prob.M):
        for j in range(prob.N):
            if cs[i, j]:
                r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
                t = ref[off[i, j]:off[i, j] + r * c].reshape(r, c)
                t[...] = prob.alpha * Pd[ro[i]:ro[i + 1], co[j]:co[j + 1]] + (prob.beta * t if prob.beta else 0)
    r = struct_elements(prob, cs, off, ref)
    den = float(np.linalg.norm(r))
    return plan, float(np.linalg.norm(g - r)) / den if den > 0 else float(np.linalg.norm(g - r))


@pytest.mark.parametrize("s,mode", [(6, P.BSMM_SPLIT_BF16), (4, P.BSMM_SPLIT_FP16), (3, P.BSMM_SPLIT_BF16)])
@pytest.mark.parametrize("seed", range(5))
def test_small_ragged(seed, s, mode):
    prob = G.as_complex(G.random_small(seed, max_blocks=6, max_size=60), seed)
    _, err = run_c(prob, s, mode)
    assert err <= BARS[s], err


def test_integer_inputs_exact():
    prob = G.as_complex(G.random_small(11, max_blocks=5, max_size=40, values="integers"), 11)
    _, err = run_c(prob, 1)
    assert err == 0.0


def test_nonuniform_dense_clusters():
    prob = G.as_complex(G.make_problem("nonuniform_dense", 3, 700, lo=64, hi=200), 3)
    for cl in (1, 2, 4):
        _, err = run_c(prob, 6, cluster=cl)
        assert err <= 1e-11, err


def test_alpha_beta_c_mask_and_split_k():
    prob = G.as_complex(G.make_problem("banded_decay", 5, 1000, lo=32, hi=200, band=3), 5)
    prob.alpha, prob.beta = -0.75, 1.5
    cm = (np.random.default_rng(2).random((prob.M, prob.N)) < 0.2).astype(np.uint8)
    run_c(prob, 6, P.BSMM_SPLIT_FP16, c_mask=cm)
    run_c(prob, 6, c_mask=cm, ksplit=3)


def test_thin_automatic_split_k():
    prob = G.as_complex(G.make_problem("thin_dense", 4, 260, hi=200, k_factor=40), 4)
    plan, _ = run_c(prob, 6)
    assert P.bsmm_plan_ksplit(plan)["n_regions"] > 0


@pytest.mark.parametrize("trans", [(1, 0), (0, 1), (1, 1)])
def test_transposed_storage(trans):
    """Complex operands supplied as the transposed block matrix: the oracle's bits (those
    of untransposed storage), ragged tiles, a C mask with beta, split k."""
    prob = G.as_complex(G.random_small(21, max_blocks=6, max_size=60), 21)
    _, err = run_c(prob, 6, trans=trans)
    assert err <= 1e-11, err
    prob = G.as_complex(G.make_problem("nonuniform_dense", 8, 600, lo=40, hi=200), 8)
    prob.alpha, prob.beta = 0.5, -1.0
    cm = (np.random.default_rng(3).random((prob.M, prob.N)) < 0.3).astype(np.uint8)
    run_c(prob, 6, P.BSMM_SPLIT_FP16, c_mask=cm, trans=trans)
    run_c(prob, 6, trans=trans, ksplit=2)


@pytest.mark.parametrize("trans", [(0, 0), (1, 1)])
def test_row_column_scaling(trans):
    """One exponent per complex row of A and column of B (over both parts): the row-scaled
    oracle's bits on ragged tiles and on rows and columns scaled up to 40 binades apart,
    where one exponent per tile loses the small lines; with split k as well."""
    prob = G.as_complex(G.random_small(23, max_blocks=6, max_size=60), 23)
    run_c(prob, 6, trans=trans, split_scale=1)
    # complex integers (both parts), then every row of A scaled by its own power of two: each
    # C element is one scale times an exact complex integer sum, so the product is exact
    base = G.as_complex(G.make_problem("nonuniform_dense", 9, 500, lo=40, hi=160, values="integers"), 9)
    rng = np.random.default_rng(9)
    ra = np.ldexp(1.0, -10 * rng.integers(0, 5, int(base.row_sizes.sum())))
    ro = np.concatenate([[0], np.cumsum(base.row_sizes)])
    A = base.A.copy()
    for i in range(base.M):
        for k in range(base.K):
            o = base.a_off[i, k]
            A[o:o + base.row_sizes[i] * base.inner_sizes[k]].reshape(base.row_sizes[i], base.inner_sizes[k])[...] *= \
                ra[ro[i]:ro[i + 1], None]
    prob = dataclasses.replace(base, A=A)
    _, err = run_c(prob, 6, trans=trans, split_scale=1)
    assert err == 0.0, err
    run_c(prob, 6, trans=trans, split_scale=1, ksplit=2)


def test_unsupported_combinations_are_rejected():
    prob = G.as_complex(G.random_small(1, max_blocks=3, max_size=30), 1)
    args = (prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask)
    for bad in (dict(mode=P.BSMM_FP64),):
        with pytest.raises(P.BsmmError):
            P.bsmm_plan(*args, elem=P.BSMM_C128, **bad)


def test_deep_complex_inner_block_runs_in_groups():
    """2 x 300 real inner lines exceed the 6-slice exact FP32 depth (512): the block is
    accumulated in several groups, with the complex oracle's bits."""
    rng = np.random.default_rng(3)
    r, c, q = np.array([40, 70], np.int32), np.array([30, 50], np.int32), np.array([300, 20], np.int32)
    am, bm = np.ones((2, 2), np.uint8), np.ones((2, 2), np.uint8)
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    real = G.Problem("deep_complex", r, c, q, am, bm, a_off, b_off, rng.uniform(-1, 1, at),
                     rng.uniform(-1, 1, bt), 1.0, 0.0)
    _, err = run_c(G.as_complex(real, 4), 6)
    assert err <= 1e-11, err
