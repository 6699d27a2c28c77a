"""Per-row / per-column split scaling on the GPU (split_scale = 1): the row-scaled split
oracle's bits on every path, exactness where the oracle is exact, and per-row accuracy
on graded rows."""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import c_arena, rel_fro, struct_elements
from test_oracle_split_rows import _scaled_integers

pytestmark = pytest.mark.gpu


def check_rows(prob, s=6, mode=P.BSMM_SPLIT_BF16, **kw):
    from gpu_helpers import run_lib
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(2))
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, s, scaling="rows")
    got, _ = run_lib(prob, cs, C0, off, mode=mode, nslices=s, split_scale=1, **kw)
    g, w = struct_elements(prob, cs, off, got), struct_elements(prob, cs, off, want)
    assert np.array_equal(g, w), rel_fro(g, w)
    return g, cs, off


@pytest.mark.parametrize("s", [3, 6])
def test_rows_match_oracle(s):
    for prob in [G.random_small(90, max_blocks=6, max_size=90),
                 G.make_problem("nonuniform_dense", 91, 600, lo=40, hi=200),
                 G.make_problem("clustered", 92, 900, lo=16, hi=160, nclusters=6, cluster_density=0.25),
                 G.make_problem("banded_decay_wide", 93, 1500, lo=32, hi=200, band=3)]:
        prob.alpha, prob.beta = 0.75, 1.5
        check_rows(prob, s)


@pytest.mark.parametrize("cluster", [1, 2, 4])
def test_rows_cluster_sizes_fp16(cluster):
    prob = G.make_problem("nonuniform_dense", 94, 777, lo=40, hi=200)
    check_rows(prob, 6, mode=P.BSMM_SPLIT_FP16, cluster=cluster)


@pytest.mark.parametrize("zero_segments", [False, True])
def test_rows_exact_on_scaled_integers(zero_segments):
    """Rows and columns up to 40 binades apart (rows below 2^-70): the row-scaled path is
    exact, i.e. equal to the FP64 oracle."""
    prob = _scaled_integers(3, zero_segments)
    got, cs, off = check_rows(prob, 6)
    _, ref = c_arena(prob, cs, fill=0.0)
    oracle.bsmm(prob, cs, ref, off)
    assert np.array_equal(got, struct_elements(prob, cs, off, ref))


def test_rows_transposed_storage():
    base = G.make_problem("nonuniform_dense", 95, 500, lo=30, hi=150)
    for ta, tb in [(True, False), (False, True), (True, True)]:
        check_rows(G.transposed_storage(base, ta, tb), 6)


def test_batch_mixed_scaling_modes():
    import torch
    probs = G.make_batch(4, 96, n_lo=150, n_hi=500, b_lo=24, b_hi=120)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x) if np.asarray(x).size else np.zeros(2)).cuda()
    items = []
    for n, p in enumerate(probs):
        cs, _, _ = oracle.structure(p)
        off, C0 = c_arena(p, cs, rng=np.random.default_rng(8))
        plan = P.bsmm_plan(p.row_sizes, p.col_sizes, p.inner_sizes, p.a_mask, p.b_mask, mode=P.BSMM_SPLIT_BF16,
                           nslices=6, split_scale=n % 2, debug_checks=1)
        items.append(dict(p=p, cs=cs, off=off, C0=C0, plan=plan, rows=n % 2, A=d(p.A), B=d(p.B), ao=d(p.a_off),
                          bo=d(p.b_off), co=d(off), C=d(C0)))
    batch = P.bsmm_batch_create([it["plan"] for it in items])
    P.bsmm_batch_set_args(batch, [it["p"].alpha for it in items], [it["A"] for it in items],
                          [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                          [it["p"].beta for it in items], [it["C"] for it in items], [it["co"] for it in items])
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    for it in items:
        want = it["C0"].copy()
        OS.bsmm_split(it["p"], it["cs"], want, it["off"], 6, scaling="rows" if it["rows"] else "tile")
        got = it["C"].cpu().numpy()
        assert np.array_equal(struct_elements(it["p"], it["cs"], it["off"], got),
                              struct_elements(it["p"], it["cs"], it["off"], want))


@pytest.mark.parametrize("cluster", [1, 2])
def test_rows_deep_inner_blocks(cluster):
    """Inner blocks deeper than the exact FP32 depth (700 and 1100 at 6 slices) with one
    scale per row of A and column of B, rows and columns up to 30 binades apart."""
    rng = np.random.default_rng(96)
    r, q, c = np.array([60, 120], np.int32), np.array([700, 64, 1100], np.int32), np.array([40, 70], np.int32)
    am, bm = np.ones((2, 3), np.uint8), np.ones((3, 2), np.uint8)
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    A, B = rng.uniform(-1, 1, at), rng.uniform(-1, 1, bt)
    for i in range(2):
        for k in range(3):
            t = A[a_off[i, k]:a_off[i, k] + r[i] * q[k]].reshape(r[i], q[k])
            t *= 2.0 ** rng.integers(-15, 16, (r[i], 1))
    for k in range(3):
        for j in range(2):
            t = B[b_off[k, j]:b_off[k, j] + q[k] * c[j]].reshape(q[k], c[j])
            t *= 2.0 ** rng.integers(-15, 16, (1, c[j]))
    prob = G.Problem("rows_deep", r, c, q, am, bm, a_off, b_off, A, B, 0.5, -1.0)
    check_rows(prob, 6, cluster=cluster)
