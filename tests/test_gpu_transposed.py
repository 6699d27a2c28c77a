"""Transposed operand storage on the GPU (options transa / transb; Sec. 2.1: transposed
multiplies such as C = A B^T): every path gives the oracle's bits for the transposed
arguments, which are also the bits of the untransposed product."""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import c_arena, struct_elements

pytestmark = pytest.mark.gpu
FLAGS = [(True, False), (False, True), (True, True)]


def _cases():
    return [G.random_small(61, max_blocks=6, max_size=90),
            G.make_problem("nonuniform_dense", 62, 700, lo=40, hi=200),
            G.make_problem("clustered", 63, 900, lo=16, hi=160, nclusters=6, cluster_density=0.25)]


def _run(prob, mode, s=6, **kw):
    from gpu_helpers import run_lib
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(5))
    want = C0.copy()
    if mode == P.BSMM_FP64:
        oracle.bsmm(prob, cs, want, off)
    else:
        OS.bsmm_split(prob, cs, want, off, s)
    got, _ = run_lib(prob, cs, C0, off, mode=mode, nslices=s, **kw)
    return struct_elements(prob, cs, off, got), struct_elements(prob, cs, off, want)


@pytest.mark.parametrize("ta,tb", FLAGS)
@pytest.mark.parametrize("mode,s", [(P.BSMM_FP64, 6), (P.BSMM_SPLIT_BF16, 6), (P.BSMM_SPLIT_FP16, 3)])
def test_transposed_matches_oracle_and_untransposed(ta, tb, mode, s):
    for prob in _cases():
        prob.alpha, prob.beta = 1.5, -0.5
        t = G.transposed_storage(prob, ta, tb)
        got_t, want_t = _run(t, mode, s)
        assert np.array_equal(got_t, want_t)
        got, _ = _run(prob, mode, s)
        assert np.array_equal(got, got_t)


def test_fp64_subtile_64_transposed():
    prob = G.transposed_storage(G.make_problem("nonuniform_dense", 64, 600, lo=40, hi=200), True, True)
    from gpu_helpers import run_lib
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(6))
    want = C0.copy()
    oracle.bsmm(prob, cs, want, off)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask, mode=P.BSMM_FP64,
                       fp64_tile=64, transa=1, transb=1, debug_checks=1)
    got, _ = run_lib(prob, cs, C0, off, plan=plan)
    assert np.array_equal(struct_elements(prob, cs, off, got), struct_elements(prob, cs, off, want))


def test_batch_of_mixed_orientations():
    import torch
    base = G.make_batch(4, 65, n_lo=150, n_hi=500, b_lo=24, b_hi=120)
    probs = [G.transposed_storage(p, bool(i & 1), bool(i & 2)) for i, p in enumerate(base)]
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x) if np.asarray(x).size else np.zeros(2)).cuda()
    items = []
    for p in probs:
        cs, _, _ = oracle.structure(p)
        off, C0 = c_arena(p, cs, rng=np.random.default_rng(7))
        plan = P.bsmm_plan(p.row_sizes, p.col_sizes, p.inner_sizes, p.a_mask, p.b_mask, mode=P.BSMM_SPLIT_BF16,
                           nslices=6, transa=int(p.transa), transb=int(p.transb), debug_checks=1)
        items.append(dict(p=p, cs=cs, off=off, C0=C0, plan=plan, A=d(p.A), B=d(p.B), ao=d(p.a_off), bo=d(p.b_off),
                          co=d(off), C=d(C0)))
    batch = P.bsmm_batch_create([it["plan"] for it in items])
    P.bsmm_batch_set_args(batch, [it["p"].alpha for it in items], [it["A"] for it in items],
                          [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                          [it["p"].beta for it in items], [it["C"] for it in items], [it["co"] for it in items])
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    for it in items:
        want = it["C0"].copy()
        OS.bsmm_split(it["p"], it["cs"], want, it["off"], 6)
        got = it["C"].cpu().numpy()
        assert np.array_equal(struct_elements(it["p"], it["cs"], it["off"], got),
                              struct_elements(it["p"], it["cs"], it["off"], want))
