"""Batched products through one persistent launch (eager and replayed from a CUDA
graph) against each product run on its own and against the oracles."""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import c_arena, struct_elements

pytestmark = pytest.mark.gpu


def _setup(mode, count=7, seed=5, fp64_tile=0, probs=None):
    import torch
    if probs is None:
        probs = G.make_batch(count, seed, n_lo=150, n_hi=900, b_lo=24, b_hi=140)
    items = []
    for i, prob in enumerate(probs):
        prob.alpha, prob.beta = [1.0, -0.5, 2.0][i % 3], [0.0, 1.0, 0.5][i % 3]
        cs, _, _ = oracle.structure(prob)
        off, C0 = c_arena(prob, cs, rng=np.random.default_rng(i))
        plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                           mode=mode, nslices=6, debug_checks=1, fp64_tile=fp64_tile)
        d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        items.append(dict(prob=prob, cs=cs, off=off, C0=C0, plan=plan, A=d(prob.A if prob.A.size else np.zeros(2)),
                          B=d(prob.B if prob.B.size else np.zeros(2)), ao=d(prob.a_off), bo=d(prob.b_off), co=d(off),
                          C=d(C0 if C0.size else np.zeros(2))))
    return items


def _reference(it, mode):
    want = it["C0"].copy()
    if mode == P.BSMM_FP64:
        oracle.bsmm(it["prob"], it["cs"], want, it["off"])
    else:
        OS.bsmm_split(it["prob"], it["cs"], want, it["off"], 6)
    return want


def test_batch_rejects_mixed_fp64_subtiles():
    import torch  # noqa: F401
    p1 = P.bsmm_plan([64], [64], [64], [[1]], [[1]], mode=P.BSMM_FP64, fp64_tile=32)
    p2 = P.bsmm_plan([64], [64], [64], [[1]], [[1]], mode=P.BSMM_FP64, fp64_tile=64)
    with pytest.raises(P.BsmmError):
        P.bsmm_batch_create([p1, p2])


@pytest.mark.parametrize("mode", [P.BSMM_FP64, P.BSMM_SPLIT_BF16])
def test_batch_matches_oracle_eager_and_graph(mode):
    import torch
    items = _setup(mode, fp64_tile=32)
    batch = P.bsmm_batch_create([it["plan"] for it in items])
    q = P.bsmm_batch_query(batch)
    assert q["n_units"] == sum(P.bsmm_plan_query(it["plan"])["n_units"] for it in items)
    P.bsmm_batch_set_args(batch, [it["prob"].alpha for it in items], [it["A"] for it in items],
                          [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                          [it["prob"].beta for it in items], [it["C"] for it in items], [it["co"] for it in items])
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    wants = [_reference(it, mode) for it in items]
    for it, want in zip(items, wants):
        got = it["C"].cpu().numpy()
        assert np.array_equal(struct_elements(it["prob"], it["cs"], it["off"], got),
                              struct_elements(it["prob"], it["cs"], it["off"], want))
    # capture the batch into a CUDA graph; replay it from the initial C twice
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        P.bsmm_batch_execute(batch)
    for _ in range(2):
        for it in items:
            if it["C0"].size:
                it["C"].copy_(torch.from_numpy(it["C0"]))
        g.replay()
        torch.cuda.synchronize()
        for it, want in zip(items, wants):
            got = it["C"].cpu().numpy()
            assert np.array_equal(struct_elements(it["prob"], it["cs"], it["off"], got),
                                  struct_elements(it["prob"], it["cs"], it["off"], want))
    P.bsmm_batch_status_device(batch)


def test_batch_reordered_costs_same_bits():
    import torch
    items = _setup(P.BSMM_SPLIT_BF16, count=5, seed=9)
    batch = P.bsmm_batch_create([it["plan"] for it in items])
    args = ([it["prob"].alpha for it in items], [it["A"] for it in items], [it["ao"] for it in items],
            [it["B"] for it in items], [it["bo"] for it in items], [it["prob"].beta for it in items],
            [it["C"] for it in items], [it["co"] for it in items])
    P.bsmm_batch_set_args(batch, *args)
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    first = [it["C"].cpu().numpy().copy() for it in items]
    n = P.bsmm_batch_query(batch)["n_units"]
    P.bsmm_batch_set_costs(batch, np.random.default_rng(1).uniform(1, 100, n))
    for it in items:
        if it["C0"].size:
            it["C"].copy_(torch.from_numpy(it["C0"]))
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    for it, f in zip(items, first):
        assert np.array_equal(it["C"].cpu().numpy(), f)


def test_batch_rejects_mixed_modes():
    import torch  # noqa: F401
    p1 = P.bsmm_plan([64], [64], [64], [[1]], [[1]], mode=P.BSMM_FP64)
    p2 = P.bsmm_plan([64], [64], [64], [[1]], [[1]], mode=P.BSMM_SPLIT_BF16)
    with pytest.raises(P.BsmmError):
        P.bsmm_batch_create([p1, p2])


@pytest.mark.parametrize("mode", [P.BSMM_FP64, P.BSMM_SPLIT_BF16])
def test_autotune_keeps_caller_c_and_bits(mode):
    """Autotuning times every candidate on a scratch C (the caller's C keeps its
    content), then the batch runs under the fastest one and still gives the oracles'
    bits; the original plans stay usable on their own."""
    import torch
    items = _setup(mode, count=5, seed=12, fp64_tile=32)
    batch = P.bsmm_batch_create([it["plan"] for it in items])
    P.bsmm_batch_set_args(batch, [it["prob"].alpha for it in items], [it["A"] for it in items],
                          [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                          [it["prob"].beta for it in items], [it["C"] for it in items], [it["co"] for it in items])
    before = [it["C"].clone() for it in items]
    space = P.bsmm_tune_space(mode, 6)
    chosen, ms = P.bsmm_batch_autotune(batch, reps=2)
    assert chosen in space and len(ms) == len(space)
    assert all(np.isfinite(ms)) and min(ms) == ms[space.index(chosen)]
    for it, b in zip(items, before):
        assert bool((it["C"] == b).all())
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    for it in items:
        want = _reference(it, mode)
        got = it["C"].cpu().numpy()
        assert np.array_equal(struct_elements(it["prob"], it["cs"], it["off"], got),
                              struct_elements(it["prob"], it["cs"], it["off"], want))
    # a second autotune (over a narrower space) re-plans from the tuned plans
    P.bsmm_batch_autotune(batch, candidates=space[:2], reps=1)
    it = items[0]
    it["C"].copy_(torch.from_numpy(it["C0"] if it["C0"].size else np.zeros(2)))
    from gpu_helpers import run_lib
    alone, _ = run_lib(it["prob"], it["cs"], it["C0"], it["off"], mode=mode, plan=it["plan"])
    assert np.array_equal(struct_elements(it["prob"], it["cs"], it["off"], alone),
                          struct_elements(it["prob"], it["cs"], it["off"], _reference(it, mode)))


@pytest.mark.parametrize("mode", [P.BSMM_FP64, P.BSMM_SPLIT_BF16])
def test_autotune_cache_file(mode, tmp_path):
    """The tuning cache: the first call tunes and writes the file (keyed by GPU, mode and
    slice count); a second batch takes the cached choice without timing; a file of
    another format is tuned over and replaced; results keep the oracles' bits."""
    import json
    import torch
    path = tmp_path / "tune.json"

    def make():
        items = _setup(mode, count=4, seed=14, fp64_tile=32)
        batch = P.bsmm_batch_create([it["plan"] for it in items])
        P.bsmm_batch_set_args(batch, [it["prob"].alpha for it in items], [it["A"] for it in items],
                              [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                              [it["prob"].beta for it in items], [it["C"] for it in items], [it["co"] for it in items])
        return items, batch

    def check(items, batch):
        for it in items:
            it["C"].copy_(torch.from_numpy(it["C0"] if it["C0"].size else np.zeros(2)))
        P.bsmm_batch_execute(batch)
        torch.cuda.synchronize()
        P.bsmm_batch_status_device(batch)
        for it in items:
            got = it["C"].cpu().numpy()
            assert np.array_equal(struct_elements(it["prob"], it["cs"], it["off"], got),
                                  struct_elements(it["prob"], it["cs"], it["off"], _reference(it, mode)))

    items, batch = make()
    chosen, cached = P.bsmm_batch_autotune_cached(batch, path, reps=1)
    assert not cached and chosen in P.bsmm_tune_space(mode, 6)
    doc = json.loads(path.read_text())
    assert doc["format"] == "bsmm-tune" and doc["version"] == 1 and len(doc["entries"]) == 1
    entry = doc["entries"][0]
    assert entry["key"].endswith("|fp64|s=0" if mode == P.BSMM_FP64 else "|split_bf16|s=6")
    assert (entry["cluster"], entry["stages"], entry["fp64_tile"]) == (chosen["cluster"], chosen["stages"],
                                                                      chosen["fp64_tile"])
    check(items, batch)
    items2, batch2 = make()
    chosen2, cached2 = P.bsmm_batch_autotune_cached(batch2, path, reps=1)
    assert cached2 and chosen2 == chosen
    check(items2, batch2)
    path.write_text('{"format": "something-else", "version": 1}\n')
    items3, batch3 = make()
    _, cached3 = P.bsmm_batch_autotune_cached(batch3, path, reps=1)
    assert not cached3 and json.loads(path.read_text())["format"] == "bsmm-tune"
    check(items3, batch3)


def test_batch_waves_on_two_streams_same_bits_as_separate():
    """Products whose slice workspaces (about 61 MB each) make every one a wave of its own,
    with small products between them: the waves alternate between the caller's stream and
    the batch's second one. Eager and graph-replayed, every C has the bits of the product
    run on its own."""
    import torch
    probs = [G.make_problem("nonuniform_dense", 40 + i, 1600, lo=64, hi=256) if i % 2 == 0 else
             G.make_problem("clustered", 40 + i, 500, lo=16, hi=120, nclusters=4, cluster_density=0.3)
             for i in range(6)]
    items = []
    for i, prob in enumerate(probs):
        prob.alpha, prob.beta = [1.0, -0.5, 2.0][i % 3], [0.0, 1.0, 0.5][i % 3]
        cs, _, _ = oracle.structure(prob)
        off, C0 = c_arena(prob, cs, rng=np.random.default_rng(i))
        plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                           mode=P.BSMM_SPLIT_BF16, nslices=6)
        d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        items.append(dict(prob=prob, C0=C0, plan=plan, A=d(prob.A), B=d(prob.B), ao=d(prob.a_off),
                          bo=d(prob.b_off), co=d(off), C=d(C0)))
    wants = []
    for it in items:
        C = torch.from_numpy(it["C0"].copy()).cuda()
        P.bsmm_execute(it["plan"], it["prob"].alpha, it["A"], it["ao"], it["B"], it["bo"], it["prob"].beta, C,
                       it["co"])
        wants.append(C.cpu().numpy())
    batch = P.bsmm_batch_create([it["plan"] for it in items])
    P.bsmm_batch_set_args(batch, [it["prob"].alpha for it in items], [it["A"] for it in items],
                          [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                          [it["prob"].beta for it in items], [it["C"] for it in items], [it["co"] for it in items])
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    for it, want in zip(items, wants):
        assert np.array_equal(it["C"].cpu().numpy(), want)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        P.bsmm_batch_execute(batch)
    for _ in range(2):
        for it in items:
            it["C"].copy_(torch.from_numpy(it["C0"]))
        g.replay()
        torch.cuda.synchronize()
        for it, want in zip(items, wants):
            assert np.array_equal(it["C"].cpu().numpy(), want)
    P.bsmm_batch_status_device(batch)


def _deep_probs():
    """Three ordinary products and two with inner blocks deeper than the exact FP32 depth
    (700, 900, 1300 at 6 slices)."""
    rng = np.random.default_rng(12)
    probs = G.make_batch(3, 8, n_lo=150, n_hi=500, b_lo=24, b_hi=140)
    for t, q in enumerate(([700, 40, 1300], [64, 900])):
        q = np.array(q, np.int32)
        r = rng.integers(30, 150, 2).astype(np.int32)
        c = rng.integers(20, 90, 3).astype(np.int32)
        am = np.ones((2, len(q)), np.uint8)
        bm = (rng.random((len(q), 3)) < 0.7).astype(np.uint8)
        bm[:, 0] = 1
        a_off, at = G.layout_arena(am, r, q)
        b_off, bt = G.layout_arena(bm, q, c)
        probs.insert(2 * t, G.Problem(f"deep{t}", r, c, q, am, bm, a_off, b_off, rng.uniform(-1, 1, at),
                                      rng.uniform(-1, 1, bt), 1.0, 0.0))
    return probs


def _check_batch_bits(items):
    for it in items:
        want = _reference(it, P.BSMM_SPLIT_BF16)
        got = it["C"].cpu().numpy()
        assert np.array_equal(struct_elements(it["prob"], it["cs"], it["off"], got),
                              struct_elements(it["prob"], it["cs"], it["off"], want)), it["prob"].name


def test_batch_with_deep_inner_blocks():
    """Deep inner blocks batched with ordinary products: the wave runs the deep kernel
    form, and every product gets the split oracle's bits."""
    import torch
    items = _setup(P.BSMM_SPLIT_BF16, probs=_deep_probs())
    batch = P.bsmm_batch_create([it["plan"] for it in items])
    P.bsmm_batch_set_args(batch, [it["prob"].alpha for it in items], [it["A"] for it in items],
                          [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                          [it["prob"].beta for it in items], [it["C"] for it in items], [it["co"] for it in items])
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    _check_batch_bits(items)


def test_autotune_skips_forms_without_deep_blocks():
    """Autotuning a batch with deep inner blocks: the 12-warp candidates cannot take them
    (their plans are refused) and are skipped with an infinite time; the batch keeps a
    store-warp form and the oracle's bits."""
    import torch
    items = _setup(P.BSMM_SPLIT_BF16, probs=_deep_probs())
    batch = P.bsmm_batch_create([it["plan"] for it in items])
    P.bsmm_batch_set_args(batch, [it["prob"].alpha for it in items], [it["A"] for it in items],
                          [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                          [it["prob"].beta for it in items], [it["C"] for it in items], [it["co"] for it in items])
    cands = [dict(cluster=1, stages=3, fp64_tile=0, store_warps=sw) for sw in (1, 2)] + \
            [dict(cluster=2, stages=3, fp64_tile=0, store_warps=sw) for sw in (1, 2)]
    chosen, ms = P.bsmm_batch_autotune(batch, candidates=cands, reps=1)
    assert ms[0] == np.inf and ms[2] == np.inf and np.isfinite(ms[1]) and np.isfinite(ms[3])
    assert chosen["store_warps"] == 2
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    _check_batch_bits(items)
