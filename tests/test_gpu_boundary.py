"""The boundary's one-call batch (bsmm_execute_batch), the learned schedule's checkpoint
(bsmm_mlp_save / bsmm_mlp_load, bsmm_options.model_path) and host-buffer products in
flight (bsmm_execute_host_async / bsmm_host_wait), through the C ABI. None may change a
single bit of any result: only the order of the work units, or of the copies, does."""
import copy

import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import c_arena, struct_elements

pytestmark = pytest.mark.gpu


def _items(count=5, seed=11):
    import torch
    probs = G.make_batch(count, seed, n_lo=150, n_hi=700, b_lo=24, b_hi=140)
    items = []
    for i, prob in enumerate(probs):
        prob.alpha, prob.beta = [1.0, -0.5, 2.0][i % 3], [0.0, 1.0, 0.5][i % 3]
        cs, _, _ = oracle.structure(prob)
        off, C0 = c_arena(prob, cs, rng=np.random.default_rng(i))
        plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                           mode=P.BSMM_SPLIT_BF16, nslices=6, debug_checks=1)
        d = lambda x: torch.from_numpy(np.ascontiguousarray(x if x.size else np.zeros(2, x.dtype))).cuda()
        items.append(dict(prob=prob, cs=cs, off=off, C0=C0, plan=plan, A=d(prob.A), B=d(prob.B), ao=d(prob.a_off),
                          bo=d(prob.b_off), co=d(off), C=d(C0)))
    return items


def _one_call(items, Cs=None):
    P.bsmm_execute_batch([it["plan"] for it in items], [it["prob"].alpha for it in items], [it["A"] for it in items],
                         [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                         [it["prob"].beta for it in items], Cs or [it["C"] for it in items],
                         [it["co"] for it in items])


def test_execute_batch_one_call_matches_the_oracle_repeatedly_and_in_a_graph():
    import torch
    items = _items()
    wants = []
    for it in items:
        w = it["C0"].copy()
        OS.bsmm_split(it["prob"], it["cs"], w, it["off"], 6)
        wants.append(struct_elements(it["prob"], it["cs"], it["off"], w))

    def check(Cs):
        torch.cuda.synchronize()
        for it, C, want in zip(items, Cs, wants):
            got = struct_elements(it["prob"], it["cs"], it["off"], C.cpu().numpy())
            assert np.array_equal(got, want)

    _one_call(items)                       # first call: the batch is created and set up
    check([it["C"] for it in items])
    for it in items:                       # same arguments: kernels only
        it["C"].copy_(torch.from_numpy(it["C0"] if it["C0"].size else np.zeros(2)))
    _one_call(items)
    check([it["C"] for it in items])
    fresh = [torch.from_numpy(it["C0"].copy() if it["C0"].size else np.zeros(2)).cuda() for it in items]
    _one_call(items, fresh)                # new C pointers: arguments re-uploaded
    check(fresh)
    # with the arguments of the previous call, the call only enqueues kernels: capture it
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        _one_call(items, fresh)
    for C, it in zip(fresh, items):
        C.copy_(torch.from_numpy(it["C0"] if it["C0"].size else np.zeros(2)))
    g.replay()
    check(fresh)
    for it in items:
        P.bsmm_status_device(it["plan"])


def test_execute_batch_after_plans_are_replaced():
    """A new plan list (even one reusing freed plans' memory) gets its own batch; results
    stay exact."""
    import torch
    for seed in (21, 22, 23, 24, 25, 26):
        items = _items(count=3, seed=seed)
        _one_call(items)
        torch.cuda.synchronize()
        for it in items:
            w = it["C0"].copy()
            OS.bsmm_split(it["prob"], it["cs"], w, it["off"], 6)
            got = struct_elements(it["prob"], it["cs"], it["off"], it["C"].cpu().numpy())
            assert np.array_equal(got, struct_elements(it["prob"], it["cs"], it["off"], w))
        del items


def _clustered():
    return G.make_problem("clustered", 41, 2000, lo=16, hi=200, nclusters=8, cluster_density=0.2)


def test_mlp_file_round_trip(tmp_path):
    m = P.bsmm_mlp_create(7)
    n = P.bsmm_mlp_num_params()
    prm = np.random.default_rng(1).normal(0, 0.3, n).astype(np.float32)
    P.bsmm_mlp_set_params(m, prm)
    xm = np.arange(12, dtype=np.float32)
    xs = np.linspace(0.5, 2.0, 12).astype(np.float32)
    P.bsmm_mlp_set_norm(m, xm, xs, 1.5, 0.25)
    P.bsmm_mlp_save(m, tmp_path / "cost.bin")
    m2 = P.bsmm_mlp_load(tmp_path / "cost.bin")
    assert np.array_equal(P.bsmm_mlp_get_params(m2), prm)
    nm = P.bsmm_mlp_get_norm(m2)
    assert np.array_equal(nm[0], xm) and np.array_equal(nm[1], xs) and nm[2:] == (1.5, 0.25)


def test_model_path_schedules_by_the_saved_model_with_the_same_bits(tmp_path):
    """A plan built with model_path packs its units by the file's predictions, exactly as
    bsmm_plan_predict_costs with the same model does; a missing or damaged file leaves the
    flop-count schedule. Every variant gives the same bits."""
    import torch
    from gpu_helpers import run_lib
    prob = _clustered()
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(2))
    m = P.bsmm_mlp_create(3)
    P.bsmm_mlp_set_params(m, np.random.default_rng(4).normal(0, 0.5, P.bsmm_mlp_num_params()).astype(np.float32))
    path = tmp_path / "cost.bin"
    P.bsmm_mlp_save(m, path)
    mk = lambda **kw: P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                                  mode=P.BSMM_SPLIT_BF16, nslices=6, **kw)
    flops = mk()
    assert P.bsmm_plan_cost_source(flops) == P.BSMM_COSTS_FLOPS
    learned = mk(model_path=path)
    assert P.bsmm_plan_cost_source(learned) == P.BSMM_COSTS_MODEL
    given = mk()
    P.bsmm_plan_predict_costs(given, m)
    assert P.bsmm_plan_cost_source(given) == P.BSMM_COSTS_GIVEN
    missing = mk(model_path=tmp_path / "none.bin")
    assert P.bsmm_plan_cost_source(missing) == P.BSMM_COSTS_FLOPS
    raw = bytearray(path.read_bytes())
    raw[40] ^= 0xFF
    (tmp_path / "bad.bin").write_bytes(bytes(raw))
    damaged = mk(model_path=tmp_path / "bad.bin")
    assert P.bsmm_plan_cost_source(damaged) == P.BSMM_COSTS_FLOPS
    outs = [run_lib(prob, cs, C0, off, plan=pl)[0] for pl in (flops, learned, given, missing, damaged)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, 6)
    assert np.array_equal(struct_elements(prob, cs, off, outs[0]), struct_elements(prob, cs, off, want))
    torch.cuda.synchronize()


def _elem_problem(elem, seed):
    """A small ragged product in the element type (float32 arenas re-laid on 16-byte tile
    starts; complex arenas with imaginary parts of their own)."""
    prob = G.make_problem("nonuniform_dense", seed, 420, lo=40, hi=160)
    prob.alpha, prob.beta = 0.75, -0.5
    if elem == P.BSMM_F32:
        return G.as_float32(prob)
    if elem == P.BSMM_C128:
        return G.as_complex(prob, seed)
    return prob


def _c0(prob, cs, off, elem, seed):
    _, C64 = c_arena(prob, cs, rng=np.random.default_rng(seed))
    if elem == P.BSMM_F32:
        return C64.astype(np.float32)
    if elem == P.BSMM_C128:
        return (C64 + 1j * np.random.default_rng(seed + 1).uniform(-1, 1, C64.size)).astype(np.complex128)
    return C64


@pytest.mark.parametrize("elem", [P.BSMM_F64, P.BSMM_F32, P.BSMM_C128])
def test_execute_host_every_element_type(elem):
    """bsmm_execute_host with host arenas of the plan's element type: the oracle's bits."""
    prob = _elem_problem(elem, 31)
    cs, _, _ = oracle.structure(prob)
    off, _ = G.layout_arena(cs, prob.row_sizes, prob.col_sizes)
    C0 = _c0(prob, cs, off, elem, 3)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, nslices=6, elem=elem, debug_checks=1)
    C = C0.copy()
    P.bsmm_execute_host(plan, prob.alpha, prob.A, prob.a_off, prob.B, prob.b_off, prob.beta, C, off)
    P.bsmm_status_device(plan)
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, 6)
    assert np.array_equal(struct_elements(prob, cs, off, C), struct_elements(prob, cs, off, want))


def test_batch_of_mixed_element_types():
    """One batch holding float64, float32 and complex products (split mode): every product
    gets the bits of its own oracle, in one launch and replayed from a CUDA graph."""
    import torch
    from gpu_helpers import to_dev
    elems = [P.BSMM_F64, P.BSMM_F32, P.BSMM_C128, P.BSMM_F32, P.BSMM_F64]
    items = []
    for n, elem in enumerate(elems):
        prob = _elem_problem(elem, 50 + n)
        cs, _, _ = oracle.structure(prob)
        off, _ = G.layout_arena(cs, prob.row_sizes, prob.col_sizes)
        C0 = _c0(prob, cs, off, elem, n)
        want = C0.copy()
        OS.bsmm_split(prob, cs, want, off, 6)
        plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                           mode=P.BSMM_SPLIT_BF16, nslices=6, elem=elem, debug_checks=1)
        items.append(dict(prob=prob, cs=cs, off=off, C0=C0, want=want, plan=plan, A=to_dev(prob.A), B=to_dev(prob.B),
                          ao=to_dev(prob.a_off), bo=to_dev(prob.b_off), co=to_dev(off), C=to_dev(C0)))
    batch = P.bsmm_batch_create([it["plan"] for it in items])
    P.bsmm_batch_set_args(batch, [it["prob"].alpha for it in items], [it["A"] for it in items],
                          [it["ao"] for it in items], [it["B"] for it in items], [it["bo"] for it in items],
                          [it["prob"].beta for it in items], [it["C"] for it in items], [it["co"] for it in items])

    def check():
        torch.cuda.synchronize()
        P.bsmm_batch_status_device(batch)
        for it in items:
            got = struct_elements(it["prob"], it["cs"], it["off"], it["C"].cpu().numpy())
            assert np.array_equal(got, struct_elements(it["prob"], it["cs"], it["off"], it["want"]))

    P.bsmm_batch_execute(batch)
    check()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        P.bsmm_batch_execute(batch)
    for it in items:
        it["C"].copy_(torch.from_numpy(it["C0"]))
    g.replay()
    check()


def test_host_products_in_flight_match_the_oracle():
    """Five host-buffer products enqueued on one plan before a single wait: staging slots
    alternate, the copies of one overlap the kernels of another, beta = 0 and beta != 0 mix,
    pinned and pageable host arrays mix, and one product's longer A arena makes its slot
    grow while the slot's previous product may still be in flight. Each C gets exactly the
    oracle's bits for its own inputs."""
    import torch
    prob = _elem_problem(P.BSMM_F64, 37)
    cs, _, _ = oracle.structure(prob)
    off, _ = G.layout_arena(cs, prob.row_sizes, prob.col_sizes)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, nslices=6, debug_checks=1)
    rng = np.random.default_rng(5)
    runs = []
    for i in range(5):
        pi = copy.copy(prob)
        pi.A = rng.uniform(-1, 1, prob.A.size)
        pi.B = rng.uniform(-1, 1, prob.B.size) * 2.0 ** (i - 2)
        pi.alpha, pi.beta = [1.0, -0.5, 3.0, 0.25, 1.0][i], [0.0, 1.0, 0.0, -2.0, 0.5][i]
        _, C0 = c_arena(pi, cs, rng=np.random.default_rng(100 + i))
        A = np.concatenate([pi.A, np.zeros(4096)]) if i == 3 else pi.A
        if i % 2 == 0:  # pinned host memory
            A, B, C = (torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (A, pi.B, C0))
        else:
            B, C = pi.B.copy(), C0.copy()
        runs.append((pi, C0, A, B, C))
    for pi, _, A, B, C in runs:
        P.bsmm_execute_host_async(plan, pi.alpha, A, prob.a_off, B, prob.b_off, pi.beta, C, off)
    P.bsmm_host_wait(plan)
    P.bsmm_status_device(plan)
    for pi, C0, _, _, C in runs:
        got = C.numpy() if hasattr(C, "numpy") else C
        want = C0.copy()
        OS.bsmm_split(pi, cs, want, off, 6)
        assert np.array_equal(struct_elements(pi, cs, off, got), struct_elements(pi, cs, off, want))
    # the synchronous form after them, on the same slots
    pi, C0, _, _, _ = runs[1]
    C = C0.copy()
    P.bsmm_execute_host(plan, pi.alpha, pi.A, prob.a_off, pi.B, prob.b_off, pi.beta, C, off)
    want = C0.copy()
    OS.bsmm_split(pi, cs, want, off, 6)
    assert np.array_equal(struct_elements(pi, cs, off, C), struct_elements(pi, cs, off, want))


def test_plan_form_reports_the_planners_choices():
    """bsmm_plan_form: a dense pattern whose column blocks fill groups of 4 exactly gets
    groups of 4 from cluster = -1, a sparse clustered one groups of 1; long k lists (72
    inner blocks) get the walking epilogue with 3 to 6 slices and store warps, and not with
    2 slices, without store warps or with short lists; FP64 plans report the neutral form."""
    dense = G.make_problem("nonuniform_dense", 5, 1024, lo=64, hi=200)
    f = P.bsmm_plan_form(P.bsmm_plan(dense.row_sizes, dense.col_sizes, dense.inner_sizes, dense.a_mask,
                                     dense.b_mask, mode=P.BSMM_SPLIT_BF16, nslices=6, cluster=-1))
    assert f["cluster"] == 4 and f["store_warps"] == 1 and f["epi_walk"] == 0 and f["stages"] >= 2
    f = P.bsmm_plan_form(P.bsmm_plan(dense.row_sizes, dense.col_sizes, dense.inner_sizes, dense.a_mask,
                                     dense.b_mask, mode=P.BSMM_SPLIT_BF16, nslices=6))
    assert f["cluster"] == 1
    sparse = G.make_problem("clustered", 6, 3000, lo=16, hi=160, nclusters=5, cluster_density=0.2)
    f = P.bsmm_plan_form(P.bsmm_plan(sparse.row_sizes, sparse.col_sizes, sparse.inner_sizes, sparse.a_mask,
                                     sparse.b_mask, mode=P.BSMM_SPLIT_BF16, nslices=6, cluster=-1))
    assert f["cluster"] == 1 and f["epi_walk"] == 0
    rng = np.random.default_rng(8)
    r, c = rng.integers(90, 200, 3).astype(np.int32), rng.integers(20, 90, 4).astype(np.int32)
    q = rng.integers(8, 25, 72).astype(np.int32)
    am, bm = np.ones((3, 72), np.uint8), np.ones((72, 4), np.uint8)
    walk = lambda **o: P.bsmm_plan_form(P.bsmm_plan(r, c, q, am, bm, mode=P.BSMM_SPLIT_BF16, **o))["epi_walk"]
    assert walk(nslices=6) == 1 and walk(nslices=3) == 1
    assert walk(nslices=2) == 0 and walk(nslices=6, store_warps=1) == 0
    f = P.bsmm_plan_form(P.bsmm_plan(r, c, q, am, bm, mode=P.BSMM_FP64))
    assert (f["cluster"], f["store_warps"], f["epi_walk"], f["stages"]) == (1, 0, 0, 0) and f["ctas"] >= 1
