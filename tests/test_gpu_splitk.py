"""GPU parity of split k (Sec. 3.2, Fig. 2: the rank-k updates of a C region run as
multiply tasks on consecutive pieces of its k-list, each into a partial sum, and a
reduction task adds the partials and applies the epilogue), through the C ABI.

* FP64 mode: with a forced cut (ksplit = n) every region's k-list of length L is cut
  into min(n, L) pieces at floor(p L / n'); the FP64 oracle with the same cut (pieces=n)
  fixes every rounding, so the comparison is bit for bit. The automatic cut is compared
  with the plain oracle at the FP64 bar.
* Split modes: the partial sums are exact integers, so any cut must give the split
  oracle's bits.
"""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import c_arena, rel_fro, struct_elements

pytestmark = pytest.mark.gpu
TOL = 1e-13


def _thin(seed, m, k):
    """Few C tiles with long inner sums: M = N = m, K = k (rounded to a multiple of m),
    blocks U-int[64,256], dense masks, U[-1,1]."""
    return G.make_problem("thin_dense", seed, m, k_factor=max(1, k // m))


def _expected_fp64_pieces(prob, cs, n, tile=32):
    """Pieces the forced cut gives: per C tile of S_C with r, c > 0, its sub-tiles times
    min(n, L) when L >= 2 (L = the tile's k-list length)."""
    ptr, _ = oracle.klists(prob)
    regions = pieces = 0
    for i in range(prob.M):
        for j in range(prob.N):
            ri, cj = int(prob.row_sizes[i]), int(prob.col_sizes[j])
            if not cs[i, j] or ri == 0 or cj == 0:
                continue
            L = int(ptr[i * prob.N + j + 1] - ptr[i * prob.N + j])
            nsub = -(-ri // tile) * -(-cj // tile)
            if min(n, L) >= 2:
                regions += nsub
                pieces += nsub * min(n, L)
    return regions, pieces


# ------------------------------------------------------------------------------ FP64
@pytest.mark.parametrize("n", [2, 3, 7])
@pytest.mark.parametrize("seed", range(4))
def test_fp64_forced_cut_bit_exact(seed, n):
    from gpu_helpers import run_lib
    prob = G.random_small(seed, max_blocks=6, max_size=70)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(seed))
    want = C0.copy()
    oracle.bsmm(prob, cs, want, off, pieces=n)
    plain = C0.copy()
    oracle.bsmm(prob, cs, plain, off)
    Cg, plan = run_lib(prob, cs, C0, off, ksplit=n)
    g, w = struct_elements(prob, cs, off, Cg), struct_elements(prob, cs, off, want)
    assert np.array_equal(g, w), rel_fro(g, w)
    assert rel_fro(g, struct_elements(prob, cs, off, plain)) <= TOL
    ks = P.bsmm_plan_ksplit(plan)
    assert (ks["n_regions"], ks["n_pieces"]) == _expected_fp64_pieces(prob, cs, n)


def test_fp64_forced_cut_alpha_beta_c_mask_and_64_tiles():
    from gpu_helpers import run_lib
    prob = G.make_problem("uniform_bernoulli", 3, 500, block=90, density=0.4)
    prob.alpha, prob.beta = -1.5, 0.75
    cm = (np.random.default_rng(4).random((prob.M, prob.N)) < 0.3).astype(np.uint8)
    cs, _, _ = oracle.structure(prob, cm)
    for tile in (32, 64):
        off, C0 = c_arena(prob, cs, rng=np.random.default_rng(1))
        want = C0.copy()
        oracle.bsmm(prob, cs, want, off, pieces=3)
        plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask, cm,
                           mode=P.BSMM_FP64, ksplit=3, fp64_tile=tile, debug_checks=1)
        Cg, _ = run_lib(prob, cs, C0, off, plan=plan)
        assert np.array_equal(struct_elements(prob, cs, off, Cg), struct_elements(prob, cs, off, want)), tile


def test_fp64_automatic_cut_on_thin_product():
    """Few 32x32 regions with long k-lists: asked for automatic cuts in FP64 mode
    (ksplit = -1), the planner cuts them (the grid would idle) and the result stays within
    the FP64 bar of the plain oracle; the default (ksplit = 0) and ksplit = 1 leave FP64
    uncut and give the plain oracle's bits."""
    from gpu_helpers import run_lib
    prob = _thin(3, 200, 6000)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, fill=0.0)
    plain = C0.copy()
    oracle.bsmm(prob, cs, plain, off)
    Cg, plan = run_lib(prob, cs, C0, off, ksplit=-1)
    ks = P.bsmm_plan_ksplit(plan)
    assert ks["n_regions"] > 0 and ks["n_pieces"] > ks["n_regions"]
    g = struct_elements(prob, cs, off, Cg)
    p = struct_elements(prob, cs, off, plain)
    assert rel_fro(g, p) <= TOL
    for k in (0, 1):
        C1, plan1 = run_lib(prob, cs, C0, off, ksplit=k)
        assert P.bsmm_plan_ksplit(plan1)["n_regions"] == 0
        assert np.array_equal(struct_elements(prob, cs, off, C1), p)


def test_fp64_batch_with_cut_products():
    import torch
    from gpu_helpers import to_dev
    probs = [G.random_small(40 + i, max_blocks=5, max_size=60) for i in range(3)]
    runs = []
    for i, prob in enumerate(probs):
        cs, _, _ = oracle.structure(prob)
        off, C0 = c_arena(prob, cs, rng=np.random.default_rng(i))
        want = C0.copy()
        oracle.bsmm(prob, cs, want, off, pieces=2 + i)
        plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                           mode=P.BSMM_FP64, ksplit=2 + i)
        runs.append((prob, cs, off, want, plan, to_dev(C0 if C0.size else np.zeros(2))))
    batch = P.bsmm_batch_create([r[4] for r in runs])
    dev = lambda x: to_dev(x if x.size else np.zeros(2))
    P.bsmm_batch_set_args(batch, [p.alpha for p in probs], [dev(p.A) for p in probs],
                          [to_dev(p.a_off.astype(np.int64)) for p in probs], [dev(p.B) for p in probs],
                          [to_dev(p.b_off.astype(np.int64)) for p in probs], [p.beta for p in probs],
                          [r[5] for r in runs], [to_dev(r[2].astype(np.int64)) for r in runs])
    P.bsmm_batch_execute(batch)
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    for prob, cs, off, want, plan, C in runs:
        got = C.cpu().numpy()
        if want.size:
            assert np.array_equal(struct_elements(prob, cs, off, got), struct_elements(prob, cs, off, want))


# ------------------------------------------------------------------------------ split modes
def _split_check(prob, s, c_mask=None, scaling="tile", **kw):
    from gpu_helpers import run_lib
    cs, _, _ = oracle.structure(prob, c_mask)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(0))
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, s, scaling=scaling)
    Cg, plan = run_lib(prob, cs, C0, off, nslices=s, c_mask=c_mask, split_scale=int(scaling == "rows"), **kw)
    g, w = struct_elements(prob, cs, off, Cg), struct_elements(prob, cs, off, want)
    assert np.array_equal(g, w), rel_fro(g, w)
    return plan


@pytest.mark.parametrize("n", [2, 3, 5, 64])
@pytest.mark.parametrize("seed", range(3))
def test_split_forced_cut_bit_exact(seed, n):
    prob = G.random_small(100 + seed, max_blocks=7, max_size=90)
    for cl in (1, 2, 4):
        plan = _split_check(prob, 6, mode=P.BSMM_SPLIT_BF16, ksplit=n, cluster=cl)
    _split_check(prob, 3, mode=P.BSMM_SPLIT_FP16, ksplit=n)


def test_split_forced_cut_alpha_beta_c_mask_row_scaling():
    prob = G.make_problem("banded_decay_wide", 7, 1500, lo=32, hi=256, band=3)
    prob.alpha, prob.beta = 0.5, -2.0
    cm = (np.random.default_rng(3).random((prob.M, prob.N)) < 0.2).astype(np.uint8)
    _split_check(prob, 6, c_mask=cm, mode=P.BSMM_SPLIT_FP16, ksplit=4)
    _split_check(prob, 6, c_mask=cm, mode=P.BSMM_SPLIT_BF16, ksplit=3, scaling="rows")


def test_split_automatic_cut_on_thin_product():
    """Few 128x64 regions with long k-lists: the planner cuts them (by default and with
    ksplit = -1); the bits equal the split oracle's and an uncut run's."""
    prob = _thin(5, 300, 40000)
    _split_check(prob, 6, mode=P.BSMM_SPLIT_BF16, ksplit=-1)
    plan = _split_check(prob, 6, mode=P.BSMM_SPLIT_BF16)
    ks = P.bsmm_plan_ksplit(plan)
    assert ks["n_regions"] > 0 and ks["n_pieces"] > ks["n_regions"]
    assert (ks["pieces"] > 1).sum() == ks["n_pieces"]
    plan1 = _split_check(prob, 6, mode=P.BSMM_SPLIT_BF16, ksplit=1)
    assert P.bsmm_plan_ksplit(plan1)["n_regions"] == 0


def test_split_cut_independent_of_schedule_and_timings():
    import torch
    from gpu_helpers import run_lib
    prob = _thin(6, 260, 9000)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, fill=0.0)
    outs = []
    for ctas, n in ((None, 5), (7, 5), (1, 13), (None, 1)):
        Cg, plan = run_lib(prob, cs, C0, off, mode=P.BSMM_SPLIT_BF16, ksplit=n, ctas=ctas, record_timings=1)
        t0, t1, cta = P.bsmm_plan_timings(plan)
        assert (t1 >= t0).all() and (t0 > 0).all()
        outs.append(Cg)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_split_batch_with_cut_products():
    import torch
    from gpu_helpers import to_dev
    probs = [G.random_small(60 + i, max_blocks=6, max_size=100) for i in range(3)] + [_thin(8, 200, 5000)]
    runs = []
    for i, prob in enumerate(probs):
        cs, _, _ = oracle.structure(prob)
        off, C0 = c_arena(prob, cs, rng=np.random.default_rng(i))
        want = C0.copy()
        OS.bsmm_split(prob, cs, want, off, 6)
        plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                           mode=P.BSMM_SPLIT_BF16, nslices=6, ksplit=(0, 2, 9, 0)[i])
        runs.append((prob, cs, off, want, plan, to_dev(C0 if C0.size else np.zeros(2))))
    assert P.bsmm_plan_ksplit(runs[-1][4])["n_regions"] > 0
    batch = P.bsmm_batch_create([r[4] for r in runs])
    dev = lambda x: to_dev(x if x.size else np.zeros(2))
    P.bsmm_batch_set_args(batch, [p.alpha for p in probs], [dev(p.A) for p in probs],
                          [to_dev(p.a_off.astype(np.int64)) for p in probs], [dev(p.B) for p in probs],
                          [to_dev(p.b_off.astype(np.int64)) for p in probs], [p.beta for p in probs],
                          [r[5] for r in runs], [to_dev(r[2].astype(np.int64)) for r in runs])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        P.bsmm_batch_execute(batch)
    g.replay()
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    for prob, cs, off, want, plan, C in runs:
        got = C.cpu().numpy()
        if want.size:
            assert np.array_equal(struct_elements(prob, cs, off, got), struct_elements(prob, cs, off, want))


def test_options_validation():
    prob = G.random_small(1)
    for bad in (-2, 65537):
        with pytest.raises(P.BsmmError):
            P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask, ksplit=bad)


def test_transposed_storage_with_cuts():
    """Transposed A and B storage under forced cuts: FP64 matches the oracle's cut bit for
    bit, the split path the split oracle."""
    from gpu_helpers import run_lib
    base = G.random_small(77, max_blocks=6, max_size=60)
    prob = G.transposed_storage(base, True, True)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(3))
    want = C0.copy()
    oracle.bsmm(prob, cs, want, off, pieces=3)
    Cg, _ = run_lib(prob, cs, C0, off, ksplit=3)
    assert np.array_equal(struct_elements(prob, cs, off, Cg), struct_elements(prob, cs, off, want))
    _split_check(prob, 6, mode=P.BSMM_SPLIT_BF16, ksplit=4)
