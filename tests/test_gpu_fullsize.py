"""GPU parity at the full sizes of the five workloads, in the launch configuration the
benchmark times (default cluster size, ring depth and persistent grid; flop-count
schedule), on sampled C tiles that the oracles compute one by one, plus properties that
hold at any size (S_C equals the boolean product of the masks; results do not depend on
the schedule).

  C1  N=2048, blocks of 128, Bernoulli(0.5) masks, FP64 path: every tile vs the oracle
  C2  N=16384, blocks U-int[64,256], dense: FP64 path and 6-slice bf16 split
  C3  N=32768, blocks U-int[32,256], band |i-j|<=6, N(0,1)exp(-|i-j|/2): FP64 and fp16 split
  C4  256 products of uneven size (n up to 8192), one batch launch replayed from a CUDA graph
  C5  M=N=24576, K=49152, log-uniform blocks [16,512], 40 clusters at 10%: split under two
      schedules
  thin  M=N=512, K=524288 dense: every region's k-list cut (split k)
  C2 with float32 elements, and the 8192 dense product with complex elements
"""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import rel_fro

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    x = np.ascontiguousarray(x)
    return torch.from_numpy(x if x.size else np.zeros(2, x.dtype)).cuda()


class Run:
    """One product planned and executed with the benchmark's defaults; C starts at zero."""

    def __init__(self, prob, mode, nslices=6, **opts):
        import torch
        self.prob = prob
        self.plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                                mode=mode, nslices=nslices, **opts)
        q = P.bsmm_plan_query(self.plan)
        self.cs = q["c_mask"]
        self.off, tot = G.layout_arena(self.cs, prob.row_sizes, prob.col_sizes)
        self.A, self.B = _dev(prob.A), _dev(prob.B)
        self.ao, self.bo, self.co = _dev(prob.a_off), _dev(prob.b_off), _dev(self.off)
        self.C = torch.zeros(max(tot, 1), dtype=torch.float64, device="cuda")

    def execute(self):
        import torch
        P.bsmm_execute(self.plan, self.prob.alpha, self.A, self.ao, self.B, self.bo, self.prob.beta, self.C, self.co)
        torch.cuda.synchronize()
        P.bsmm_status_device(self.plan)
        return self

    def tile(self, i, j):
        o = int(self.off[i, j])
        r, c = int(self.prob.row_sizes[i]), int(self.prob.col_sizes[j])
        return self.C[o:o + r * c].cpu().numpy().reshape(r, c)


def sample_tiles(cs, n, seed):
    """The first and last stored C tiles (the last carries the ragged remainder blocks)
    and n - 2 more drawn at random."""
    idx = np.argwhere(cs)
    rng = np.random.default_rng(seed)
    pick = [0, len(idx) - 1] + list(rng.choice(len(idx), size=max(0, n - 2), replace=False))
    return [tuple(int(v) for v in idx[p]) for p in dict.fromkeys(pick)]


def split_tile(prob, i, j, s):
    """One C tile of the split oracle (beta = 0)."""
    r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
    off = np.full((len(prob.row_sizes), len(prob.col_sizes)), -1, np.int64)
    off[i, j] = 0
    C = np.zeros(r * c)
    OS.bsmm_split(prob, None, C, off, s, tiles=[(i, j)])
    return C.reshape(r, c)


def check_structure(prob, run):
    want, _, _ = oracle.structure(prob)
    assert np.array_equal(run.cs, want)


def check_fp64_tiles(run, tiles):
    for (i, j) in tiles:
        got = run.tile(i, j)
        want = oracle.bsmm_tile(run.prob, i, j)
        assert np.array_equal(got, want), (i, j, rel_fro(got, want))


def check_split_tiles(run, s, tiles_exact, tiles_err, bar):
    for (i, j) in tiles_exact:
        got = run.tile(i, j)
        want = split_tile(run.prob, i, j, s)
        assert np.array_equal(got, want), (i, j, rel_fro(got, want))
    got = np.concatenate([run.tile(i, j).ravel() for (i, j) in tiles_err])
    ref = np.concatenate([oracle.bsmm_tile(run.prob, i, j).ravel() for (i, j) in tiles_err])
    err = rel_fro(got, ref)
    assert err <= bar, err
    return err


# ---------------------------------------------------------------------------- C1
def test_c1_fp64_every_tile():
    prob = G.make_problem("uniform_bernoulli", 2024, 2048, block=128, density=0.5)
    run = Run(prob, P.BSMM_FP64).execute()
    check_structure(prob, run)
    want = np.zeros(run.C.numel())
    oracle.bsmm(prob, run.cs, want, run.off)
    got = run.C.cpu().numpy()
    assert np.array_equal(got, want)
    split = Run(prob, P.BSMM_SPLIT_BF16, 6).execute()
    tiles = sample_tiles(run.cs, 6, 1)
    check_split_tiles(split, 6, tiles[:3], tiles, 1e-11)


# ---------------------------------------------------------------------------- C2
@pytest.fixture(scope="module")
def c2():
    return G.make_problem("nonuniform_dense", 2024, 16384, lo=64, hi=256)


def test_c2_split6_bf16(c2):
    run = Run(c2, P.BSMM_SPLIT_BF16, 6).execute()
    check_structure(c2, run)
    tiles = sample_tiles(run.cs, 4, 2)
    check_split_tiles(run, 6, tiles[:1], tiles, 1e-11)
    # a second launch from zero gives the same bits (no state carried between launches)
    first = run.C.clone()
    run.C.zero_()
    run.execute()
    assert bool((run.C == first).all())


def test_c2_split3_bf16(c2):
    run = Run(c2, P.BSMM_SPLIT_BF16, 3).execute()
    tiles = sample_tiles(run.cs, 3, 3)
    check_split_tiles(run, 3, tiles[-1:], tiles, 1e-5)


def test_c2_fp64(c2):
    run = Run(c2, P.BSMM_FP64).execute()
    check_fp64_tiles(run, sample_tiles(run.cs, 3, 4))


# ---------------------------------------------------------------------------- C3
@pytest.mark.parametrize("recipe", ["banded_decay", "banded_decay_wide"])
def test_c3_banded(recipe):
    prob = G.make_problem(recipe, 2024, 32768, lo=32, hi=256, band=6)
    run64 = Run(prob, P.BSMM_FP64).execute()
    check_structure(prob, run64)
    tiles = sample_tiles(run64.cs, 5, 5)
    check_fp64_tiles(run64, tiles)
    run = Run(prob, P.BSMM_SPLIT_FP16, 6).execute()
    check_split_tiles(run, 6, tiles[:3], tiles, 1e-11)


# ---------------------------------------------------------------------------- C4
def test_c4_batch_graph_full_sizes():
    """The 256 products of the batch workload at their stated sizes (n ~ U-int[512, 8192],
    blocks U-int[32, 192], density ~ U[0.1, 1]) in one batch launch replayed from a CUDA
    graph: sampled tiles of 8 products, the largest among them, bit for bit against the
    split oracle and within the 6-slice bar of the FP64 oracle; two products run on their
    own give the same bits."""
    import torch
    probs = G.make_batch(256, 2024)
    runs = [Run(p, P.BSMM_SPLIT_BF16, 6) for p in probs]
    batch = P.bsmm_batch_create([r.plan for r in runs])
    P.bsmm_batch_set_args(batch, [p.alpha for p in probs], [r.A for r in runs], [r.ao for r in runs],
                          [r.B for r in runs], [r.bo for r in runs], [p.beta for p in probs],
                          [r.C for r in runs], [r.co for r in runs])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        P.bsmm_batch_execute(batch)
    g.replay()
    torch.cuda.synchronize()
    P.bsmm_batch_status_device(batch)
    sizes = np.array([int(p.row_sizes.sum()) for p in probs])
    assert sizes.max() > 7000 and sizes.min() < 1200  # the stated range is covered
    rng = np.random.default_rng(6)
    picks = [int(np.argmax(sizes)), int(np.argmin(sizes))]
    picks += [int(x) for x in rng.choice(len(probs), size=12, replace=False) if int(x) not in picks][:6]
    checked = 0
    for p in picks:
        run = runs[p]
        if not run.cs.any():
            continue
        tiles = sample_tiles(run.cs, 2, p)
        check_split_tiles(run, 6, tiles[:1], tiles, 1e-11)
        checked += 1
    assert checked >= 8
    for p in picks[:2]:
        run = runs[p]
        batched = run.C.clone()
        run.C.zero_()
        run.execute()
        assert bool((run.C == batched).all())


# ---------------------------------------------------------------------------- C5
def test_c5_clustered_two_schedules():
    prob = G.make_problem("clustered", 2024, 24576, lo=16, hi=512, nclusters=40, cluster_density=0.10)
    assert max(prob.inner_sizes) <= 512
    run = Run(prob, P.BSMM_SPLIT_BF16, 6).execute()
    check_structure(prob, run)
    tiles = sample_tiles(run.cs, 3, 7)
    check_split_tiles(run, 6, tiles[:1], tiles, 1e-11)
    first = run.C.clone()
    n = P.bsmm_plan_query(run.plan)["n_units"]
    P.bsmm_plan_set_costs(run.plan, np.random.default_rng(8).uniform(1, 100, n))
    run.C.zero_()
    run.execute()
    assert bool((run.C == first).all())


# ---------------------------------------------------------------- split k, element types
def test_thin_split_k_full_size():
    """The thin workload (M = N = 512, K = 524288) in the benchmark's configuration: the
    planner cuts every region's k-list; a sampled tile matches the split oracle bit for bit
    and the FP64 oracle within the 6-slice bar."""
    prob = G.make_problem("thin_dense", 2024, 512, lo=64, hi=256, k_factor=1024)
    run = Run(prob, P.BSMM_SPLIT_BF16, 6).execute()
    check_structure(prob, run)
    assert P.bsmm_plan_ksplit(run.plan)["n_regions"] > 0
    check_split_tiles(run, 6, [(0, 0)], [(0, 0)], 1e-11)


def test_float32_elements_full_size():
    """The 16384 dense workload with float32 elements: sampled tiles match the float32 split
    oracle bit for bit."""
    import torch
    prob = G.as_float32(G.make_problem("nonuniform_dense", 2024, 16384, lo=64, hi=256))
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, nslices=6, elem=P.BSMM_F32)
    cs = P.bsmm_plan_query(plan)["c_mask"]
    off, tot = G.layout_arena(cs, prob.row_sizes, prob.col_sizes)
    C = torch.zeros(tot, dtype=torch.float32, device="cuda")
    P.bsmm_execute_f32(plan, 1.0, _dev(prob.A), _dev(prob.a_off), _dev(prob.B), _dev(prob.b_off), 0.0, C, _dev(off))
    torch.cuda.synchronize()
    P.bsmm_status_device(plan)
    for (i, j) in sample_tiles(cs, 2, 9):
        r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
        o = int(off[i, j])
        got = C[o:o + r * c].cpu().numpy()
        want = np.zeros(r * c, np.float32)
        offs = np.full((prob.M, prob.N), -1, np.int64)
        offs[i, j] = 0
        OS.bsmm_split(prob, None, want, offs, 6, tiles=[(i, j)])
        assert np.array_equal(got, want), (i, j)


def test_complex_elements_full_size():
    """The 8192 dense product with complex entries (the benchmark's complex line): sampled
    tiles match the complex split oracle bit for bit."""
    import torch
    prob = G.as_complex(G.make_problem("nonuniform_dense", 2031, 8192, lo=64, hi=256), 2031)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, nslices=6, elem=P.BSMM_C128)
    cs = P.bsmm_plan_query(plan)["c_mask"]
    off, tot = G.layout_arena(cs, prob.row_sizes, prob.col_sizes)
    C = torch.zeros(tot, dtype=torch.complex128, device="cuda")
    P.bsmm_execute(plan, 1.0, _dev(prob.A), _dev(prob.a_off), _dev(prob.B), _dev(prob.b_off), 0.0, C, _dev(off))
    torch.cuda.synchronize()
    P.bsmm_status_device(plan)
    for (i, j) in sample_tiles(cs, 2, 10):
        r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
        o = int(off[i, j])
        got = C[o:o + r * c].cpu().numpy()
        want = np.zeros(r * c, np.complex128)
        offs = np.full((prob.M, prob.N), -1, np.int64)
        offs[i, j] = 0
        OS.bsmm_split(prob, None, want, offs, 6, tiles=[(i, j)])
        assert np.array_equal(got, want), (i, j)
