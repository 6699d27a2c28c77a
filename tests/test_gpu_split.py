"""GPU parity of the split-precision tensor-core path, through the C ABI.

Two comparisons per case:
  * against the split oracle (the slicing algorithm's steps in numpy): the tile
    products are summed exactly and rounded once, so the GPU must agree bit for bit
    whatever its accumulation order;
  * against the FP64 oracle, at the stated accuracy bars: 6 slices <= 1e-11 and
    3 slices <= 1e-5 relative Frobenius error.
"""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
import paper_1504_05046_gb300 as P
from helpers import c_arena, rel_fro, struct_elements

pytestmark = pytest.mark.gpu
BARS = {1: 1e-1, 2: 1e-3, 3: 1e-5, 4: 1e-7, 5: 1e-9, 6: 1e-11}


def check(prob, s, mode=P.BSMM_SPLIT_BF16, c_mask=None, bar=None, **kw):
    from gpu_helpers import run_lib
    cs, _, _ = oracle.structure(prob, c_mask)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(0))
    Csplit = C0.copy()
    OS.bsmm_split(prob, cs, Csplit, off, s)
    C64 = C0.copy()
    oracle.bsmm(prob, cs, C64, off)
    Cg, plan = run_lib(prob, cs, C0, off, mode=mode, nslices=s, c_mask=c_mask, **kw)
    got = struct_elements(prob, cs, off, Cg)
    want = struct_elements(prob, cs, off, Csplit)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{bad.size} of {got.size} elements differ from the split oracle; "
                             f"first {bad[:5]}: got {got[bad[:5]]} want {want[bad[:5]]}; "
                             f"rel err {rel_fro(got, want):.3e}")
    err = rel_fro(got, struct_elements(prob, cs, off, C64))
    assert err <= (bar if bar is not None else BARS[s]), err
    return Cg, plan, err


def test_tiny_single_unit():
    rng = np.random.default_rng(0)
    r = np.array([20], np.int32)
    q = np.array([24], np.int32)
    c = np.array([12], np.int32)
    am = np.ones((1, 1), np.uint8)
    bm = np.ones((1, 1), np.uint8)
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    prob = G.Problem("tiny", r, c, q, am, bm, a_off, b_off, rng.integers(-3, 4, at).astype(float),
                     rng.integers(-3, 4, bt).astype(float), 1.0, 0.0)
    check(prob, 1, bar=0.0)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 6])
def test_slices_dense_nonuniform(s):
    prob = G.make_problem("nonuniform_dense", 20 + s, 700, lo=64, hi=256)
    check(prob, s)


@pytest.mark.parametrize("seed", range(6))
def test_small_ragged(seed):
    prob = G.random_small(seed, max_blocks=6, max_size=70)
    check(prob, 6)


def test_fp16_storage_bit_identical_to_bf16():
    prob = G.make_problem("uniform_bernoulli", 3, 600, block=100, density=0.5)
    a, _, _ = check(prob, 6, mode=P.BSMM_SPLIT_BF16)
    b, _, _ = check(prob, 6, mode=P.BSMM_SPLIT_FP16)
    assert np.array_equal(a, b)


def test_banded_decay_wide_range():
    prob = G.make_problem("banded_decay_wide", 5, 1500, lo=32, hi=160, band=4)
    check(prob, 6, mode=P.BSMM_SPLIT_FP16)


def test_clustered_small_blocks():
    prob = G.make_problem("clustered", 6, 1200, lo=16, hi=200, nclusters=8, cluster_density=0.2)
    check(prob, 6)


def test_integer_inputs_equal_fp64():
    prob = G.make_problem("nonuniform_dense", 7, 500, lo=30, hi=120, values="integers")
    Cg, _, err = check(prob, 2, bar=0.0)
    assert err == 0.0


def test_alpha_beta_c_mask():
    prob = G.make_problem("uniform_bernoulli", 8, 450, block=70, density=0.4)
    prob.alpha, prob.beta = 0.5, -2.0
    cm = (np.random.default_rng(3).random((prob.M, prob.N)) < 0.25).astype(np.uint8)
    check(prob, 6, c_mask=cm)


def test_max_depth_inner_block():
    rng = np.random.default_rng(2)
    r = np.array([130, 70], np.int32)
    q = np.array([512, 1, 300], np.int32)
    c = np.array([40, 96], np.int32)
    am = np.ones((2, 3), np.uint8)
    bm = np.ones((3, 2), np.uint8)
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    prob = G.Problem("deep", r, c, q, am, bm, a_off, b_off, rng.uniform(-1, 1, at), rng.uniform(-1, 1, bt), 1.0, 0.0)
    check(prob, 6)


# The kernel's exact accumulator: 128-bit integers in units of 2^L per C element, with
# L = Emax_A(row block) + Emax_B(column block) - 7(s+1) - KERNEL_GUARD_BITS, where Emax is the
# largest exponent of the stored tiles of that tile row (column). A tile pair's term below
# 2^L enters rounded down to a multiple of 2^L, so each such term moves the sum by less
# than 2^L; every other term is exact.
KERNEL_GUARD_BITS = 55


def _window(prob, s):
    """Per C tile (i, j): the kernel's unit exponent L and whether a term of its k-list
    lies below 2^L (tile scaling, untransposed storage)."""
    te = OS.tile_exponent
    eA = {(i, k): te(G.tile_view(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes, i, k))
          for i in range(prob.M) for k in range(prob.K)
          if prob.a_mask[i, k] and prob.row_sizes[i] > 0 and prob.inner_sizes[k] > 0}
    eB = {(k, j): te(G.tile_view(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes, k, j))
          for k in range(prob.K) for j in range(prob.N)
          if prob.b_mask[k, j] and prob.inner_sizes[k] > 0 and prob.col_sizes[j] > 0}
    out = {}
    for i in range(prob.M):
        ea = max((v for (ii, _), v in eA.items() if ii == i), default=0)
        for j in range(prob.N):
            eb = max((v for (_, jj), v in eB.items() if jj == j), default=0)
            L = ea + eb - 7 * (s + 1) - KERNEL_GUARD_BITS
            terms = [eA[i, k] + eB[k, j] - 7 * (s + 1) for k in range(prob.K) if (i, k) in eA and (k, j) in eB]
            out[i, j] = (L, len(terms), any(t < L for t in terms))
    return out


def check_window(prob, s, **kw):
    """Exponent spans beyond the kernel's window: bit for bit with the split oracle on every
    C tile whose terms all lie within it; elsewhere |GPU - oracle| <= n_k 2^L + ulp(oracle)
    (alpha = 1, beta = 0), n_k the tile's k-list length."""
    from gpu_helpers import run_lib
    assert prob.alpha == 1.0 and prob.beta == 0.0
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, fill=0.0)
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, s)
    Cg, _ = run_lib(prob, cs, C0, off, mode=P.BSMM_SPLIT_BF16, nslices=s, **kw)
    win = _window(prob, s)
    below = 0
    for i in range(prob.M):
        for j in range(prob.N):
            if not cs[i, j]:
                continue
            n = int(prob.row_sizes[i]) * int(prob.col_sizes[j])
            g, w = Cg[off[i, j]:off[i, j] + n], want[off[i, j]:off[i, j] + n]
            L, nk, floored = win[i, j]
            if not floored:
                assert np.array_equal(g, w), (i, j)
                continue
            below += 1
            ulp = np.spacing(np.abs(w))
            assert (np.abs(g - w) <= nk * 2.0 ** L + ulp).all(), (i, j)
    return below


def test_exponent_span_beyond_the_kernel_window():
    """Tiles of one row scaled 2^0 .. 2^-120: products more than the kernel's guard width
    below the largest scale lose bits below its accumulator unit; the result stays within
    the stated bound of the exact sum rounded once, and is bit for bit elsewhere."""
    rng = np.random.default_rng(4)
    r = np.array([50, 70], np.int32)
    q = np.array([40, 33, 64, 20], np.int32)
    c = np.array([45, 30], np.int32)
    am = np.ones((2, 4), np.uint8)
    bm = np.ones((4, 2), np.uint8)
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    A = rng.uniform(-1, 1, at)
    B = rng.uniform(-1, 1, bt)
    for k, sc in enumerate([0, -40, -80, -120]):
        for i in range(2):
            o = a_off[i, k]
            A[o:o + r[i] * q[k]] *= 2.0 ** sc
    prob = G.Problem("span", r, c, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)
    assert check_window(prob, 6) > 0
    assert check_window(prob, 3) > 0


def test_far_term_tie_within_the_window_bound():
    """The oracle's tie case 1 + 2^-53 + 2^-150 (1 x 1 tiles): the exact sum rounds up to
    1 + 2^-52; the kernel's unit at this scale is far above 2^-150, so its result may be 1,
    within the bound."""
    one = np.ones(1, np.int32)
    q = np.ones(3, np.int32)
    am, bm = np.ones((1, 3), np.uint8), np.ones((3, 1), np.uint8)
    a_off, at = G.layout_arena(am, one, q)
    b_off, bt = G.layout_arena(bm, q, one)
    A, B = np.zeros(at), np.zeros(bt)
    A[a_off[0, :]] = [1.0, 2.0 ** -53, 2.0 ** -150]
    B[b_off[:, 0]] = 1.0
    prob = G.Problem("tie", one, one, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)
    assert check_window(prob, 6) == 1


@pytest.mark.parametrize("s", [1, 6])
def test_subnormal_result_rounded_once_on_the_grid(s):
    """Terms 1.5 * 2^-1074 and -2^-1144 (1 x 1 tiles; both within the kernel's window):
    the exact sum (1.5 - 2^-70) 2^-1074 rounds once to 2^-1074; rounding to 53 bits first
    would make it a tie and give 2^-1073. Float32 elements: (1.5 - 2^-40) 2^-149 rounds to
    2^-149."""
    from gpu_helpers import to_dev
    import torch
    one = np.ones(1, np.int32)
    q = np.ones(2, np.int32)
    am, bm = np.ones((1, 2), np.uint8), np.ones((2, 1), np.uint8)
    a_off, at = G.layout_arena(am, one, q)
    b_off, bt = G.layout_arena(bm, q, one)
    cs = np.ones((1, 1), np.uint8)
    off, _ = G.layout_arena(cs, one, one)
    for a_vals, b_vals, dt, want in (
            ([1.5 * 2.0 ** -600, -2.0 ** -572], [2.0 ** -474, 2.0 ** -572], np.float64, 2.0 ** -1074),
            ([1.5 * 2.0 ** -80, -2.0 ** -95], [2.0 ** -69, 2.0 ** -94], np.float32, 2.0 ** -149)):
        A, B = np.zeros(at), np.zeros(bt)
        A[a_off[0, :]] = a_vals
        B[b_off[:, 0]] = b_vals
        prob = G.Problem("sub", one, one, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)
        if dt == np.float32:
            prob = G.as_float32(prob)
        C = np.zeros(1, dt)
        OS.bsmm_split(prob, cs, C, off, s)
        assert C[0] == dt(want)
        plan = P.bsmm_plan(one, one, q, am, bm, mode=P.BSMM_SPLIT_BF16, nslices=s, debug_checks=1,
                           elem=P.BSMM_F32 if dt == np.float32 else P.BSMM_F64)
        dC = torch.zeros(1, dtype=torch.float32 if dt == np.float32 else torch.float64, device="cuda")
        args = (plan, 1.0, to_dev(prob.A), to_dev(prob.a_off), to_dev(prob.B), to_dev(prob.b_off), 0.0, dC,
                to_dev(off))
        (P.bsmm_execute_f32 if dt == np.float32 else P.bsmm_execute)(*args)
        P.bsmm_status_device(plan)
        assert dC.cpu().numpy()[0] == dt(want), (dt, dC.cpu().numpy()[0])
        P.bsmm_destroy(plan)


def test_deep_uniform_classes_are_not_merged():
    """Two consecutive k blocks with the same scale class 60 binades below the row block's
    largest tile (a stored A tile whose B partner is absent): their products enter the
    kernel's accumulator rounded down to its unit, block by block, so they must not share
    one TMEM accumulation (a merged group would take one floor of their sum). The result
    stays within the window bound of the exact sum."""
    rng = np.random.default_rng(9)
    r = np.array([128], np.int32)
    q = np.array([16, 16, 16, 16], np.int32)
    c = np.array([32], np.int32)
    am = np.ones((1, 4), np.uint8)
    bm = np.array([[0], [1], [1], [1]], np.uint8)
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    A = rng.uniform(-1, 1, at)
    B = rng.uniform(-1, 1, bt)
    for k in (1, 2, 3):
        A[a_off[0, k]:a_off[0, k] + 128 * 16] *= 2.0 ** -60
    prob = G.Problem("deep_classes", r, c, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)
    for s in (6, 3):
        assert check_window(prob, s) == 1


def test_deep_inner_block_limits():
    """Inner blocks deeper than the exact FP32 depth are accepted with store warps (the
    default) and refused without them; an inner dimension of more than 2^22 elements is
    refused (the 128-bit sums' headroom), all with BSMM_ERR_UNSUPPORTED."""
    P.bsmm_plan([8], [8], [513], [[1]], [[1]], mode=P.BSMM_SPLIT_BF16, nslices=6)
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_plan([8], [8], [513], [[1]], [[1]], mode=P.BSMM_SPLIT_BF16, nslices=6, store_warps=1)
    assert ei.value.status == 5
    q = [8192] * 512 + [1]
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_plan([8], [8], q, np.ones((1, len(q)), np.uint8), np.ones((len(q), 1), np.uint8),
                    mode=P.BSMM_SPLIT_BF16, nslices=6)
    assert ei.value.status == 5


@pytest.mark.parametrize("cluster", [1, 2, 4, -1])
@pytest.mark.parametrize("recipe", ["nonuniform_dense", "clustered", "ragged"])
def test_column_block_group_sizes(cluster, recipe):
    """Units of 1, 2 or 4 column blocks (or the planner's choice, -1), one per CTA of a group: same bits, including
    groups whose last members fall beyond the matrix and CTAs whose own column block has
    no B tile at some k block of the group's list."""
    if recipe == "nonuniform_dense":
        prob = G.make_problem("nonuniform_dense", 31, 777, lo=40, hi=200)
    elif recipe == "clustered":
        prob = G.make_problem("clustered", 32, 1100, lo=16, hi=180, nclusters=7, cluster_density=0.2)
    else:
        prob = G.random_small(33, max_blocks=6, max_size=90)
    check(prob, 6, cluster=cluster)


@pytest.mark.parametrize("ctas", [1, 5, 151])
def test_schedule_independent_bits(ctas):
    prob = G.make_problem("clustered", 9, 900, lo=16, hi=160, nclusters=6, cluster_density=0.25)
    base, plan, _ = check(prob, 6)
    n = P.bsmm_plan_query(plan)["n_units"]
    again, _, _ = check(prob, 6, ctas=ctas, costs=np.random.default_rng(ctas).uniform(1, 5, n))
    assert np.array_equal(base, again)


def _scaled_problem(seed, r, q, c, a_scale, b_scale):
    """Dense problem whose A tile (i,k) is scaled by 2^a_scale(i,k) and B tile (k,j) by 2^b_scale(k,j)."""
    rng = np.random.default_rng(seed)
    r, q, c = (np.asarray(x, np.int32) for x in (r, q, c))
    am = np.ones((len(r), len(q)), np.uint8)
    bm = np.ones((len(q), len(c)), np.uint8)
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    A = rng.uniform(-1, 1, at)
    B = rng.uniform(-1, 1, bt)
    for i in range(len(r)):
        for k in range(len(q)):
            A[a_off[i, k]:a_off[i, k] + r[i] * q[k]] *= 2.0 ** a_scale(i, k)
    for k in range(len(q)):
        for j in range(len(c)):
            B[b_off[k, j]:b_off[k, j] + q[k] * c[j]] *= 2.0 ** b_scale(k, j)
    return G.Problem("scaled", r, c, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)


@pytest.mark.parametrize("case", ["same_position", "shifting_position", "row_tiles_differ", "col_tiles_differ",
                                  "emax_differs"])
def test_merged_accumulation_groups(case):
    """k blocks whose products land at the same binary position share one TMEM
    accumulation (up to the exact depth); the others are drained one by one. Every
    variant must give the split oracle's bits."""
    r = [100, 60, 90, 140]            # 128-row blocks straddle row tiles
    q = [256, 256, 128, 384, 1, 511, 64, 64, 64, 40]  # group depths hitting exactly 512
    c = [50, 20, 70]
    if case == "same_position":       # e_A + e_B constant over k: merged
        fa, fb = (lambda i, k: k % 3), (lambda k, j: -(k % 3))
    elif case == "shifting_position":  # uniform classes whose sums differ: one k block per group
        fa, fb = (lambda i, k: k % 3), (lambda k, j: 0)
    elif case == "row_tiles_differ":   # row blocks whose tiles have different exponents
        fa, fb = (lambda i, k: 3 * (i % 2) - k % 2), (lambda k, j: k % 2)
    elif case == "col_tiles_differ":   # column blocks straddling tiles of different exponents
        fa, fb = (lambda i, k: 0), (lambda k, j: 2 * (j % 2))
    else:                              # one tile lifts its row tile's (column tile's) largest exponent:
        # blocks straddling it share exponents at every other k, so they still merge there
        fa, fb = (lambda i, k: 3 if (i, k) == (1, 2) else 0), (lambda k, j: 2 if (k, j) == (4, 0) else 0)
    prob = _scaled_problem(11, r, q, c, fa, fb)
    for cl in (1, 2):
        check(prob, 6, cluster=cl)
    check(prob, 3)


def test_zero_size_blocks_empty_rows_and_zero_tiles():
    """Zero-size row, column and inner blocks, a row block without A tiles, and stored
    tiles that are all zero (exponent 0, every slice zero)."""
    rng = np.random.default_rng(8)
    r = np.array([0, 33, 0, 165, 1], np.int32)
    q = np.array([17, 0, 80, 3], np.int32)
    c = np.array([64, 0, 9, 130], np.int32)
    am = (rng.random((5, 4)) < 0.7).astype(np.uint8)
    bm = (rng.random((4, 4)) < 0.7).astype(np.uint8)
    am[3, :] = 0
    am[1, :] = 1
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    A, B = rng.uniform(-1, 1, at), rng.uniform(-1, 1, bt)
    o = a_off[1, 2]
    A[o:o + 33 * 80] = 0.0  # an all-zero stored tile
    prob = G.Problem("zeros", r, c, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)
    for s in (6, 3):
        check(prob, s)


def test_empty_product_keeps_beta_c():
    """No nonzero triple: every C tile of the user mask is beta*C."""
    prob = G.random_small(3)
    prob.a_mask[:] = 0
    prob.a_off[:] = -1
    prob.A = np.zeros(0)
    prob.beta = 2.0
    cm = np.ones((prob.M, prob.N), np.uint8)
    check(prob, 6, c_mask=cm, bar=0.0)


def test_beta_zero_ignores_nan_in_c():
    from gpu_helpers import run_lib
    prob = G.make_problem("nonuniform_dense", 5, 300, lo=40, hi=90)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, fill=np.nan)
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, 6)
    Cg, _ = run_lib(prob, cs, C0, off, mode=P.BSMM_SPLIT_BF16, nslices=6)
    got = struct_elements(prob, cs, off, Cg)
    assert not np.isnan(got).any()
    assert np.array_equal(got, struct_elements(prob, cs, off, want))


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_input_is_reported(bad):
    """A NaN or infinity in A has no slicing; the exponent kernel records it in the
    device error word and bsmm_status_device returns BSMM_ERR_DEVICE (no trap)."""
    from gpu_helpers import run_lib
    prob = G.make_problem("nonuniform_dense", 7, 200, lo=40, hi=90)
    prob.A = prob.A.copy()
    prob.A[5] = bad
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(1))
    with pytest.raises(P.BsmmError) as ei:
        run_lib(prob, cs, C0, off, mode=P.BSMM_SPLIT_BF16, nslices=6)
    assert ei.value.status == 6
    # the context stays usable: the same structure with finite values runs clean
    prob.A[5] = 0.25
    check(prob, 6)


def test_stages_option():
    """Every ring depth that fits gives the same bits; one that does not fit is refused."""
    prob = G.make_problem("nonuniform_dense", 12, 600, lo=40, hi=200)
    base, _, _ = check(prob, 6)
    again, _, _ = check(prob, 6, stages=2)
    assert np.array_equal(base, again)
    for st in (2, 4, 6):
        check(prob, 3, stages=st)
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_plan([8], [8], [8], [[1]], [[1]], mode=P.BSMM_SPLIT_BF16, nslices=6, stages=4)
    assert ei.value.status == 5


def test_subnormal_results_match_split_oracle():
    """Tiles scaled by 2^-528 put every result in the subnormal range: the rounding takes its
    library-scaling path for results below the normal range, as the oracle does (one
    rounding to 53 bits, then the scaling)."""
    prob = G.make_problem("nonuniform_dense", 13, 300, lo=40, hi=120)
    prob.A = prob.A * 2.0 ** -528
    prob.B = prob.B * 2.0 ** -528
    from gpu_helpers import run_lib
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, fill=0.0)
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, 6)
    Cg, _ = run_lib(prob, cs, C0, off, mode=P.BSMM_SPLIT_BF16, nslices=6)
    got = struct_elements(prob, cs, off, Cg)
    w = struct_elements(prob, cs, off, want)
    assert np.all(np.abs(w) < 2.0 ** -1022) and np.any(w != 0)
    assert np.array_equal(got, w)


@pytest.mark.parametrize("split_scale", [0, 1])
def test_subnormal_inputs(split_scale):
    """A tiles in the subnormal range (about 2^-1060) and B tiles near 2^1000: the tile and
    line exponents of subnormal maxima follow frexp, as the oracle's do."""
    from gpu_helpers import run_lib
    prob = G.make_problem("nonuniform_dense", 14, 300, lo=40, hi=120)
    prob.A = prob.A * 2.0 ** -1060
    prob.B = prob.B * 2.0 ** 1000
    assert np.any((np.abs(prob.A) < 2.0 ** -1022) & (prob.A != 0))
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, fill=0.0)
    want = C0.copy()
    OS.bsmm_split(prob, cs, want, off, 6, scaling="rows" if split_scale else "tile")
    Cg, _ = run_lib(prob, cs, C0, off, mode=P.BSMM_SPLIT_BF16, nslices=6, split_scale=split_scale)
    assert np.array_equal(struct_elements(prob, cs, off, Cg), struct_elements(prob, cs, off, want))


@pytest.mark.parametrize("cluster,s", [(1, 6), (2, 6), (1, 4), (4, 3)])
@pytest.mark.parametrize("case", ["uniform", "mixed_scales"])
def test_long_k_lists_epilogue_walks(cluster, s, case):
    """Units of about 70 k blocks (inner blocks of 8..24): the planner lets the epilogue
    find the accumulation groups on its own k list instead of taking the MMA warps'
    descriptors. The groups, and so the bits, are the split oracle's: merged groups on
    uniform scales, and lone or shifting groups when tiles are scaled by k."""
    rng = np.random.default_rng(77)
    r = rng.integers(90, 200, 4).astype(np.int32)
    c = rng.integers(20, 90, 5).astype(np.int32)
    q = rng.integers(8, 25, 72).astype(np.int32)
    if case == "uniform":
        fa, fb = (lambda i, k: 0), (lambda k, j: 0)
    else:
        fa, fb = (lambda i, k: (k // 5) % 3 - i % 2), (lambda k, j: (k % 4 == 0) * 2 - j % 2)
    prob = _scaled_problem(78 + cluster, r, q, c, fa, fb)
    prob.alpha, prob.beta = 0.5, -1.5
    check(prob, s, cluster=cluster)


@pytest.mark.parametrize("s", [3, 6])
@pytest.mark.parametrize("layout", ["deep_blocks", "deep_long_lists"])
@pytest.mark.parametrize("cluster", [1, 2])
def test_inner_blocks_deeper_than_the_exact_depth(s, layout, cluster):
    """Inner blocks deeper than the exact FP32 depth (512 for 6 slices, 819 for 3) are
    accumulated in several groups of 32-deep chunks, by the MMA warps and by the walking
    epilogue alike (long k lists), and through the descriptors otherwise; the last group
    of such a block takes the following blocks when they fit. Every bit is the split
    oracle's; blocks up to 1700 deep, tile exponents varying with k."""
    rng = np.random.default_rng(90 + s * 10)
    r = rng.integers(60, 200, 3).astype(np.int32)
    c = rng.integers(20, 90, 4).astype(np.int32)
    if layout == "deep_blocks":
        q = np.array([150, 1700, 33, 290, 512, 513, 900, 64], np.int32)
    else:
        q = np.concatenate([rng.integers(8, 40, 40), [1100], rng.integers(8, 40, 30)]).astype(np.int32)
    fa, fb = (lambda i, k: (k // 3) % 2 - i % 2), (lambda k, j: (k % 5 == 0) - j % 2)
    prob = _scaled_problem(91 + s, r, q, c, fa, fb)
    prob.alpha, prob.beta = 1.25, -0.5
    _, plan, _ = check(prob, s, cluster=cluster)
    f = P.bsmm_plan_form(plan)
    assert f["store_warps"] == 1 and f["epi_walk"] == (1 if layout == "deep_long_lists" else 0)


def _same_sign_problem(seed, r, q, c):
    """Dense problem with entries in [0.997, 0.9999): every first slice is 2^7 and every
    slice-pair product has the same sign, the largest sums the exact accumulation sees."""
    rng = np.random.default_rng(seed)
    r, q, c = (np.asarray(x, np.int32) for x in (r, q, c))
    am = np.ones((len(r), len(q)), np.uint8)
    bm = np.ones((len(q), len(c)), np.uint8)
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    return G.Problem("same_sign", r, c, q, am, bm, a_off, b_off, rng.uniform(0.997, 0.9999, at),
                     rng.uniform(0.997, 0.9999, bt), 1.0, 0.0)


@pytest.mark.parametrize("ksplit", [0, 1])
def test_maximum_inner_dimension_at_full_magnitude(ksplit):
    """The largest inner dimension a split plan takes (2^22 elements in 8192 blocks of 512),
    with same-sign entries at the top of their binade: the 128-bit sums reach about 2^126
    units and must not overflow; bits equal the split oracle's, with k uncut and cut."""
    prob = _same_sign_problem(5, [16], [512] * 8192, [8])
    check(prob, 6, ksplit=ksplit)


@pytest.mark.parametrize("ksplit", [0, 1])
def test_deep_block_beyond_int64_pair_sums(ksplit):
    """A 20000-deep inner block of same-sign entries (its tile pair's integer passes 2^63;
    40 accumulation groups) followed by a shallow block that joins the last group."""
    prob = _same_sign_problem(6, [40, 100], [20000, 100], [30, 40])
    check(prob, 6, ksplit=ksplit)
