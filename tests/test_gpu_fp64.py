"""GPU parity of the plain FP64 path against the CPU oracle, through the C ABI.

The oracle's rounding is one fused multiply-add per scalar update in ascending
k (and the epilogue's two separate roundings), which the FP64 kernel follows, so
the comparison is bit for bit; the stated bar (relative Frobenius error <= 1e-13)
is asserted as well."""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
import paper_1504_05046_gb300 as P
from helpers import c_arena, rel_fro, struct_elements

pytestmark = pytest.mark.gpu
TOL = 1e-13


def check(prob, c_mask=None, fill_rng=0, **kw):
    from gpu_helpers import run_lib
    cs, _, _ = oracle.structure(prob, c_mask)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(fill_rng))
    Cref = C0.copy()
    oracle.bsmm(prob, cs, Cref, off)
    Cg, plan = run_lib(prob, cs, C0, off, c_mask=c_mask, **kw)
    got, want = struct_elements(prob, cs, off, Cg), struct_elements(prob, cs, off, Cref)
    assert rel_fro(got, want) <= TOL
    assert np.array_equal(got, want), "FP64 path is not bit-identical to the oracle"
    return Cg, plan


@pytest.mark.parametrize("seed", range(8))
def test_small_ragged(seed):
    prob = G.random_small(seed, max_blocks=6, max_size=70)
    check(prob)


def test_uniform_bernoulli_several_tiles():
    # the uniform-block Bernoulli(0.5) recipe, 6x6 tiles of 128 with a ragged last block
    prob = G.make_problem("uniform_bernoulli", 1, 6 * 128 - 37)
    check(prob)


def test_nonuniform_dense():
    prob = G.make_problem("nonuniform_dense", 2, 700, lo=64, hi=256)
    check(prob)


def test_alpha_beta_and_c_mask():
    prob = G.make_problem("uniform_bernoulli", 3, 400, block=90, density=0.3)
    prob.alpha, prob.beta = -1.5, 0.75
    rng = np.random.default_rng(4)
    cm = (rng.random((prob.M, prob.N)) < 0.3).astype(np.uint8)
    check(prob, c_mask=cm)


def test_beta_zero_ignores_nan_in_c():
    from gpu_helpers import run_lib
    prob = G.make_problem("nonuniform_dense", 5, 300, lo=40, hi=90)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, fill=np.nan)
    Cref = C0.copy()
    oracle.bsmm(prob, cs, Cref, off)
    Cg, _ = run_lib(prob, cs, C0, off)
    assert np.array_equal(struct_elements(prob, cs, off, Cg), struct_elements(prob, cs, off, Cref))


def test_zero_size_blocks_and_empty_rows():
    rng = np.random.default_rng(8)
    r = np.array([0, 33, 0, 65, 1], np.int32)
    q = np.array([17, 0, 80, 3], np.int32)
    c = np.array([64, 0, 9, 130], np.int32)
    am = (rng.random((5, 4)) < 0.7).astype(np.uint8)
    bm = (rng.random((4, 4)) < 0.7).astype(np.uint8)
    am[3, :] = 0  # a row block with no A tiles
    a_off, at = G.layout_arena(am, r, q)
    b_off, bt = G.layout_arena(bm, q, c)
    prob = G.Problem("zeros", r, c, q, am, bm, a_off, b_off, rng.uniform(-1, 1, at), rng.uniform(-1, 1, bt), 1.0, 0.0)
    check(prob)


def test_empty_product():
    prob = G.random_small(3)
    prob.a_mask[:] = 0
    prob.a_off[:] = -1
    prob.A = np.zeros(0)
    prob.beta = 2.0
    cm = np.ones((prob.M, prob.N), np.uint8)
    check(prob, c_mask=cm)


def test_integer_inputs_exact():
    prob = G.make_problem("nonuniform_dense", 6, 500, lo=30, hi=120, values="integers")
    check(prob)


@pytest.mark.parametrize("ctas", [1, 7, 300])
def test_schedule_independent_bits(ctas):
    prob = G.make_problem("uniform_bernoulli", 9, 520, block=64, density=0.6)
    base, plan = check(prob)
    n = P.bsmm_plan_query(plan)["n_units"]
    rng = np.random.default_rng(ctas)
    again, _ = check(prob, ctas=ctas, costs=rng.uniform(1, 10, n))
    assert np.array_equal(base, again)
    nat, _ = check(prob, schedule=P.BSMM_SCHED_NATURAL)
    assert np.array_equal(base, nat)


def test_host_buffers_entry_point():
    prob = G.make_problem("nonuniform_dense", 11, 400, lo=50, hi=150)
    prob.beta = 0.5
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(1))
    Cref = C0.copy()
    oracle.bsmm(prob, cs, Cref, off)
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask)
    C = C0.copy()
    P.bsmm_execute_host(plan, prob.alpha, prob.A, prob.a_off, prob.B, prob.b_off, prob.beta, C, off)
    assert np.array_equal(struct_elements(prob, cs, off, C), struct_elements(prob, cs, off, Cref))


def test_timings_recorded():
    prob = G.make_problem("nonuniform_dense", 12, 600, lo=64, hi=200)
    _, plan = check(prob, record_timings=1)
    s, e, cta = P.bsmm_plan_timings(plan)
    assert np.all(e >= s) and np.all(s > 0)
    n_ctas = P.bsmm_plan_query(plan)["n_units"]
    assert cta.min() >= 0 and cta.max() < max(1, n_ctas)
