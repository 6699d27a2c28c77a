"""Pins of the FP64 CPU oracle against facts fixed outside it (no GPU).

Each test is chosen so that a plausible slip in the oracle (dropped alpha or beta,
a transposed operand, a wrong tile index or offset, a skipped or duplicated k
block, a mask ANDed the wrong way) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import bsmm_gen as G
import oracle
from helpers import (c_arena, dense_reference, exact_tile_fraction, golden_problem, parse_matrix,
                     read_golden, rel_fro, struct_elements)


# ------------------------------------------------------------------------------------------
# hand-worked golden example (paper Sec. 2.1 definition; values worked by hand)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["case1", "case2"])
def test_golden_hand_product(case):
    g = read_golden("tiny_hand_product.txt")
    alpha, beta = float(g[f"{case}_alpha"]), float(g[f"{case}_beta"])
    prob = golden_problem(g, alpha, beta)
    cmask = parse_matrix(g[f"{case}_c_mask"]).astype(np.uint8) if f"{case}_c_mask" in g else None
    cs, nt, fl = oracle.structure(prob, cmask)
    assert nt == int(g["triples"])
    assert fl == float(g["flops"])
    expect_struct = parse_matrix(g["c_struct"]).astype(np.uint8)
    if cmask is not None:
        expect_struct = expect_struct | cmask
    assert np.array_equal(cs, expect_struct)
    off, C = c_arena(prob, cs, fill=1.0)
    oracle.bsmm(prob, cs, C, off)
    for i, j in itertools.product(range(prob.M), range(prob.N)):
        key = f"{case} C {i}{j}"
        if cs[i, j]:
            want = parse_matrix(g[key])
            o = off[i, j]
            got = C[o:o + want.size].reshape(want.shape)
            assert np.array_equal(got, want), (key, got, want)
        else:
            assert key not in g


# ------------------------------------------------------------------------------------------
# structure: boolean product, triples, flop count, k-lists (brute force)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_structure_brute_force(seed):
    prob = G.random_small(seed, max_blocks=7, max_size=9)
    rng = np.random.default_rng(seed + 100)
    cm = (rng.random((prob.M, prob.N)) < 0.2).astype(np.uint8) if seed % 2 else None
    cs, nt, fl = oracle.structure(prob, cm)
    bt, bf = 0, 0
    for i in range(prob.M):
        for j in range(prob.N):
            hit = False
            for k in range(prob.K):
                if prob.a_mask[i, k] == 1 and prob.b_mask[k, j] == 1:
                    hit = True
                    bt += 1
                    bf += 2 * int(prob.row_sizes[i]) * int(prob.col_sizes[j]) * int(prob.inner_sizes[k])
            want = hit or (cm is not None and cm[i, j] == 1)
            assert bool(cs[i, j]) == want
    assert nt == bt
    assert fl == float(bf)
    ptr, kl = oracle.klists(prob)
    assert ptr[-1] == nt
    for i in range(prob.M):
        for j in range(prob.N):
            t = i * prob.N + j
            ks = kl[ptr[t]:ptr[t + 1]].tolist()
            assert ks == [k for k in range(prob.K) if prob.a_mask[i, k] and prob.b_mask[k, j]]
            assert ks == sorted(ks)


def test_structure_matches_matrix_product_of_masks():
    prob = G.make_problem("uniform_bernoulli", 5, 16 * 8, block=8)
    cs, _, _ = oracle.structure(prob)
    # boolean product through integer matrix multiplication (independent route)
    prod = (prob.a_mask.astype(np.int64) @ prob.b_mask.astype(np.int64)) > 0
    assert np.array_equal(cs.astype(bool), prod)


# ------------------------------------------------------------------------------------------
# numerics: dense brute force, exact rationals, integers, identity, block-diagonal
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(16))
def test_vs_dense_matmul(seed):
    """Library cross-check: numpy float64 matmul on the densified operands."""
    prob = G.random_small(seed, max_blocks=6, max_size=24)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(seed))
    C = C0.copy()
    oracle.bsmm(prob, cs, C, off)
    ref = dense_reference(prob, cs, C0, off)
    got = struct_elements(prob, cs, off, C)
    want = struct_elements(prob, cs, off, ref)
    assert rel_fro(got, want) <= 1e-14


@pytest.mark.parametrize("seed", range(6))
def test_vs_exact_rationals(seed):
    """Brute force in exact rational arithmetic: each oracle element is within the
    classical dot-product error bound of the exact value."""
    prob = G.random_small(seed + 50, max_blocks=4, max_size=7)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(seed))
    C = C0.copy()
    oracle.bsmm(prob, cs, C, off)
    u = 2.0 ** -53
    for i in range(prob.M):
        for j in range(prob.N):
            if not cs[i, j]:
                continue
            r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
            o = off[i, j]
            cin = C0[o:o + r * c].reshape(r, c)
            ex = exact_tile_fraction(prob, i, j, cin)
            got = C[o:o + r * c].reshape(r, c)
            depth = sum(int(prob.inner_sizes[k]) for k in range(prob.K)
                        if prob.a_mask[i, k] and prob.b_mask[k, j])
            for ii in range(r):
                for jj in range(c):
                    # |fl(sum) - sum| <= gamma_n * sum |a||b| (+ epilogue roundings)
                    absum = 0.0
                    for k in range(prob.K):
                        if prob.a_mask[i, k] and prob.b_mask[k, j]:
                            At = G.tile_view(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes, i, k)
                            Bt = G.tile_view(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes, k, j)
                            absum += float(np.abs(At[ii, :]) @ np.abs(Bt[:, jj]))
                    n = depth + 2
                    bound = (n * u / (1 - n * u)) * (abs(prob.alpha) * absum + abs(prob.beta) * abs(cin[ii, jj])) \
                        + 4 * u * abs(float(ex[ii][jj])) + 1e-300
                    assert abs(got[ii, jj] - float(ex[ii][jj])) <= bound


@pytest.mark.parametrize("seed", range(6))
def test_integer_inputs_exact(seed):
    """Entries in [-8, 8], alpha and beta powers of two: every partial sum is an
    integer far below 2^53, so the result equals the exact integer product."""
    prob = G.random_small(seed + 200, max_blocks=6, max_size=30, values="integers")
    prob.alpha = [1.0, 2.0, -0.5, 4.0][seed % 4]
    prob.beta = [0.0, 1.0, -2.0, 0.25][seed % 4]
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(seed))
    C0 = np.rint(C0 * 8)
    C = C0.copy()
    oracle.bsmm(prob, cs, C, off)
    Ad = G.densify(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes).astype(np.int64)
    Bd = G.densify(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes).astype(np.int64)
    P = Ad @ Bd
    ro = np.concatenate([[0], np.cumsum(prob.row_sizes.astype(np.int64))])
    co = np.concatenate([[0], np.cumsum(prob.col_sizes.astype(np.int64))])
    for i in range(prob.M):
        for j in range(prob.N):
            if not cs[i, j]:
                continue
            r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
            o = off[i, j]
            want = prob.alpha * P[ro[i]:ro[i + 1], co[j]:co[j + 1]].astype(np.float64)
            if prob.beta != 0:
                want = want + prob.beta * C0[o:o + r * c].reshape(r, c)
            assert np.array_equal(C[o:o + r * c].reshape(r, c), want)


def test_block_identity():
    """A = block-diagonal identity with a = I and r = q: C = alpha*B + beta*C exactly."""
    rng = np.random.default_rng(11)
    q = np.array([3, 0, 5, 1, 4], np.int32)
    c = np.array([2, 6, 1], np.int32)
    K = len(q)
    am = np.eye(K, dtype=np.uint8)
    bm = (rng.random((K, len(c))) < 0.7).astype(np.uint8)
    a_off, a_tot = G.layout_arena(am, q, q)
    b_off, b_tot = G.layout_arena(bm, q, c)
    A = np.zeros(a_tot)
    for k in range(K):
        o = a_off[k, k]
        A[o:o + q[k] * q[k]] = np.eye(q[k]).reshape(-1)
    B = rng.uniform(-1, 1, b_tot)
    for alpha, beta in [(1.0, 0.0), (-0.5, 0.0), (2.0, 1.0), (1.0, -3.0)]:
        prob = G.Problem("ident", q, c, q, am, bm, a_off, b_off, A, B, alpha, beta)
        cs, _, _ = oracle.structure(prob)
        assert np.array_equal(cs, bm)
        off, C0 = c_arena(prob, cs, rng=rng)
        C = C0.copy()
        oracle.bsmm(prob, cs, C, off)
        for k in range(K):
            for j in range(len(c)):
                if not bm[k, j]:
                    continue
                n = int(q[k]) * int(c[j])
                want = alpha * B[b_off[k, j]:b_off[k, j] + n]
                if beta != 0:
                    want = want + beta * C0[off[k, j]:off[k, j] + n]
                assert np.array_equal(C[off[k, j]:off[k, j] + n], want)


def test_block_diagonal():
    """Diagonal masks: C_ii = A_ii B_ii, every other C tile absent."""
    rng = np.random.default_rng(5)
    r = np.array([4, 7, 3, 5], np.int32)
    q = np.array([6, 2, 8, 3], np.int32)
    c = np.array([5, 5, 2, 9], np.int32)
    n = len(r)
    am = np.eye(n, dtype=np.uint8)
    bm = np.eye(n, dtype=np.uint8)
    a_off, a_tot = G.layout_arena(am, r, q)
    b_off, b_tot = G.layout_arena(bm, q, c)
    prob = G.Problem("bdiag", r, c, q, am, bm, a_off, b_off, rng.uniform(-1, 1, a_tot),
                     rng.uniform(-1, 1, b_tot), 1.0, 0.0)
    cs, nt, fl = oracle.structure(prob)
    assert np.array_equal(cs, np.eye(n, dtype=np.uint8))
    assert nt == n
    assert fl == float(sum(2 * r[i] * c[i] * q[i] for i in range(n)))
    off, C = c_arena(prob, cs, fill=np.nan)
    oracle.bsmm(prob, cs, C, off)
    for i in range(n):
        At = G.tile_view(prob.A, a_off, r, q, i, i)
        Bt = G.tile_view(prob.B, b_off, q, c, i, i)
        got = C[off[i, i]:off[i, i] + r[i] * c[i]].reshape(r[i], c[i])
        assert rel_fro(got, At @ Bt) <= 1e-15


def test_empty_masks_give_beta_c():
    """No triples at all: the C tiles kept by the C mask become beta*C; with beta = 0
    a NaN already in C is never read."""
    rng = np.random.default_rng(2)
    r = np.array([3, 4], np.int32)
    q = np.array([2, 5], np.int32)
    c = np.array([3, 1], np.int32)
    am = np.zeros((2, 2), np.uint8)
    bm = np.ones((2, 2), np.uint8)
    a_off, _ = G.layout_arena(am, r, q)
    b_off, b_tot = G.layout_arena(bm, q, c)
    cm = np.array([[1, 0], [1, 1]], np.uint8)
    for beta in (0.0, -1.5):
        prob = G.Problem("empty", r, c, q, am, bm, a_off, b_off, np.zeros(0), rng.uniform(-1, 1, b_tot), 2.0, beta)
        cs, nt, fl = oracle.structure(prob, cm)
        assert nt == 0 and fl == 0.0
        assert np.array_equal(cs, cm)
        off, C0 = c_arena(prob, cs, rng=rng)
        if beta == 0.0:
            C0[:] = np.nan
        C = C0.copy()
        oracle.bsmm(prob, cs, C, off)
        got = struct_elements(prob, cs, off, C)
        if beta == 0.0:
            assert np.all(got == 0.0)
        else:
            assert np.array_equal(got, beta * struct_elements(prob, cs, off, C0))


def test_beta_zero_ignores_nan():
    prob = G.random_small(4, max_blocks=5, max_size=12)
    prob.beta = 0.0
    cs, _, _ = oracle.structure(prob)
    off, C = c_arena(prob, cs, fill=np.nan)
    oracle.bsmm(prob, cs, C, off)
    assert np.all(np.isfinite(struct_elements(prob, cs, off, C)))


def test_single_tile_matches_full():
    prob = G.random_small(9, max_blocks=5, max_size=20)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(1))
    C = C0.copy()
    oracle.bsmm(prob, cs, C, off, nthreads=2)
    for i in range(prob.M):
        for j in range(prob.N):
            if cs[i, j]:
                r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
                o = off[i, j]
                t = oracle.bsmm_tile(prob, i, j, C0[o:o + r * c].reshape(r, c))
                assert np.array_equal(t, C[o:o + r * c].reshape(r, c))


def test_thread_count_does_not_change_bits():
    prob = G.make_problem("nonuniform_dense", 3, 600, lo=16, hi=70)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(0))
    outs = []
    for nt in (1, 3, 8):
        C = C0.copy()
        oracle.bsmm(prob, cs, C, off, nthreads=nt)
        outs.append(C)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_fma_rounding_statement():
    """The oracle's stated rounding: one fused multiply-add per scalar update in
    ascending k. A two-term dot product whose fused and unfused results differ."""
    # term 1: (-1) * (1 + 2^-29) = -(1 + 2^-29), exact either way
    # term 2: (1 + 2^-30)^2 = 1 + 2^-29 + 2^-60 exactly; fused into the accumulator it
    # leaves 2^-60, while rounding the product first (to 1 + 2^-29) would leave 0
    a = 1.0 + 2.0 ** -30
    r = np.array([1], np.int32)
    q = np.array([2], np.int32)
    c = np.array([1], np.int32)
    am = np.ones((1, 1), np.uint8)
    bm = np.ones((1, 1), np.uint8)
    a_off, a_tot = G.layout_arena(am, r, q)
    b_off, b_tot = G.layout_arena(bm, q, c)
    A = np.array([-1.0, a] + [0.0] * (a_tot - 2))
    B = np.array([1.0 + 2.0 ** -29, a] + [0.0] * (b_tot - 2))
    prob = G.Problem("fma", r, c, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)
    cs, _, _ = oracle.structure(prob)
    off, C = c_arena(prob, cs, fill=0.0)
    oracle.bsmm(prob, cs, C, off)
    assert C[0] == math.ldexp(1.0, -60)
