"""Pins of the split-precision oracle (Ozaki-style slicing) against facts fixed
outside it: exact rational reconstruction, the slicing bounds, a pure-integer
brute force of the pair sums, the analytic truncation bound, integer inputs,
bfloat16/float16 representability, and the error against the FP64 oracle."""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import bsmm_gen as G
import oracle
from oracle import split as S
from helpers import c_arena, exact_tile_fraction, rel_fro, struct_elements


def _wide_tile(rng, r, c, spread):
    """Entries with random signs and magnitudes spread over ``spread`` binades."""
    mag = np.ldexp(rng.uniform(0.5, 1.0, (r, c)), rng.integers(-spread, 1, (r, c)))
    return mag * rng.choice([-1.0, 1.0], (r, c)) * 2.0 ** rng.integers(-30, 30)


def test_tile_exponent_definition():
    cases = [np.array([[1.0]]), np.array([[0.75, -0.5]]), np.array([[-2.0, 1.0]]),
             np.array([[3.0e-310]]), np.array([[1.5e300, -1.0]]), np.array([[0.0, 0.0]]),
             np.array([[2.0 ** -1074]]), np.array([[np.nextafter(1.0, 0.0)]])]
    for x in cases:
        e = S.tile_exponent(x)
        mu = float(np.max(np.abs(x)))
        if mu == 0.0:
            assert e == 0
            continue
        # smallest integer e with mu < 2^e, checked with exact rationals
        assert Fraction(mu) < Fraction(2) ** e
        assert not (Fraction(mu) < Fraction(2) ** (e - 1))


@pytest.mark.parametrize("beta", [7, 8])
@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("seed", range(4))
def test_slicing_exact_reconstruction_and_bounds(s, seed, beta):
    rng = np.random.default_rng(seed * 10 + s)
    x = _wide_tile(rng, 5, 7, spread=60)
    e, sl, rho = S.slice_tile(x, s, beta)
    assert len(sl) == s
    for t, n in enumerate(sl, start=1):
        assert np.array_equal(n, np.rint(n))                 # integers
        lim = 2 ** beta if t == 1 else 2 ** (beta - 1)
        assert np.max(np.abs(n)) <= lim
    assert np.max(np.abs(rho)) <= 2.0 ** (-beta * s - 1)
    for ii in range(x.shape[0]):
        for jj in range(x.shape[1]):
            rec = sum(Fraction(float(sl[t - 1][ii, jj])) * Fraction(2) ** (-beta * t) for t in range(1, s + 1))
            rec += Fraction(float(rho[ii, jj]))
            assert rec * Fraction(2) ** e == Fraction(float(x[ii, jj]))


@pytest.mark.parametrize("s", [6, 7, 8])
def test_slicing_narrow_range_is_error_free(s):
    """Elements within a few binades of the tile maximum: s*beta >= 53 + spread leaves
    a zero residual, so the slices alone reproduce every element."""
    rng = np.random.default_rng(s)
    x = _wide_tile(rng, 6, 6, spread=2)
    e, sl, rho = S.slice_tile(x, s)
    if s * S.BETA_BITS >= 53 + 3:
        assert np.all(rho == 0.0)
        back = sum(np.ldexp(sl[t - 1], e - S.BETA_BITS * t) for t in range(1, s + 1))
        assert np.array_equal(back, x)


@pytest.mark.parametrize("s,beta", [(6, 7), (5, 8)])
def test_slices_representable_in_bf16_and_fp16(s, beta):
    """|N_1| <= 2^beta and |N_t| <= 2^(beta-1): at most 8 significant bits, exact in bf16
    (8-bit significand) and fp16 for beta = 7 and 8 alike."""
    rng = np.random.default_rng(1)
    x = _wide_tile(rng, 32, 32, spread=40)
    x[0, 0] = 1.0 - 2.0 ** -30  # rounds up to the first slice's largest value, 2^beta
    _, sl, _ = S.slice_tile(x, s, beta)
    assert np.max(np.abs(sl[0])) == 2 ** beta
    for n in sl:
        t = torch.from_numpy(n.astype(np.float32))
        assert torch.equal(t.to(torch.bfloat16).to(torch.float32), t)
        assert torch.equal(t.to(torch.float16).to(torch.float32), t)


@pytest.mark.parametrize("s,beta", [(1, 7), (3, 7), (6, 7), (3, 8), (5, 8)])
def test_pair_integer_brute_force(s, beta):
    """T = sum_{p+q<=s+1} N^A_p N^B_q 2^(beta(s+1-p-q)) by explicit Python-integer loops."""
    rng = np.random.default_rng(s)
    a = _wide_tile(rng, 4, 5, 20)
    b = _wide_tile(rng, 5, 3, 20)
    _, na, _ = S.slice_tile(a, s, beta)
    _, nb, _ = S.slice_tile(b, s, beta)
    T = S.pair_integer(na, nb, s, beta)
    for i in range(4):
        for j in range(3):
            tot = 0
            for p in range(1, s + 1):
                for q in range(1, s + 1):
                    if p + q > s + 1:
                        continue
                    dot = 0
                    for k in range(5):
                        dot += int(na[p - 1][i, k]) * int(nb[q - 1][k, j])
                    tot += dot << (beta * (s + 1 - p - q))
            assert int(T[i, j]) == tot


def test_pair_integer_beyond_int64():
    """A 20000-deep tile pair of same-sign entries near the top of their binade: every first
    slice is 2^7, |T| passes 2^63, and T must still be the exact integer (formed here by
    int64 slice-pair products, exact at this depth, combined in Python integers)."""
    s, beta, n = 6, 7, 20000
    rng = np.random.default_rng(11)
    a = rng.uniform(0.997, 0.9999, (2, n))
    b = rng.uniform(0.997, 0.9999, (n, 2))
    ea, na, _ = S.slice_tile(a, s, beta)
    eb, nb, _ = S.slice_tile(b, s, beta)
    assert ea == eb == 0 and np.all(na[0] == 2 ** beta) and np.all(nb[0] == 2 ** beta)
    T = S.pair_integer(na, nb, s, beta)
    ia = [x.astype(np.int64) for x in na]
    ib = [x.astype(np.int64) for x in nb]
    for i in range(2):
        for j in range(2):
            tot = 0
            for p in range(1, s + 1):
                for q in range(1, s + 2 - p):
                    tot += int(ia[p - 1][i] @ ib[q - 1][:, j]) << (beta * (s + 1 - p - q))
            assert tot > 2 ** 63 and int(T[i, j]) == tot


def _span_tiles(prob, seed, binades):
    """Scale every A tile of inner block k by 2^(-binades * k / K): the k blocks of one C
    element then contribute at positions up to ``binades`` binades apart."""
    rng = np.random.default_rng(seed)
    for i in range(prob.M):
        for k in range(prob.K):
            if prob.a_mask[i, k]:
                o = prob.a_off[i, k]
                n = int(prob.row_sizes[i]) * int(prob.inner_sizes[k])
                prob.A[o:o + n] *= 2.0 ** (-(binades * k) // max(prob.K, 1) - int(rng.integers(0, 3)))
    return prob


@pytest.mark.parametrize("span", [0, 120])
@pytest.mark.parametrize("s,beta", [(2, 7), (3, 7), (6, 7), (3, 8), (5, 8)])
@pytest.mark.parametrize("seed", range(3))
def test_split_result_is_exact_sum_rounded_once(s, beta, seed, span):
    """Independent route: the exact rational sum over k blocks, kept slice pairs and
    inner indices of N^A_p N^B_q 2^(eA+eB-beta(p+q)), rounded once (Fraction -> float is
    correctly rounded). The oracle's value must equal it bit for bit, also when the k
    blocks' products lie up to 120 binades apart; for 7- and 8-bit slices."""
    prob = G.random_small(seed + 500, max_blocks=4, max_size=9)
    prob.alpha, prob.beta = 1.0, 0.0
    if span:
        prob = _span_tiles(prob, seed, span)
    cs, _, _ = oracle.structure(prob)
    off, C = c_arena(prob, cs, fill=0.0)
    S.bsmm_split(prob, cs, C, off, s, beta=beta)
    for i in range(prob.M):
        for j in range(prob.N):
            if not cs[i, j]:
                continue
            r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
            exact = [[Fraction(0)] * c for _ in range(r)]
            for k in range(prob.K):
                if not (prob.a_mask[i, k] and prob.b_mask[k, j]):
                    continue
                At = G.tile_view(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes, i, k)
                Bt = G.tile_view(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes, k, j)
                eA, na, _ = S.slice_tile(At, s, beta)
                eB, nb, _ = S.slice_tile(Bt, s, beta)
                for p in range(1, s + 1):
                    for qq in range(1, s + 2 - p):
                        w = Fraction(2) ** (eA + eB - beta * (p + qq))
                        for ii in range(r):
                            for jj in range(c):
                                dot = sum(int(na[p - 1][ii, kk]) * int(nb[qq - 1][kk, jj])
                                          for kk in range(At.shape[1]))
                                exact[ii][jj] += w * dot
            got = C[off[i, j]:off[i, j] + r * c].reshape(r, c)
            for ii in range(r):
                for jj in range(c):
                    assert got[ii, jj] == float(exact[ii][jj])


@pytest.mark.parametrize("s,beta", [(2, 7), (3, 7), (4, 7), (6, 7), (3, 8), (5, 8)])
@pytest.mark.parametrize("seed", range(3))
def test_split_within_truncation_bound(s, beta, seed):
    """|C_split - C_exact| <= sum_k q_k (s+3) 2^(-beta s) 2^(eA+eB) |alpha| + rounding, where the
    first term bounds the dropped slice pairs (p+q > s+1) and the slicing residuals."""
    prob = G.random_small(seed + 300, max_blocks=4, max_size=8)
    prob.beta = 0.0
    cs, _, _ = oracle.structure(prob)
    off, C = c_arena(prob, cs, fill=0.0)
    S.bsmm_split(prob, cs, C, off, s, beta=beta)
    u = 2.0 ** -53
    for i in range(prob.M):
        for j in range(prob.N):
            if not cs[i, j]:
                continue
            ex = exact_tile_fraction(prob, i, j)
            r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
            got = C[off[i, j]:off[i, j] + r * c].reshape(r, c)
            bound = 0.0
            mag = 0.0
            nk = 0
            for k in range(prob.K):
                if prob.a_mask[i, k] and prob.b_mask[k, j]:
                    At = G.tile_view(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes, i, k)
                    Bt = G.tile_view(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes, k, j)
                    eA, eB = S.tile_exponent(At), S.tile_exponent(Bt)
                    bound += int(prob.inner_sizes[k]) * (s + 3) * 2.0 ** (-beta * s + eA + eB)
                    mag += int(prob.inner_sizes[k]) * 2.0 ** (eA + eB)
                    nk += 1
            bound = abs(prob.alpha) * (bound + (nk + 2) * u * mag) + 1e-300
            for ii in range(r):
                for jj in range(c):
                    assert abs(float(Fraction(float(got[ii, jj])) - ex[ii][jj])) <= bound


def test_dropping_a_pair_diagonal_breaks_the_bound():
    """Sanity of the bound above: keeping only p+q <= s (one diagonal short) exceeds it."""
    rng = np.random.default_rng(0)
    a = rng.uniform(-1, 1, (8, 16))
    b = rng.uniform(-1, 1, (16, 8))
    s = 4
    eA, na, _ = S.slice_tile(a, s)
    eB, nb, _ = S.slice_tile(b, s)
    beta = S.BETA_BITS
    T_short = S.pair_integer(na[:s - 1] + [np.zeros_like(na[0])], nb[:s - 1] + [np.zeros_like(nb[0])], s)
    approx = np.ldexp(T_short.astype(np.float64), eA + eB - beta * (s + 1))
    err = np.max(np.abs(approx - a @ b))
    assert err > 16 * (s + 3) * 2.0 ** (-beta * s + eA + eB)


@pytest.mark.parametrize("s", [1, 2, 6])
def test_integer_inputs_split_equals_exact(s):
    """Entries in [-8, 8]: each tile scaled by 2^-e has at most 4 significant bits, the
    first slice holds it exactly, and the split product is the exact integer product."""
    prob = G.random_small(77 + s, max_blocks=5, max_size=20, values="integers")
    prob.alpha, prob.beta = 2.0, 0.0
    cs, _, _ = oracle.structure(prob)
    off, C64 = c_arena(prob, cs, fill=0.0)
    oracle.bsmm(prob, cs, C64, off)
    Cs = np.zeros_like(C64)
    S.bsmm_split(prob, cs, Cs, off, s)
    assert np.array_equal(struct_elements(prob, cs, off, Cs), struct_elements(prob, cs, off, C64))


@pytest.mark.parametrize("s,tol", [(3, 1e-5), (4, 1e-7), (5, 1e-9), (6, 1e-11)])
def test_split_error_vs_fp64_oracle(s, tol):
    prob = G.make_problem("nonuniform_dense", 21, 300, lo=24, hi=80)
    cs, _, _ = oracle.structure(prob)
    off, C64 = c_arena(prob, cs, fill=0.0)
    oracle.bsmm(prob, cs, C64, off)
    Cs = np.zeros_like(C64)
    S.bsmm_split(prob, cs, Cs, off, s)
    err = rel_fro(struct_elements(prob, cs, off, Cs), struct_elements(prob, cs, off, C64))
    assert err <= tol


def test_split_decay_tiles_keep_relative_accuracy():
    """Banded tiles with norms over ~6 orders: per-tile scales keep the error relative."""
    prob = G.make_problem("banded_decay_wide", 4, 400, lo=16, hi=48, band=3)
    cs, _, _ = oracle.structure(prob)
    off, C64 = c_arena(prob, cs, fill=0.0)
    oracle.bsmm(prob, cs, C64, off)
    Cs = np.zeros_like(C64)
    S.bsmm_split(prob, cs, Cs, off, 6)
    assert rel_fro(struct_elements(prob, cs, off, Cs), struct_elements(prob, cs, off, C64)) <= 1e-11


def test_split_alpha_beta_epilogue():
    prob = G.random_small(5, max_blocks=4, max_size=10)
    prob.alpha, prob.beta = -0.75, 2.0
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(3))
    C1 = C0.copy()
    S.bsmm_split(prob, cs, C1, off, 6)
    prob2 = G.Problem(**{**prob.__dict__})
    prob2.alpha, prob2.beta = 1.0, 0.0
    Cp = np.zeros_like(C0)
    S.bsmm_split(prob2, cs, Cp, off, 6)
    want = -0.75 * struct_elements(prob, cs, off, Cp) + 2.0 * struct_elements(prob, cs, off, C0)
    assert np.array_equal(struct_elements(prob, cs, off, C1), want)


def test_hand_worked_slices_with_ties():
    """A hand-worked tile (tests/golden/split_slices_hand.txt): the exponent rule and the
    ties-to-even rounding of each slice, including a negative tie."""
    from helpers import read_golden
    g = read_golden("split_slices_hand.txt")
    x = np.array([float.fromhex(v) for v in g["tile"].split()])
    e, sl, rho = S.slice_tile(x.reshape(1, -1), 3)
    assert e == int(g["exponent"])
    for u in range(x.size):
        want = [int(v) for v in g[f"slices_{u}"].split()]
        assert [int(sl[t][0, u]) for t in range(3)] == want, u
    assert not rho.any()


def _one_by_one(a_vals, b_vals):
    """A 1 x 1 C tile whose k-th term is a_vals[k] * b_vals[k] (1 x 1 tiles, K = len)."""
    one = np.ones(1, np.int32)
    q = np.ones(len(a_vals), np.int32)
    am, bm = np.ones((1, len(a_vals)), np.uint8), np.ones((len(a_vals), 1), np.uint8)
    a_off, at = G.layout_arena(am, one, q)
    b_off, bt = G.layout_arena(bm, q, one)
    A, B = np.zeros(at), np.zeros(bt)
    A[a_off[0, :]] = a_vals
    B[b_off[:, 0]] = b_vals
    prob = G.Problem("terms", one, one, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)
    cs = np.ones((1, 1), np.uint8)
    off, _ = G.layout_arena(cs, one, one)
    return prob, cs, off


@pytest.mark.parametrize("s", [1, 6])
def test_far_term_decides_a_tie(s):
    """Terms 1, 2^-53 and 2^-150 (each a power of two, sliced exactly): 1 + 2^-53 is a tie
    between 1 and 1 + 2^-52, and the term 97 binades further down puts the exact sum above
    it, so the one rounding gives 1 + 2^-52. An accumulation that dropped bits far below
    the largest term (a fixed-width window, say 55 bits under it) would see the tie and
    round to 1."""
    prob, cs, off = _one_by_one([1.0, 2.0 ** -53, 2.0 ** -150], [1.0, 1.0, 1.0])
    C = np.zeros(1)
    S.bsmm_split(prob, cs, C, off, s)
    assert C[0] == 1.0 + 2.0 ** -52
    prob2, cs2, off2 = _one_by_one([1.0, 2.0 ** -53, -2.0 ** -150], [1.0, 1.0, 1.0])
    S.bsmm_split(prob2, cs2, C, off2, s)
    assert C[0] == 1.0  # just below the tie


def test_subnormal_result_rounded_once():
    """Terms 1.5 * 2^-1074 and -2^-1144 (products of powers of two and 1.5): the exact sum
    (1.5 - 2^-70) 2^-1074 lies just below the midpoint of the two smallest subnormals, so
    it rounds to 2^-1074. Rounding to a 53-bit significand first (1.5 * 2^-1074, a tie)
    and then to the subnormal grid would give 2^-1073."""
    prob, cs, off = _one_by_one([1.5 * 2.0 ** -600, -2.0 ** -572], [2.0 ** -474, 2.0 ** -572])
    for s in (1, 6):
        C = np.zeros(1)
        S.bsmm_split(prob, cs, C, off, s)
        assert C[0] == 2.0 ** -1074, (s, C[0])
        assert C[0] == float(Fraction(3, 2) * Fraction(2) ** -1074 - Fraction(2) ** -1144)
    C32 = np.zeros(1, np.float32)
    prob32, _, _ = _one_by_one([1.5 * 2.0 ** -80, -2.0 ** -95], [2.0 ** -69, 2.0 ** -94])
    S.bsmm_split(prob32, cs, C32, off, 6)
    assert C32[0] == np.float32(2.0 ** -149)  # (1.5 - 2^-40) 2^-149: below the tie


def test_overflowing_sum_rounds_to_infinity():
    """Two terms of 2^1023 each: the exact sum 2^1024 is beyond binary64, so the result is
    +inf (round to nearest); with opposite signs it is 0."""
    prob, cs, off = _one_by_one([2.0 ** 600, 2.0 ** 600], [2.0 ** 423, 2.0 ** 423])
    C = np.zeros(1)
    S.bsmm_split(prob, cs, C, off, 6)
    assert C[0] == math.inf
    prob2, _, _ = _one_by_one([2.0 ** 600, -2.0 ** 600], [2.0 ** 423, 2.0 ** 423])
    S.bsmm_split(prob2, cs, C, off, 6)
    assert C[0] == 0.0
