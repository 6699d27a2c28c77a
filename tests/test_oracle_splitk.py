"""Pins of the FP64 oracle's split-k reduction (Sec. 3.2, Fig. 2: multiply tasks on
pieces of a tile's k-list, then a reduction of the partials in piece order) against
facts fixed outside it (no GPU).

A slip in the piece boundaries (ceiling instead of floor, a dropped or doubled k block),
in the reduction order or in its rounding fails the hand-worked fixture or the exact
integer case; the error bound catches a wrong sign or operand.
"""
from fractions import Fraction

import numpy as np
import pytest

import bsmm_gen as G
import oracle
from helpers import c_arena, exact_tile_fraction, read_golden


def _column_problem(a_vals):
    """One 1x1 C tile over len(a_vals) inner blocks of size 1; B = 1."""
    K = len(a_vals)
    one = np.ones(1, np.int32)
    q = np.ones(K, np.int32)
    am = np.ones((1, K), np.uint8)
    bm = np.ones((K, 1), np.uint8)
    a_off, a_tot = G.layout_arena(am, one, q)  # tiles start at even offsets (16-byte alignment)
    b_off, b_tot = G.layout_arena(bm, q, one)
    A = np.zeros(a_tot)
    B = np.zeros(b_tot)
    A[a_off[0, :]] = np.array(a_vals, np.float64)
    B[b_off[:, 0]] = 1.0
    return G.Problem("splitk_hand", one, one, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)


@pytest.mark.parametrize("case,n", [("case3", 1), ("case3", 2), ("case3", 3), ("case3", 7),
                                    ("case4", 2), ("case4", 3), ("case4", 4),
                                    ("case4r", 1), ("case4r", 2), ("case4r", 4)])
def test_hand_worked_pieces(case, n):
    g = read_golden("split_k_hand.txt")
    prob = _column_problem([float.fromhex(x) for x in g[f"{case}_A"].split()])
    want = float.fromhex(g[f"{case}_n{n}"])
    cs = np.ones((1, 1), np.uint8)
    off, C = c_arena(prob, cs, fill=0.0)
    oracle.bsmm(prob, cs, C, off, pieces=n)
    assert C[0] == want, (C[0].hex(), want.hex())
    assert oracle.bsmm_tile(prob, 0, 0, pieces=n)[0, 0] == want


@pytest.mark.parametrize("seed", range(8))
def test_integer_inputs_exact_for_any_pieces(seed):
    """Small integers: every partial sum and every reduction is exact, so the result is
    the plain one bit for bit whatever the cut."""
    prob = G.random_small(seed, max_blocks=6, max_size=12, values="integers")
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, fill=3.0)
    want = C0.copy()
    oracle.bsmm(prob, cs, want, off)
    for n in (2, 3, 5, 64):
        got = C0.copy()
        oracle.bsmm(prob, cs, got, off, pieces=n)
        assert np.array_equal(got, want), n


@pytest.mark.parametrize("seed", range(6))
def test_error_bound_vs_exact(seed):
    """|C - exact| <= gamma_m (|alpha| sum|a||b| + |beta||c|) with m = inner depth + pieces
    + 2 roundings (the pieces' fma chains, the n' - 1 reduction additions, the epilogue)."""
    prob = G.random_small(seed + 20, max_blocks=5, max_size=10, allow_zero=False)
    cs, _, _ = oracle.structure(prob)
    off, C0 = c_arena(prob, cs, rng=np.random.default_rng(seed))
    u = 2.0 ** -53
    for n in (2, 4):
        C = C0.copy()
        oracle.bsmm(prob, cs, C, off, pieces=n)
        for i in range(prob.M):
            for j in range(prob.N):
                if not cs[i, j]:
                    continue
                r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
                o = off[i, j]
                cin = C0[o:o + r * c].reshape(r, c)
                ex = exact_tile_fraction(prob, i, j, cin)
                got = C[o:o + r * c].reshape(r, c)
                depth = sum(int(prob.inner_sizes[k]) for k in range(prob.K) if prob.a_mask[i, k] and prob.b_mask[k, j])
                m = depth + n + 2
                gam = m * u / (1 - m * u)
                for ii in range(r):
                    for jj in range(c):
                        absum = Fraction(0)
                        for k in range(prob.K):
                            if not (prob.a_mask[i, k] and prob.b_mask[k, j]):
                                continue
                            At = G.tile_view(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes, i, k)
                            Bt = G.tile_view(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes, k, j)
                            absum += sum(Fraction(abs(float(At[ii, kk]))) * Fraction(abs(float(Bt[kk, jj])))
                                         for kk in range(int(prob.inner_sizes[k])))
                        bound = gam * (abs(prob.alpha) * float(absum) + abs(prob.beta) * abs(cin[ii, jj]))
                        assert abs(got[ii, jj] - float(ex[ii][jj])) <= bound + 1e-300


def test_one_piece_per_block_is_blockwise_sum():
    """n >= L: every k block is a piece of its own, so the result is the ordered sum of
    the per-block products; with a single inner element per block each product is one
    rounded multiplication (fma with a zero addend)."""
    rng = np.random.default_rng(5)
    prob = _column_problem(list(rng.uniform(-1, 1, 9)))
    b = rng.uniform(-1, 1, 9)
    prob.B[prob.b_off[:, 0]] = b
    cs = np.ones((1, 1), np.uint8)
    off, C = c_arena(prob, cs, fill=0.0)
    oracle.bsmm(prob, cs, C, off, pieces=9)
    acc = 0.0
    for a, bb in zip(prob.A[prob.a_off[0, :]], b):
        acc = acc + float(a) * float(bb)
    assert C[0] == acc


@pytest.mark.parametrize("seed", range(3))
def test_transposed_storage_gives_the_same_cut(seed):
    """Only the element addressing inside a tile changes with transposed storage, so every
    cut gives the untransposed bits."""
    base = G.random_small(seed + 40, max_blocks=5, max_size=14)
    cs, _, _ = oracle.structure(base)
    off, C0 = c_arena(base, cs, fill=0.5)
    for n in (2, 5):
        want = C0.copy()
        oracle.bsmm(base, cs, want, off, pieces=n)
        for ta, tb in ((True, False), (False, True), (True, True)):
            got = C0.copy()
            oracle.bsmm(G.transposed_storage(base, ta, tb), cs, got, off, pieces=n)
            assert np.array_equal(got, want), (n, ta, tb)
