"""Pins of the split oracle's row/column scaling (one exponent per row of A and per
column of B; an all-zero row takes no part in the row maxima)."""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
from helpers import c_arena, rel_fro, struct_elements


def test_slice_rows_reconstructs_each_row():
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, (9, 13)) * np.ldexp(1.0, rng.integers(-60, 60, 9))[:, None]
    x[4] = 0.0
    e, nz, sl, rho = OS.slice_rows(x, 6)
    assert not nz[4] and e[4] == 0 and all(np.all(t[4] == 0) for t in sl)
    for ii in range(9):
        if not nz[ii]:
            continue
        mu = np.max(np.abs(x[ii]))
        assert 2.0 ** (e[ii] - 1) <= mu < 2.0 ** e[ii]
        assert np.max(np.abs(sl[0][ii])) <= 2 ** 7 and all(np.max(np.abs(t[ii])) <= 2 ** 6 for t in sl[1:])
        back = sum(np.ldexp(sl[t][ii], e[ii] - 7 * (t + 1)) for t in range(6)) + np.ldexp(rho[ii], e[ii])
        assert np.array_equal(back, x[ii])
        assert np.max(np.abs(rho[ii])) <= 2.0 ** (-7 * 6 - 1)


def _fix_row_and_col_exponents(p):
    """Give every row of every A tile and every column of every B tile an element of
    magnitude 0.75, so that each row's (column's) exponent equals its tile's."""
    A, B = p.A.copy(), p.B.copy()
    for i in range(p.M):
        for k in range(p.K):
            if p.a_mask[i, k] and p.row_sizes[i] and p.inner_sizes[k]:
                o = p.a_off[i, k]
                t = A[o:o + p.row_sizes[i] * p.inner_sizes[k]].reshape(p.row_sizes[i], p.inner_sizes[k])
                t[:, 0] = 0.75
    for k in range(p.K):
        for j in range(p.N):
            if p.b_mask[k, j] and p.col_sizes[j] and p.inner_sizes[k]:
                o = p.b_off[k, j]
                t = B[o:o + p.inner_sizes[k] * p.col_sizes[j]].reshape(p.inner_sizes[k], p.col_sizes[j])
                t[0, :] = -0.75
    p.A, p.B = A, B
    return p


@pytest.mark.parametrize("s", [3, 6])
def test_rows_reduce_to_tile_scaling(s):
    for seed in range(3):
        p = _fix_row_and_col_exponents(G.random_small(80 + seed, max_blocks=5, max_size=30))
        p.alpha, p.beta = 1.25, 0.5
        cs, _, _ = oracle.structure(p)
        off, C0 = c_arena(p, cs, rng=np.random.default_rng(1))
        a, b = C0.copy(), C0.copy()
        OS.bsmm_split(p, cs, a, off, s)
        OS.bsmm_split(p, cs, b, off, s, scaling="rows")
        assert np.array_equal(a, b)


def _scaled_integers(seed, zero_segments=False):
    """Small integers with every row of A and every column of B scaled by its own power
    of two, up to 40 binades apart: each C element is 2^(a_row + b_col) times an exact
    integer sum, and every row (column) fits one 7-bit slice of its own exponent."""
    p = G.make_problem("nonuniform_dense", seed, 180, lo=20, hi=60, values="integers")
    rng = np.random.default_rng(seed)
    # rows 2^-70 .. 2^-110: far below an all-zero row segment's exponent 0, so a rule that
    # let such a segment set the row's scale would lose the row's real terms
    ra = np.ldexp(1.0, -70 - 10 * rng.integers(0, 5, int(p.row_sizes.sum())))
    cb = np.ldexp(1.0, -10 * rng.integers(0, 5, int(p.col_sizes.sum())))
    ro = np.concatenate([[0], np.cumsum(p.row_sizes)])
    co = np.concatenate([[0], np.cumsum(p.col_sizes)])
    A, B = p.A.copy(), p.B.copy()
    for i in range(p.M):
        for k in range(p.K):
            o = p.a_off[i, k]
            t = A[o:o + p.row_sizes[i] * p.inner_sizes[k]].reshape(p.row_sizes[i], p.inner_sizes[k])
            t *= ra[ro[i]:ro[i + 1], None]
            if zero_segments and (i + k) % 3 == 0:
                t[1] = 0.0  # a row segment that is all zero in this k block only
    for k in range(p.K):
        for j in range(p.N):
            o = p.b_off[k, j]
            t = B[o:o + p.inner_sizes[k] * p.col_sizes[j]].reshape(p.inner_sizes[k], p.col_sizes[j])
            t *= cb[None, co[j]:co[j + 1]]
    p.A, p.B = A, B
    return p


@pytest.mark.parametrize("zero_segments", [False, True])
def test_rows_exact_on_scaled_integers(zero_segments):
    p = _scaled_integers(3, zero_segments)
    cs, _, _ = oracle.structure(p)
    off, C0 = c_arena(p, cs, fill=0.0)
    want, rows, tile = C0.copy(), C0.copy(), C0.copy()
    oracle.bsmm(p, cs, want, off)
    OS.bsmm_split(p, cs, rows, off, 6, scaling="rows")
    OS.bsmm_split(p, cs, tile, off, 6)
    assert np.array_equal(rows, want)
    assert not np.array_equal(tile, want)  # one exponent per tile cannot hold 40 binades in 42 bits


def test_rows_keep_small_rows_accurate():
    """Graded rows (2^(-3 m) for row m mod 17): with one exponent per row every row of C keeps
    its own relative accuracy; with one per tile the small rows lose theirs."""
    p = G.make_problem("nonuniform_dense", 4, 240, lo=30, hi=90)
    ro = np.concatenate([[0], np.cumsum(p.row_sizes)])
    A = p.A.copy()
    for i in range(p.M):
        for k in range(p.K):
            o = p.a_off[i, k]
            t = A[o:o + p.row_sizes[i] * p.inner_sizes[k]].reshape(p.row_sizes[i], p.inner_sizes[k])
            t *= np.ldexp(1.0, -3 * (np.arange(ro[i], ro[i + 1]) % 17))[:, None]
    p.A = A
    cs, _, _ = oracle.structure(p)
    off, C0 = c_arena(p, cs, fill=0.0)
    ref, rows, tile = C0.copy(), C0.copy(), C0.copy()
    oracle.bsmm(p, cs, ref, off)
    OS.bsmm_split(p, cs, rows, off, 6, scaling="rows")
    OS.bsmm_split(p, cs, tile, off, 6)

    def worst_row_err(x):
        worst = 0.0
        for i in range(p.M):
            for j in range(p.N):
                n = int(p.row_sizes[i]) * int(p.col_sizes[j])
                g = x[off[i, j]:off[i, j] + n].reshape(p.row_sizes[i], p.col_sizes[j])
                w = ref[off[i, j]:off[i, j] + n].reshape(p.row_sizes[i], p.col_sizes[j])
                num = np.linalg.norm(g - w, axis=1)
                den = np.linalg.norm(w, axis=1)
                worst = max(worst, float(np.max(num / np.maximum(den, 1e-300))))
        return worst
    assert worst_row_err(rows) <= 1e-11
    assert worst_row_err(tile) > 1e-9
