"""Pins of the split oracle with float32 elements (no GPU): the slicing and the exact sum
are those of float64 elements, the sum is rounded once to float32 (ties to even) and the
epilogue runs in float32.

The reference here is the plain definition: the exact sum of the products by brute force
over Fractions, rounded to binary32 by the rounding rule written out below. A slip in the
float32 rounding (double rounding through float64, a wrong significand width, truncation),
in the epilogue's precision or in the float32 arena handling fails one of these.
"""
import dataclasses
import math
from fractions import Fraction

import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
from helpers import c_arena, exact_tile_fraction


def f32_of(x: Fraction) -> np.float32:
    """x rounded to binary32, ties to even (normal and subnormal range)."""
    if x == 0:
        return np.float32(0.0)
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()  # 2^e <= a < 2^(e+2)
    if Fraction(2) ** (e + 1) <= a:
        e += 1
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)                       # subnormals share the smallest exponent
    scaled = a / Fraction(2) ** (e - 23)   # significand in units of the last place
    q = scaled.numerator // scaled.denominator
    rem = scaled - q
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and q % 2 == 1):
        q += 1
    v = math.ldexp(float(q), e - 23)
    return np.float32(v if x > 0 else -v)


def _f32_problem(seed, values="uniform", spread=4):
    prob = G.random_small(seed, max_blocks=4, max_size=9, allow_zero=False, values=values)
    if values == "uniform":  # magnitudes in [2^-spread, 2^spread]: every element sliced exactly
        rng = np.random.default_rng(seed + 1000)
        for arr in (prob.A, prob.B):
            arr[:] = np.sign(rng.uniform(-1, 1, arr.size)) * rng.uniform(0.5, 1.0, arr.size) * \
                2.0 ** rng.integers(-spread, spread + 1, arr.size)
    return G.as_float32(prob)


def _oracle_f32(prob, s, scaling="tile", fill_seed=0):
    cs, _, _ = oracle.structure(prob)
    off, C64 = c_arena(prob, cs, rng=np.random.default_rng(fill_seed))
    C0 = C64.astype(np.float32)
    C = C0.copy()
    OS.bsmm_split(prob, cs, C, off, s, scaling=scaling)
    return cs, off, C0, C


@pytest.mark.parametrize("scaling", ["tile", "rows"])
@pytest.mark.parametrize("seed", range(6))
def test_correctly_rounded_float32(seed, scaling):
    prob = _f32_problem(seed)
    assert prob.A.dtype == np.float32 and (prob.a_off[prob.a_off >= 0] % 4 == 0).all()
    cs, off, C0, C = _oracle_f32(prob, 6, scaling)
    a32, b32 = np.float32(prob.alpha), np.float32(prob.beta)
    for i in range(prob.M):
        for j in range(prob.N):
            if not cs[i, j]:
                continue
            r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
            o = off[i, j]
            cin = C0[o:o + r * c].reshape(r, c)
            ex = exact_tile_fraction(dataclasses.replace(prob, alpha=1.0, beta=0.0), i, j)
            got = C[o:o + r * c].reshape(r, c)
            for ii in range(r):
                for jj in range(c):
                    acc = f32_of(ex[ii][jj])
                    want = a32 * acc
                    if prob.beta != 0.0:
                        want = want + b32 * cin[ii, jj]
                    assert got[ii, jj] == want, (i, j, ii, jj, got[ii, jj], want)


@pytest.mark.parametrize("seed", range(4))
def test_integer_inputs_exact(seed):
    prob = _f32_problem(seed + 10, values="integers")
    for s in (1, 3, 6):
        cs, off, C0, C = _oracle_f32(prob, s)
        C64 = C0.astype(np.float64)
        oracle.bsmm(dataclasses.replace(prob, A=prob.A.astype(np.float64), B=prob.B.astype(np.float64)),
                    cs, C64, off)
        assert np.array_equal(C, C64.astype(np.float32)), s


def test_subnormal_float32_results():
    """Products of 2^-70 scaled integers land in binary32's subnormal range (below 2^-126)
    and are exact there."""
    prob = _f32_problem(3, values="integers")
    prob.A *= np.float32(2.0 ** -70)
    prob.B *= np.float32(2.0 ** -70)
    prob.alpha, prob.beta = 1.0, 0.0
    cs, off, C0, C = _oracle_f32(prob, 6)
    nz = C[C != 0]
    assert nz.size and (np.abs(nz) < np.float32(2.0 ** -126)).all()
    for i in range(prob.M):
        for j in range(prob.N):
            if cs[i, j]:
                r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
                ex = exact_tile_fraction(prob, i, j)
                got = C[off[i, j]:off[i, j] + r * c].reshape(r, c)
                for ii in range(r):
                    for jj in range(c):
                        assert got[ii, jj] == f32_of(ex[ii][jj])


def test_no_double_rounding_through_float64():
    """Inner blocks holding 1, 2^-24 and 2^-60 (each its own tile exponent): the exact sum
    1 + 2^-24 + 2^-60 lies just above a binary32 tie and rounds up to 1 + 2^-23; going
    through float64 first (1 + 2^-24) would make it a tie and round to 1."""
    one = np.ones(1, np.int32)
    q = np.ones(3, np.int32)
    am, bm = np.ones((1, 3), np.uint8), np.ones((3, 1), np.uint8)
    a_off, at = G.layout_arena(am, one, q)
    b_off, bt = G.layout_arena(bm, q, one)
    A, B = np.zeros(at), np.zeros(bt)
    A[a_off[0, :]] = [1.0, 2.0 ** -24, 2.0 ** -60]
    B[b_off[:, 0]] = 1.0
    prob = G.as_float32(G.Problem("tie", one, one, q, am, bm, a_off, b_off, A, B, 1.0, 0.0))
    cs = np.ones((1, 1), np.uint8)
    off, _ = G.layout_arena(cs, one, one)
    C = np.zeros(1, np.float32)
    OS.bsmm_split(prob, cs, C, off, 6)
    assert C[0] == np.float32(1.0 + 2.0 ** -23)
    C64 = np.zeros(1)
    OS.bsmm_split(prob, cs, C64, off, 6)
    assert C64[0] == 1.0 + 2.0 ** -24


def test_rounding_helper_ties_and_subnormals():
    """The binary32 rounding rule above, on hand-worked cases."""
    one = Fraction(1)
    ulp = Fraction(1, 2 ** 23)
    assert f32_of(one + ulp / 2) == np.float32(1.0)                        # tie, even stays
    assert f32_of(one + 3 * ulp / 2) == np.float32(1.0 + 2.0 ** -22)       # tie, odd rounds up
    assert f32_of(one + ulp / 2 + Fraction(1, 2 ** 60)) == np.float32(1.0 + 2.0 ** -23)
    assert f32_of(Fraction(3, 2 ** 150)) == np.float32(2.0 ** -148)        # 1.5 subnormal units -> 2
    assert f32_of(Fraction(5, 2 ** 150)) == np.float32(2.0 ** -148)        # 2.5 -> 2 (even)
    assert f32_of(-Fraction(7, 3)) == -np.float32(7.0 / 3.0)
