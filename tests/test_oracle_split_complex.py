"""Pins of the split oracle with complex elements (no GPU): one exponent per tile over
both parts, the exact real and imaginary sums (T_re = T(Ar,Br) - T(Ai,Bi), T_im =
T(Ar,Bi) + T(Ai,Br)) each rounded once, real alpha and beta applied to each part.

References fixed outside the oracle: numpy's complex matmul on small integers (exact),
exact Fraction sums of the complex products rounded once per part (Python's float() of a
Fraction is correctly rounded), and the real oracle on inputs with zero imaginary parts.
A swapped part, a sign slip in Ai*Bi, or a per-part exponent would fail one of them.
"""
import dataclasses
from fractions import Fraction

import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
from helpers import c_arena


def _c_arena(prob, cs, seed):
    off, C64 = c_arena(prob, cs, rng=np.random.default_rng(seed))
    rng = np.random.default_rng(seed + 1)
    return off, (C64 + 1j * rng.uniform(-1, 1, C64.size)).astype(np.complex128)


def _dense(prob, arena, off, rows, cols):
    ro = np.concatenate([[0], np.cumsum(np.asarray(rows, np.int64))])
    co = np.concatenate([[0], np.cumsum(np.asarray(cols, np.int64))])
    out = np.zeros((ro[-1], co[-1]), np.complex128)
    for u in range(len(rows)):
        for v in range(len(cols)):
            if off[u, v] >= 0:
                n = int(rows[u]) * int(cols[v])
                out[ro[u]:ro[u + 1], co[v]:co[v + 1]] = arena[off[u, v]:off[u, v] + n].reshape(rows[u], cols[v])
    return out


@pytest.mark.parametrize("s", [1, 3, 6])
@pytest.mark.parametrize("seed", range(4))
def test_integer_inputs_equal_complex_matmul(seed, s):
    prob = G.as_complex(G.random_small(seed, max_blocks=5, max_size=12, values="integers"), seed)
    prob.alpha, prob.beta = 2.0, -0.5
    cs, _, _ = oracle.structure(prob)
    off, C0 = _c_arena(prob, cs, seed)
    C0 = np.round(C0 * 4) / 4  # exact in any sum below
    C = C0.copy()
    OS.bsmm_split(prob, cs, C, off, s)
    Ad = _dense(prob, prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes)
    Bd = _dense(prob, prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes)
    P = Ad @ Bd
    ro = np.concatenate([[0], np.cumsum(prob.row_sizes.astype(np.int64))])
    co = np.concatenate([[0], np.cumsum(prob.col_sizes.astype(np.int64))])
    for i in range(prob.M):
        for j in range(prob.N):
            if cs[i, j]:
                r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
                o = off[i, j]
                want = prob.alpha * P[ro[i]:ro[i + 1], co[j]:co[j + 1]] + prob.beta * C0[o:o + r * c].reshape(r, c)
                assert np.array_equal(C[o:o + r * c].reshape(r, c), want)


@pytest.mark.parametrize("seed", range(5))
def test_correctly_rounded_parts(seed):
    """Values of 20 bits in [0.5, 1): three 7-bit slices hold each exactly, and with 6
    slices every product of those slices is kept (3 + 3 <= s + 1), so each part is the
    exact sum rounded once."""
    prob = G.random_small(seed + 30, max_blocks=4, max_size=8, allow_zero=False)
    rng = np.random.default_rng(seed)
    val = lambda n: rng.choice([-1, 1], n) * rng.integers(1 << 19, 1 << 20, n) * 2.0 ** -20
    prob = dataclasses.replace(prob, A=val(prob.A.size) + 1j * val(prob.A.size),
                               B=val(prob.B.size) + 1j * val(prob.B.size), alpha=1.0, beta=0.0)
    cs, _, _ = oracle.structure(prob)
    off, C0 = _c_arena(prob, cs, seed)
    C = C0.copy()
    OS.bsmm_split(prob, cs, C, off, 6)
    for i in range(prob.M):
        for j in range(prob.N):
            if not cs[i, j]:
                continue
            r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
            got = C[off[i, j]:off[i, j] + r * c].reshape(r, c)
            re = [[Fraction(0)] * c for _ in range(r)]
            im = [[Fraction(0)] * c for _ in range(r)]
            for k in range(prob.K):
                if not (prob.a_mask[i, k] and prob.b_mask[k, j]):
                    continue
                At = G.tile_view(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes, i, k)
                Bt = G.tile_view(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes, k, j)
                for ii in range(r):
                    for jj in range(c):
                        for kk in range(int(prob.inner_sizes[k])):
                            ar, ai = Fraction(At[ii, kk].real), Fraction(At[ii, kk].imag)
                            br, bi = Fraction(Bt[kk, jj].real), Fraction(Bt[kk, jj].imag)
                            re[ii][jj] += ar * br - ai * bi
                            im[ii][jj] += ar * bi + ai * br
            for ii in range(r):
                for jj in range(c):
                    assert got[ii, jj].real == float(re[ii][jj]) and got[ii, jj].imag == float(im[ii][jj])


@pytest.mark.parametrize("seed", range(3))
def test_zero_imaginary_parts_equal_the_real_oracle(seed):
    real = G.random_small(seed + 50, max_blocks=5, max_size=20)
    prob = dataclasses.replace(real, A=real.A.astype(np.complex128), B=real.B.astype(np.complex128))
    cs, _, _ = oracle.structure(real)
    off, C0 = _c_arena(real, cs, seed)
    C = C0.copy()
    OS.bsmm_split(prob, cs, C, off, 6)
    Cr = C0.real.copy()
    OS.bsmm_split(real, cs, Cr, off, 6)
    assert np.array_equal(C.real, Cr)
    want_im = C0.imag * real.beta if real.beta != 0.0 else np.zeros_like(C0.imag)
    mask = np.zeros(C.size, bool)
    for i in range(real.M):
        for j in range(real.N):
            if cs[i, j]:
                n = int(real.row_sizes[i]) * int(real.col_sizes[j])
                mask[off[i, j]:off[i, j] + n] = True
    assert np.array_equal(C.imag[mask], (real.alpha * 0.0 + want_im)[mask])


def test_exponent_is_shared_by_both_parts():
    """A tile whose imaginary part is 2^30 times its real part: the real part is sliced
    against the shared exponent, so with 3 slices it is lost (below 2^-21 of the tile's
    scale), which a per-part exponent would keep."""
    one = np.ones(1, np.int32)
    q = np.ones(1, np.int32)
    am, bm = np.ones((1, 1), np.uint8), np.ones((1, 1), np.uint8)
    a_off, at = G.layout_arena(am, one, q)
    b_off, bt = G.layout_arena(bm, q, one)
    A = np.zeros(at, np.complex128)
    B = np.zeros(bt, np.complex128)
    A[0] = 1.0 + 1j * 2.0 ** 30
    B[0] = 1.0
    prob = G.Problem("shared_e", one, one, q, am, bm, a_off, b_off, A, B, 1.0, 0.0)
    cs = np.ones((1, 1), np.uint8)
    C = np.zeros(2, np.complex128)
    OS.bsmm_split(prob, cs, C, np.zeros((1, 1), np.int64), 3)
    assert C[0] == 1j * 2.0 ** 30
    OS.bsmm_split(prob, cs, C, np.zeros((1, 1), np.int64), 6)
    assert C[0] == 1.0 + 1j * 2.0 ** 30


@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("seed", range(3))
def test_transposed_storage(seed, ta, tb):
    """A and/or B supplied as the transposed block matrix (tile (k,i) is q_k x r_i, complex
    elements): the same bits as untransposed storage, and on integer inputs the exact
    product of numpy's complex matmul of the untransposed operands."""
    for values in ("uniform", "integers"):
        base = G.as_complex(G.random_small(seed + 40, max_blocks=5, max_size=12, values=values), seed)
        base.alpha, base.beta = 1.0, 0.0
        tr = G.transposed_storage(base, bool(ta), bool(tb))
        assert tr.A.dtype == np.complex128 and tr.B.dtype == np.complex128
        cs, _, _ = oracle.structure(base)
        off, C0 = _c_arena(base, cs, seed)
        C1, C2 = C0.copy(), C0.copy()
        OS.bsmm_split(base, cs, C1, off, 6)
        OS.bsmm_split(tr, cs, C2, off, 6)
        assert np.array_equal(C1, C2)
        if values == "integers":
            P = _dense(base, base.A, base.a_off, base.row_sizes, base.inner_sizes) @ \
                _dense(base, base.B, base.b_off, base.inner_sizes, base.col_sizes)
            ro = np.concatenate([[0], np.cumsum(base.row_sizes.astype(np.int64))])
            co = np.concatenate([[0], np.cumsum(base.col_sizes.astype(np.int64))])
            for i in range(base.M):
                for j in range(base.N):
                    if cs[i, j]:
                        r, c = int(base.row_sizes[i]), int(base.col_sizes[j])
                        o = off[i, j]
                        assert np.array_equal(C2[o:o + r * c].reshape(r, c), P[ro[i]:ro[i + 1], co[j]:co[j + 1]])


def _row_scaled_complex(seed):
    """Complex integers with every row of A and every column of B scaled by its own power
    of two, up to 40 binades apart: each C element is 2^(a_row + b_col) times an exact
    complex integer sum, so numpy's complex product of the dense operands is exact."""
    base = G.random_small(seed + 60, max_blocks=4, max_size=10, allow_zero=False, values="integers")
    base.alpha, base.beta = 1.0, 0.0
    prob = G.as_complex(base, seed)
    rng = np.random.default_rng(seed)
    ra = np.ldexp(1.0, -10 * rng.integers(0, 5, int(prob.row_sizes.sum())))
    cb = np.ldexp(1.0, -10 * rng.integers(0, 5, int(prob.col_sizes.sum())))
    ro = np.concatenate([[0], np.cumsum(prob.row_sizes)])
    co = np.concatenate([[0], np.cumsum(prob.col_sizes)])
    A, B = prob.A.copy(), prob.B.copy()
    for i in range(prob.M):
        for k in range(prob.K):
            if prob.a_mask[i, k]:
                o = prob.a_off[i, k]
                A[o:o + prob.row_sizes[i] * prob.inner_sizes[k]].reshape(prob.row_sizes[i], prob.inner_sizes[k])[...] *= \
                    ra[ro[i]:ro[i + 1], None]
    for k in range(prob.K):
        for j in range(prob.N):
            if prob.b_mask[k, j]:
                o = prob.b_off[k, j]
                B[o:o + prob.inner_sizes[k] * prob.col_sizes[j]].reshape(prob.inner_sizes[k], prob.col_sizes[j])[...] *= \
                    cb[None, co[j]:co[j + 1]]
    return dataclasses.replace(prob, A=A, B=B)


@pytest.mark.parametrize("seed", range(4))
def test_row_scaling_exact_on_scaled_complex_integers(seed):
    prob = _row_scaled_complex(seed)
    cs, _, _ = oracle.structure(prob)
    off, C0 = _c_arena(prob, cs, seed)
    C = np.zeros_like(C0)
    OS.bsmm_split(prob, cs, C, off, 6, scaling="rows")
    P = _dense(prob, prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes) @ \
        _dense(prob, prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes)
    ro = np.concatenate([[0], np.cumsum(prob.row_sizes.astype(np.int64))])
    co = np.concatenate([[0], np.cumsum(prob.col_sizes.astype(np.int64))])
    for i in range(prob.M):
        for j in range(prob.N):
            if cs[i, j]:
                r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
                o = off[i, j]
                assert np.array_equal(C[o:o + r * c].reshape(r, c), P[ro[i]:ro[i + 1], co[j]:co[j + 1]])


@pytest.mark.parametrize("seed", range(3))
def test_row_scaling_zero_imaginary_parts_equal_the_real_oracle(seed):
    base = G.random_small(seed + 70, max_blocks=5, max_size=12)
    prob = dataclasses.replace(base, A=base.A.astype(np.complex128), B=base.B.astype(np.complex128))
    cs, _, _ = oracle.structure(base)
    off, C0 = c_arena(base, cs, rng=np.random.default_rng(seed))
    real = C0.copy()
    OS.bsmm_split(base, cs, real, off, 6, scaling="rows")
    cpx = C0.astype(np.complex128)
    OS.bsmm_split(prob, cs, cpx, off, 6, scaling="rows")
    assert np.array_equal(cpx.real, real)
    assert np.array_equal(cpx.imag, np.zeros_like(real))  # beta times a zero imaginary part
