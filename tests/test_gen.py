"""Input generators: reproducible from the seed, tilings total n within bounds, the
paper's nonuniform blocking keeps block count and mean (Sec. 4.1), masks as stated."""
import numpy as np
import pytest

import bsmm_gen as G


@pytest.mark.parametrize("n,lo,hi", [(16384, 64, 256), (32768, 32, 256), (1000, 16, 512), (77, 16, 40)])
def test_uniform_int_tiling(n, lo, hi):
    r = G.tiling_uniform_int(n, lo, hi, np.random.default_rng(1))
    assert int(r.sum()) == n
    assert np.all(r[:-1] >= lo) and np.all(r[:-1] <= hi)
    assert r[-1] >= lo or len(r) == 1
    assert r[-1] < hi + lo


def test_log_uniform_tiling():
    r = G.tiling_log_uniform(24576, 16, 512, np.random.default_rng(2))
    assert int(r.sum()) == 24576
    assert r.min() >= 16 and r.max() < 512 + 16
    # log-uniform: the median sits near the geometric mean sqrt(16*512) ~ 90
    assert 60 < np.median(r) < 130


def test_paper_tiling_keeps_count_and_mean():
    n, nb = 32768, 128
    r = G.tiling_paper(n, nb, np.random.default_rng(3))
    assert len(r) == nb and int(r.sum()) == n
    assert r.mean() == n / nb
    assert r.min() < 256 < r.max()


def test_masks():
    rng = np.random.default_rng(4)
    m = G.mask_bernoulli(200, 200, 0.5, rng)
    assert 0.45 < m.mean() < 0.55
    b = G.mask_band(20, 20, 6)
    assert b[0, 6] == 1 and b[0, 7] == 0 and b[10, 4] == 1 and b[10, 3] == 0
    c = G.mask_clusters(172, 344, 40, 0.10, rng)
    assert abs(c.mean() - 0.10) <= 0.011


def test_reproducible():
    p1 = G.make_problem("nonuniform_dense", 9, 500)
    p2 = G.make_problem("nonuniform_dense", 9, 500)
    p3 = G.make_problem("nonuniform_dense", 10, 500)
    assert np.array_equal(p1.A, p2.A) and np.array_equal(p1.row_sizes, p2.row_sizes)
    assert not np.array_equal(p1.A[:100], p3.A[:100])


def test_arena_layout():
    r = np.array([3, 0, 2], np.int32)
    c = np.array([1, 5], np.int32)
    mask = np.array([[1, 1], [1, 0], [0, 1]], np.uint8)
    off, tot = G.layout_arena(mask, r, c)
    # every stored tile starts on an even element and tiles do not overlap
    spans = []
    for i in range(3):
        for j in range(2):
            if mask[i, j]:
                assert off[i, j] % 2 == 0
                spans.append((int(off[i, j]), int(off[i, j]) + int(r[i] * c[j])))
            else:
                assert off[i, j] == -1
    spans.sort()
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert a1 <= b0
    assert tot >= spans[-1][1]


def test_batch():
    probs = G.make_batch(4, 1, n_lo=300, n_hi=900)
    assert len(probs) == 4
    for p in probs:
        assert 300 <= int(p.row_sizes.sum()) <= 900
        assert p.row_sizes.min() >= 32


def test_float32_and_complex_arenas():
    prob = G.make_problem("nonuniform_dense", 3, 300, lo=32, hi=90)
    p32 = G.as_float32(prob)
    assert p32.A.dtype == np.float32 and p32.B.dtype == np.float32
    for mask, off, src_off, src, dst, rows, cols in ((prob.a_mask, p32.a_off, prob.a_off, prob.A, p32.A,
                                                      prob.row_sizes, prob.inner_sizes),
                                                     (prob.b_mask, p32.b_off, prob.b_off, prob.B, p32.B,
                                                      prob.inner_sizes, prob.col_sizes)):
        assert (off[mask != 0] % 4 == 0).all() and (off[mask == 0] == -1).all()
        for u, v in zip(*np.nonzero(mask)):
            n = int(rows[u]) * int(cols[v])
            assert np.array_equal(dst[off[u, v]:off[u, v] + n], src[src_off[u, v]:src_off[u, v] + n].astype(np.float32))
    pc = G.as_complex(prob, 7)
    assert pc.A.dtype == np.complex128 and np.array_equal(pc.A.real, prob.A)
    assert np.array_equal(pc.a_off, prob.a_off)
    assert np.abs(pc.A.imag).max() <= 1.0 and pc.A.imag.std() > 0.5  # U[-1,1]: std 0.577
    assert np.array_equal(G.as_complex(prob, 7).B, pc.B)  # a pure function of the seed
