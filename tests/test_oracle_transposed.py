"""Pins of transposed operand storage (Sec. 2.1: transposed multiplies such as C = A B^T
are handled like the plain product). With A and/or B supplied as the transposed block
matrix, both oracles must give the untransposed oracle's bits, and the product must
match a dense product assembled independently from the transposed tiles."""
import numpy as np
import pytest

import bsmm_gen as G
import oracle
from oracle import split as OS
from helpers import c_arena, rel_fro

FLAGS = [(True, False), (False, True), (True, True)]


def _problems():
    out = []
    for seed in range(5):
        p = G.random_small(40 + seed, max_blocks=5, max_size=30)
        p.alpha, p.beta = [1.0, -0.75, 2.0, 0.5, 1.5][seed], [0.0, 1.0, -2.0, 0.0, 0.25][seed]
        out.append(p)
    return out


@pytest.mark.parametrize("ta,tb", FLAGS)
def test_generator_stores_every_tile_transposed(ta, tb):
    p = G.random_small(7, max_blocks=5, max_size=30)
    t = G.transposed_storage(p, ta, tb)
    for (m, off, arena, mt, offt, arenat, rows, cols, flag) in [
            (p.a_mask, p.a_off, p.A, t.a_mask, t.a_off, t.A, p.row_sizes, p.inner_sizes, ta),
            (p.b_mask, p.b_off, p.B, t.b_mask, t.b_off, t.B, p.inner_sizes, p.col_sizes, tb)]:
        if not flag:
            assert mt is m and offt is off
            continue
        assert np.array_equal(mt, m.T)
        for u in range(m.shape[0]):
            for v in range(m.shape[1]):
                if m[u, v]:
                    n = int(rows[u]) * int(cols[v])
                    x = arena[off[u, v]:off[u, v] + n].reshape(int(rows[u]), int(cols[v]))
                    y = arenat[offt[v, u]:offt[v, u] + n].reshape(int(cols[v]), int(rows[u]))
                    assert np.array_equal(x.T, y)


@pytest.mark.parametrize("ta,tb", FLAGS)
def test_transposed_storage_gives_the_same_bits(ta, tb):
    for p in _problems():
        t = G.transposed_storage(p, ta, tb)
        cm = (np.random.default_rng(1).random((p.M, p.N)) < 0.3).astype(np.uint8) if p.beta != 0 else None
        cs, nt, fl = oracle.structure(p, cm)
        cs2, nt2, fl2 = oracle.structure(t, cm)
        assert np.array_equal(cs, cs2) and nt == nt2 and fl == fl2
        off, C0 = c_arena(p, cs, rng=np.random.default_rng(3))
        want, got = C0.copy(), C0.copy()
        oracle.bsmm(p, cs, want, off)
        oracle.bsmm(t, cs, got, off)
        assert np.array_equal(want, got)
        for s in (3, 6):
            w2, g2 = C0.copy(), C0.copy()
            OS.bsmm_split(p, cs, w2, off, s)
            OS.bsmm_split(t, cs, g2, off, s)
            assert np.array_equal(w2, g2)
        for (i, j) in np.argwhere(cs)[:3]:
            cin = C0[off[i, j]:off[i, j] + int(p.row_sizes[i]) * int(p.col_sizes[j])].reshape(
                int(p.row_sizes[i]), int(p.col_sizes[j]))
            assert np.array_equal(oracle.bsmm_tile(p, i, j, cin), oracle.bsmm_tile(t, i, j, cin))


@pytest.mark.parametrize("ta,tb", FLAGS)
def test_transposed_storage_matches_dense_product(ta, tb):
    """Dense A and B rebuilt from the transposed arenas with numpy alone; C = A B by
    numpy matmul, within the dot-product error bound of the oracle."""
    p = G.make_problem("nonuniform_dense", 5, 160, lo=16, hi=48)
    t = G.transposed_storage(p, ta, tb)
    r, c, q = p.row_sizes, p.col_sizes, p.inner_sizes
    ro, co, qo = (np.concatenate([[0], np.cumsum(x)]) for x in (r, c, q))
    A = np.zeros((ro[-1], qo[-1]))
    B = np.zeros((qo[-1], co[-1]))
    for i in range(p.M):
        for k in range(p.K):
            n = int(r[i]) * int(q[k])
            if ta:
                A[ro[i]:ro[i + 1], qo[k]:qo[k + 1]] = t.A[t.a_off[k, i]:t.a_off[k, i] + n].reshape(q[k], r[i]).T
            else:
                A[ro[i]:ro[i + 1], qo[k]:qo[k + 1]] = t.A[t.a_off[i, k]:t.a_off[i, k] + n].reshape(r[i], q[k])
    for k in range(p.K):
        for j in range(p.N):
            n = int(q[k]) * int(c[j])
            if tb:
                B[qo[k]:qo[k + 1], co[j]:co[j + 1]] = t.B[t.b_off[j, k]:t.b_off[j, k] + n].reshape(c[j], q[k]).T
            else:
                B[qo[k]:qo[k + 1], co[j]:co[j + 1]] = t.B[t.b_off[k, j]:t.b_off[k, j] + n].reshape(q[k], c[j])
    dense = A @ B
    cs, _, _ = oracle.structure(t)
    off, C0 = c_arena(t, cs, fill=0.0)
    oracle.bsmm(t, cs, C0, off)
    got = np.concatenate([C0[off[i, j]:off[i, j] + int(r[i]) * int(c[j])] for i in range(p.M) for j in range(p.N)])
    want = np.concatenate([dense[ro[i]:ro[i + 1], co[j]:co[j + 1]].reshape(-1) for i in range(p.M) for j in range(p.N)])
    assert rel_fro(got, want) <= 1e-14
