"""Shared test helpers: golden-file parsing, C arenas, comparisons, exact references."""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np

import bsmm_gen as G

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse_matrix(text: str) -> np.ndarray:
    rows = [r.split() for r in text.split("/")]
    return np.array([[float(x) for x in r] for r in rows], np.float64)


def read_golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(":", 1)
            out[key.strip()] = val.strip()
    return out


def golden_problem(g: dict, alpha: float, beta: float) -> G.Problem:
    r = np.array([int(x) for x in g["rows"].split()], np.int32)
    q = np.array([int(x) for x in g["inner"].split()], np.int32)
    c = np.array([int(x) for x in g["cols"].split()], np.int32)
    am = parse_matrix(g["a_mask"]).astype(np.uint8)
    bm = parse_matrix(g["b_mask"]).astype(np.uint8)
    a_off, a_tot = G.layout_arena(am, r, q)
    b_off, b_tot = G.layout_arena(bm, q, c)
    A = np.zeros(a_tot)
    B = np.zeros(b_tot)
    for key, val in g.items():
        if key.startswith("A ") or key.startswith("B "):
            which, ij = key.split()
            i, j = int(ij[0]), int(ij[1])
            m = parse_matrix(val)
            if which == "A":
                o = a_off[i, j]
                A[o:o + m.size] = m.reshape(-1)
            else:
                o = b_off[i, j]
                B[o:o + m.size] = m.reshape(-1)
    return G.Problem("golden", r, c, q, am, bm, a_off, b_off, A, B, alpha, beta)


def c_arena(prob, c_struct, fill=None, rng=None):
    """C arena over the given C tile set; filled with U[-1,1] (rng), a constant, or NaN."""
    off, tot = G.layout_arena(c_struct, prob.row_sizes, prob.col_sizes)
    if fill is None:
        C = (rng or np.random.default_rng(7)).uniform(-1, 1, tot)
    else:
        C = np.full(tot, fill, np.float64)
    return off, C


def dense_reference(prob, c_struct, C0, c_off) -> np.ndarray:
    """Library cross-check: alpha*(A_dense @ B_dense) + beta*C0 on the tiles of c_struct,
    with numpy's float64 matmul on the densified operands."""
    Ad = G.densify(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes)
    Bd = G.densify(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes)
    P = Ad @ Bd
    out = C0.copy()
    ro = np.concatenate([[0], np.cumsum(prob.row_sizes.astype(np.int64))])
    co = np.concatenate([[0], np.cumsum(prob.col_sizes.astype(np.int64))])
    for i in range(prob.M):
        for j in range(prob.N):
            if not c_struct[i, j]:
                continue
            o = c_off[i, j]
            r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
            blk = P[ro[i]:ro[i + 1], co[j]:co[j + 1]]
            t = out[o:o + r * c].reshape(r, c)
            if prob.beta != 0:
                t[...] = prob.alpha * blk + prob.beta * t
            else:
                t[...] = prob.alpha * blk
    return out


def exact_tile_fraction(prob, i, j, cin=None):
    """Exact rational value of C tile (i,j): alpha * sum_k A_ik B_kj + beta * cin,
    by brute force over the nonzero triples with Python Fractions."""
    r, c = int(prob.row_sizes[i]), int(prob.col_sizes[j])
    acc = [[Fraction(0)] * c for _ in range(r)]
    for k in range(prob.K):
        if not (prob.a_mask[i, k] and prob.b_mask[k, j]):
            continue
        qk = int(prob.inner_sizes[k])
        At = G.tile_view(prob.A, prob.a_off, prob.row_sizes, prob.inner_sizes, i, k)
        Bt = G.tile_view(prob.B, prob.b_off, prob.inner_sizes, prob.col_sizes, k, j)
        for ii in range(r):
            for jj in range(c):
                s = Fraction(0)
                for kk in range(qk):
                    s += Fraction(float(At[ii, kk])) * Fraction(float(Bt[kk, jj]))
                acc[ii][jj] += s
    al, be = Fraction(prob.alpha), Fraction(prob.beta)
    out = [[al * acc[ii][jj] + (be * Fraction(float(cin[ii, jj])) if prob.beta != 0 else 0)
            for jj in range(c)] for ii in range(r)]
    return out


def rel_fro(x, ref) -> float:
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    den = float(np.linalg.norm(ref))
    num = float(np.linalg.norm(x - ref))
    return num / den if den > 0 else num


def struct_elements(prob, c_struct, c_off, arena):
    """Concatenate the elements of the tiles in c_struct (row-major tile order)."""
    parts = []
    for i in range(prob.M):
        for j in range(prob.N):
            if c_struct[i, j]:
                o = c_off[i, j]
                n = int(prob.row_sizes[i]) * int(prob.col_sizes[j])
                parts.append(arena[o:o + n])
    return np.concatenate(parts) if parts else np.zeros(0)
