"""Seeded synthetic inputs for block-sparse C = alpha*A*B + beta*C.

This module only draws numbers and lays tiles out in memory. It holds none of
the product's arithmetic (no mask product, no flop count, no tile multiply):
both the CPU oracle and the CUDA path receive what it produces as plain arrays.

Storage format shared by every consumer:
  * a tiling is an int32 vector of block sizes (zero-size blocks allowed);
  * a tile mask is a uint8 matrix, 1 = the tile is stored (nonzero);
  * an arena is one float64 vector holding every stored tile row-major and
    contiguous (leading dimension = the tile's column-block size); the offset
    table (int64, same shape as the mask) gives each tile's first element, -1
    for an absent tile. Offsets are even, so every tile starts 16-byte aligned.

Random numbers come from numpy's PCG64 (``np.random.default_rng(seed)``), with
one child stream per role (tilings, masks, values) spawned from the seed, so a
problem is a pure function of (recipe, sizes, seed).

The workload recipes follow the paper's experiments (Sec. 4.1: square
matrices, uniform block sizes and nonuniform block sizes with the same mean)
widened to block sparsity: Bernoulli tile masks, dense masks, banded masks with
distance decay of the tile norms (the block sparsity of Sec. 1), random dense
clusters, and batches of independent products.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Problem", "tiling_uniform", "tiling_uniform_int", "tiling_log_uniform", "tiling_paper",
    "mask_bernoulli", "mask_dense", "mask_band", "mask_clusters", "layout_arena",
    "fill_uniform", "fill_band_decay", "fill_integers", "make_problem", "make_batch", "as_float32", "as_complex",
    "tile_view", "densify", "RECIPES",
]


# --------------------------------------------------------------------------------------
# tilings
# --------------------------------------------------------------------------------------

def tiling_uniform(n: int, block: int) -> np.ndarray:
    """Blocks of size ``block``; the last block holds the remainder."""
    if n <= 0:
        return np.zeros(0, np.int32)
    full, rem = divmod(n, block)
    sizes = [block] * full + ([rem] if rem else [])
    return np.asarray(sizes, np.int32)


def _close_tiling(draws: List[int], n: int, lo: int) -> np.ndarray:
    """Trim i.i.d. block draws so they total n: the last block takes the remainder,
    and a remainder shorter than ``lo`` is merged into the previous block."""
    sizes: List[int] = []
    total = 0
    for s in draws:
        if total + s >= n:
            rem = n - total
            if rem >= lo or not sizes:
                sizes.append(rem)
            else:
                sizes[-1] += rem
            total = n
            break
        sizes.append(s)
        total += s
    assert total == n, "not enough draws"
    return np.asarray(sizes, np.int32)


def tiling_uniform_int(n: int, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    """Block sizes drawn i.i.d. uniform-integer in [lo, hi] until they reach n."""
    count = n // lo + 2
    draws = rng.integers(lo, hi + 1, size=count).tolist()
    return _close_tiling(draws, n, lo)


def tiling_log_uniform(n: int, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    """Block sizes round(exp(U[ln lo, ln hi])) until they reach n."""
    count = n // lo + 2
    u = rng.uniform(math.log(lo), math.log(hi), size=count)
    draws = np.clip(np.rint(np.exp(u)), lo, hi).astype(np.int64).tolist()
    return _close_tiling(draws, n, lo)


def tiling_paper(n: int, nblocks: int, rng: np.random.Generator) -> np.ndarray:
    """The nonuniform blocking of the paper's Sec. 4.1: start from ``nblocks`` empty
    blocks and repeatedly grow a randomly chosen block by one row until the
    blocks total n. The mean block size equals that of the uniform tiling with the
    same block count. Zero-size blocks can occur."""
    picks = rng.integers(0, nblocks, size=n)
    return np.bincount(picks, minlength=nblocks).astype(np.int32)


# --------------------------------------------------------------------------------------
# masks
# --------------------------------------------------------------------------------------

def mask_dense(m: int, n: int) -> np.ndarray:
    return np.ones((m, n), np.uint8)


def mask_bernoulli(m: int, n: int, p: float, rng: np.random.Generator) -> np.ndarray:
    return (rng.random((m, n)) < p).astype(np.uint8)


def mask_band(m: int, n: int, width: int) -> np.ndarray:
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    return (np.abs(i - j) <= width).astype(np.uint8)


def mask_clusters(m: int, n: int, nclusters: int, density: float, rng: np.random.Generator,
                  tol: float = 0.01, max_tries: int = 200) -> np.ndarray:
    """Union of ``nclusters`` axis-aligned dense rectangles of tiles with random
    centres; the rectangle sides are scaled (bisection on a common factor) until the
    union covers density +- tol of the tile grid."""
    if m == 0 or n == 0:
        return np.zeros((m, n), np.uint8)
    for _ in range(max_tries):
        ci = rng.uniform(0, m, nclusters)
        cj = rng.uniform(0, n, nclusters)
        shape_i = rng.uniform(0.3, 1.0, nclusters)
        shape_j = rng.uniform(0.3, 1.0, nclusters)

        def build(scale: float) -> np.ndarray:
            mk = np.zeros((m, n), np.uint8)
            hi_ = np.maximum(1, np.rint(scale * shape_i * m / 2)).astype(int)
            hj_ = np.maximum(1, np.rint(scale * shape_j * n / 2)).astype(int)
            for c in range(nclusters):
                i0 = int(max(0, ci[c] - hi_[c])); i1 = int(min(m, ci[c] + hi_[c]))
                j0 = int(max(0, cj[c] - hj_[c])); j1 = int(min(n, cj[c] + hj_[c]))
                mk[i0:i1, j0:j1] = 1
            return mk

        lo_s, hi_s = 0.0, 1.0
        for _ in range(40):
            mid = 0.5 * (lo_s + hi_s)
            d = build(mid).mean()
            if abs(d - density) <= tol:
                return build(mid)
            if d < density:
                lo_s = mid
            else:
                hi_s = mid
    raise RuntimeError("could not place clusters at the requested density")


# --------------------------------------------------------------------------------------
# arenas
# --------------------------------------------------------------------------------------

def layout_arena(mask: np.ndarray, row_sizes: np.ndarray, col_sizes: np.ndarray, align: int = 2):
    """Offsets (int64, -1 = absent) of the stored tiles of ``mask`` in row-major tile
    order, each tile row-major with ld = its column-block size, each start rounded up
    to a multiple of ``align`` elements (2 float64 or 4 float32 elements = 16 bytes).
    Returns (offsets, total_elements)."""
    mask = np.asarray(mask, np.uint8)
    r = np.asarray(row_sizes, np.int64)
    c = np.asarray(col_sizes, np.int64)
    sizes = r[:, None] * c[None, :]
    sizes = np.where(mask != 0, (sizes + align - 1) // align * align, 0)
    flat = sizes.reshape(-1)
    starts = np.concatenate([[0], np.cumsum(flat)[:-1]]) if flat.size else np.zeros(0, np.int64)
    off = np.where(mask.reshape(-1) != 0, starts, -1).reshape(mask.shape).astype(np.int64)
    total = int(flat.sum()) if flat.size else 0
    return off, total


def tile_view(arena: np.ndarray, off: np.ndarray, row_sizes, col_sizes, i: int, j: int) -> Optional[np.ndarray]:
    o = int(off[i, j])
    if o < 0:
        return None
    r, c = int(row_sizes[i]), int(col_sizes[j])
    return arena[o:o + r * c].reshape(r, c)


def densify(arena, off, row_sizes, col_sizes) -> np.ndarray:
    """Dense matrix with the stored tiles in place and zeros elsewhere."""
    ro = np.concatenate([[0], np.cumsum(np.asarray(row_sizes, np.int64))])
    co = np.concatenate([[0], np.cumsum(np.asarray(col_sizes, np.int64))])
    out = np.zeros((int(ro[-1]), int(co[-1])), np.float64)
    for i in range(len(row_sizes)):
        for j in range(len(col_sizes)):
            t = tile_view(arena, off, row_sizes, col_sizes, i, j)
            if t is not None:
                out[ro[i]:ro[i + 1], co[j]:co[j + 1]] = t
    return out


def fill_uniform(total: int, rng: np.random.Generator, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return rng.uniform(lo, hi, size=total).astype(np.float64)


def fill_integers(total: int, rng: np.random.Generator, lo: int = -8, hi: int = 8) -> np.ndarray:
    return rng.integers(lo, hi + 1, size=total).astype(np.float64)


def fill_band_decay(mask, off, total, row_sizes, col_sizes, rng: np.random.Generator,
                    rate: float = 0.5) -> np.ndarray:
    """Tile (i, j) holds N(0,1) * exp(-rate * |i - j|) (distance decay of the tile norms)."""
    arena = np.zeros(total, np.float64)
    g = rng.standard_normal(total)
    m, n = mask.shape
    for i in range(m):
        for j in range(n):
            o = off[i, j]
            if o < 0:
                continue
            sz = int(row_sizes[i]) * int(col_sizes[j])
            arena[o:o + sz] = g[o:o + sz] * math.exp(-rate * abs(i - j))
    return arena


# --------------------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """One block-sparse product C = alpha*A*B + beta*C (inputs only)."""
    name: str
    row_sizes: np.ndarray    # M blocks
    col_sizes: np.ndarray    # N blocks
    inner_sizes: np.ndarray  # K blocks
    a_mask: np.ndarray       # M x K uint8
    b_mask: np.ndarray       # K x N uint8
    a_off: np.ndarray        # M x K int64
    b_off: np.ndarray        # K x N int64
    A: np.ndarray            # float64 arena
    B: np.ndarray            # float64 arena
    alpha: float = 1.0
    beta: float = 0.0
    c_mask: Optional[np.ndarray] = None   # extra C tiles kept (None = only the mask product)
    recipe: str = ""
    # transposed storage: the A arguments describe the K x M block matrix A' = A^T (a_mask
    # and a_off K x M, every tile A'_ki = (A_ik)^T stored q_k x r_i row-major); likewise B
    # as the N x K block matrix B' (b_mask and b_off N x K, tiles c_j x q_k)
    transa: bool = False
    transb: bool = False

    @property
    def M(self):
        return len(self.row_sizes)

    @property
    def N(self):
        return len(self.col_sizes)

    @property
    def K(self):
        return len(self.inner_sizes)


def _streams(seed: int):
    ss = np.random.SeedSequence(seed)
    kids = ss.spawn(4)
    return [np.random.default_rng(k) for k in kids]


def _assemble(name, r, c, q, am, bm, rng_v, values: str, recipe: str, alpha=1.0, beta=0.0,
              decay_rate: float = 0.5) -> Problem:
    a_off, a_tot = layout_arena(am, r, q)
    b_off, b_tot = layout_arena(bm, q, c)
    if values == "uniform":
        A = fill_uniform(a_tot, rng_v)
        B = fill_uniform(b_tot, rng_v)
    elif values == "integers":
        A = fill_integers(a_tot, rng_v)
        B = fill_integers(b_tot, rng_v)
    elif values == "band_decay":
        A = fill_band_decay(am, a_off, a_tot, r, q, rng_v, decay_rate)
        B = fill_band_decay(bm, b_off, b_tot, q, c, rng_v, decay_rate)
    else:
        raise ValueError(values)
    return Problem(name, r, c, q, am, bm, a_off, b_off, A, B, alpha, beta, None, recipe)


RECIPES = {
    # name: description (sizes are the full workload; tests pass smaller n)
    "uniform_bernoulli": "square n, uniform block 128, A/B tile masks Bernoulli(0.5), U[-1,1]",
    "nonuniform_dense": "square n, block sizes U-int[64,256] on rows, cols and inner, dense, U[-1,1]",
    "banded_decay": "square n, block sizes U-int[32,256], tile (i,j) nonzero iff |i-j|<=6, N(0,1)*exp(-|i-j|/2)",
    "banded_decay_wide": "as banded_decay with exp(-2.3|i-j|) (about 10^-|i-j|, six orders over the band)",
    "clustered": "M=N=n, K=2n, block sizes round(log-uniform[16,512]), 40 dense clusters at ~10% density, U[-1,1]",
    "paper_nonuniform": "square n, the paper's Sec. 4.1 generator with mean block 256, dense, U[-1,1]",
    "thin_dense": "M=N=n, K=k_factor*n, block sizes U-int[64,256] on rows, cols and inner, dense, U[-1,1] "
                  "(few C tiles, long inner sums)",
}


def make_problem(recipe: str, seed: int, n: int, *, values: Optional[str] = None,
                 alpha: float = 1.0, beta: float = 0.0, block: int = 128,
                 lo: Optional[int] = None, hi: Optional[int] = None, density: float = 0.5,
                 band: int = 6, nclusters: int = 40, cluster_density: float = 0.10,
                 k_factor: int = 2) -> Problem:
    rt, rm, rv, _ = _streams(seed)
    if recipe == "uniform_bernoulli":
        r = tiling_uniform(n, block)
        am = mask_bernoulli(len(r), len(r), density, rm)
        bm = mask_bernoulli(len(r), len(r), density, rm)
        return _assemble(f"{recipe}_n{n}_s{seed}", r, r, r, am, bm, rv, values or "uniform", recipe, alpha, beta)
    if recipe == "nonuniform_dense":
        r = tiling_uniform_int(n, lo or 64, hi or 256, rt)
        am = mask_dense(len(r), len(r))
        bm = mask_dense(len(r), len(r))
        return _assemble(f"{recipe}_n{n}_s{seed}", r, r, r, am, bm, rv, values or "uniform", recipe, alpha, beta)
    if recipe in ("banded_decay", "banded_decay_wide"):
        r = tiling_uniform_int(n, lo or 32, hi or 256, rt)
        am = mask_band(len(r), len(r), band)
        bm = mask_band(len(r), len(r), band)
        rate = 0.5 if recipe == "banded_decay" else 2.3
        return _assemble(f"{recipe}_n{n}_s{seed}", r, r, r, am, bm, rv, values or "band_decay", recipe,
                         alpha, beta, decay_rate=rate)
    if recipe == "clustered":
        r = tiling_log_uniform(n, lo or 16, hi or 512, rt)
        c = tiling_log_uniform(n, lo or 16, hi or 512, rt)
        q = tiling_log_uniform(k_factor * n, lo or 16, hi or 512, rt)
        am = mask_clusters(len(r), len(q), nclusters, cluster_density, rm)
        bm = mask_clusters(len(q), len(c), nclusters, cluster_density, rm)
        return _assemble(f"{recipe}_n{n}_s{seed}", r, c, q, am, bm, rv, values or "uniform", recipe, alpha, beta)
    if recipe == "thin_dense":
        r = tiling_uniform_int(n, lo or 64, hi or 256, rt)
        q = tiling_uniform_int(k_factor * n, lo or 64, hi or 256, rt)
        am = mask_dense(len(r), len(q))
        bm = mask_dense(len(q), len(r))
        return _assemble(f"{recipe}_n{n}_k{k_factor * n}_s{seed}", r, r, q, am, bm, rv, values or "uniform", recipe,
                         alpha, beta)
    if recipe == "paper_nonuniform":
        nb = max(1, n // block)
        r = tiling_paper(n, nb, rt)
        am = mask_dense(nb, nb)
        bm = mask_dense(nb, nb)
        return _assemble(f"{recipe}_n{n}_s{seed}", r, r, r, am, bm, rv, values or "uniform", recipe, alpha, beta)
    raise ValueError(f"unknown recipe {recipe}")


def transposed_storage(prob: Problem, transa: bool, transb: bool) -> Problem:
    """The same product with A and/or B supplied as the transposed block matrix: masks and
    offset tables transposed, every tile copied as its transpose into a fresh arena."""
    def move(mask, off, arena, rows, cols):
        # tile (u, v) of a rows[u] x cols[v] grid -> tile (v, u) of the transposed grid
        mt = np.ascontiguousarray(mask.T)
        new_off, tot = layout_arena(mt, cols, rows)
        out = np.zeros(tot, arena.dtype)
        for u in range(mask.shape[0]):
            for v in range(mask.shape[1]):
                if mask[u, v]:
                    n = int(rows[u]) * int(cols[v])
                    x = arena[off[u, v]:off[u, v] + n].reshape(int(rows[u]), int(cols[v]))
                    out[new_off[v, u]:new_off[v, u] + n] = x.T.reshape(-1)
        return mt, new_off, out
    am, ao, A = (prob.a_mask, prob.a_off, prob.A)
    bm, bo, B = (prob.b_mask, prob.b_off, prob.B)
    if transa:
        am, ao, A = move(prob.a_mask, prob.a_off, prob.A, prob.row_sizes, prob.inner_sizes)
    if transb:
        bm, bo, B = move(prob.b_mask, prob.b_off, prob.B, prob.inner_sizes, prob.col_sizes)
    return Problem(prob.name + f"_t{int(transa)}{int(transb)}", prob.row_sizes, prob.col_sizes, prob.inner_sizes,
                   am, bm, ao, bo, A, B, prob.alpha, prob.beta, prob.c_mask, prob.recipe, bool(transa),
                   bool(transb))


def as_float32(prob: Problem) -> Problem:
    """The same product with float32 arenas: every stored value rounded to float32 (ties
    to even), the tiles laid out again with starts on multiples of 4 elements (16 bytes)."""
    def move(mask, off, arena, rows, cols):
        new_off, tot = layout_arena(mask, rows, cols, align=4)
        out = np.zeros(tot, np.float32)
        for u, v in zip(*np.nonzero(mask)):
            n = int(rows[u]) * int(cols[v])
            out[new_off[u, v]:new_off[u, v] + n] = arena[off[u, v]:off[u, v] + n].astype(np.float32)
        return new_off, out
    ar, ac = (prob.inner_sizes, prob.row_sizes) if prob.transa else (prob.row_sizes, prob.inner_sizes)
    br, bc = (prob.col_sizes, prob.inner_sizes) if prob.transb else (prob.inner_sizes, prob.col_sizes)
    ao, A = move(prob.a_mask, prob.a_off, prob.A, ar, ac)
    bo, B = move(prob.b_mask, prob.b_off, prob.B, br, bc)
    return dataclasses.replace(prob, name=prob.name + "_f32", a_off=ao, b_off=bo, A=A, B=B)


def as_complex(prob: Problem, seed: int) -> Problem:
    """The same structure with complex128 arenas: the real parts are the problem's values,
    the imaginary parts drawn alike (integers in [-8, 8] when the real parts are all
    integers, else U[-1,1]) from a stream of ``seed``. Offsets count complex elements."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(1)[0])
    def im(x):
        if x.size and np.all(x == np.round(x)):
            return fill_integers(x.size, rng)
        return fill_uniform(x.size, rng)
    A = (prob.A + 1j * im(prob.A)).astype(np.complex128)
    B = (prob.B + 1j * im(prob.B)).astype(np.complex128)
    return dataclasses.replace(prob, name=prob.name + "_c128", A=A, B=B)


def make_batch(count: int, seed: int, n_lo: int = 512, n_hi: int = 8192, b_lo: int = 32,
               b_hi: int = 192, d_lo: float = 0.1, d_hi: float = 1.0) -> List[Problem]:
    """Independent square products of uneven sizes: n ~ U-int[n_lo, n_hi], block sizes
    U-int[b_lo, b_hi], one tile density d ~ U[d_lo, d_hi] per product used for both
    masks, U[-1,1] entries."""
    top = np.random.default_rng(np.random.SeedSequence(seed).spawn(1)[0])
    probs = []
    for p in range(count):
        n = int(top.integers(n_lo, n_hi + 1))
        d = float(top.uniform(d_lo, d_hi))
        rt, rm, rv, _ = _streams(seed * 100003 + p + 1)
        r = tiling_uniform_int(n, b_lo, b_hi, rt)
        am = mask_bernoulli(len(r), len(r), d, rm)
        bm = mask_bernoulli(len(r), len(r), d, rm)
        probs.append(_assemble(f"batch{p}_n{n}_d{d:.2f}", r, r, r, am, bm, rv, "uniform", "batch"))
    return probs


def random_small(seed: int, max_blocks: int = 6, max_size: int = 40, allow_zero: bool = True,
                 density: float = 0.6, values: str = "uniform") -> Problem:
    """Tiny random problem with ragged tilings (zero-size blocks allowed) for brute-force pins."""
    rng = np.random.default_rng(seed)
    M, N, K = (int(x) for x in rng.integers(1, max_blocks + 1, 3))
    lo = 0 if allow_zero else 1
    r = rng.integers(lo, max_size + 1, M).astype(np.int32)
    c = rng.integers(lo, max_size + 1, N).astype(np.int32)
    q = rng.integers(lo, max_size + 1, K).astype(np.int32)
    am = (rng.random((M, K)) < density).astype(np.uint8)
    bm = (rng.random((K, N)) < density).astype(np.uint8)
    alpha = float(rng.choice([1.0, -0.5, 2.0, 0.75]))
    beta = float(rng.choice([0.0, 1.0, -2.0, 0.5]))
    return _assemble(f"small_s{seed}", r, c, q, am, bm, rng, values, "small", alpha, beta)
