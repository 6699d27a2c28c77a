"""Oracle for the split-precision modes (Ozaki-style error-free slicing).

TEST INFRASTRUCTURE ONLY: the library never imports this module.

The paper multiplies in FP64 with a BLAS DGEMM per tile task (Sec. 4.1). The
split modes compute the same tile tasks C_ij += A_ik B_kj (Sec. 2.1) with the
bulk of the arithmetic on low-precision integers, following the error-free
splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012), with one
power-of-two scale per tile:

  slicing of a tile X (beta = bits per slice, s = slices):
    mu = max |x|;  e = the smallest integer with mu < 2^e  (mu == 0: e = 0, slices 0)
    rho_0 = X * 2^-e                               (exact, |rho_0| < 1)
    for t = 1..s:  N_t = rint(rho_{t-1} * 2^(beta*t))    (round half to even)
                   rho_t = rho_{t-1} - N_t * 2^(-beta*t)  (exact)
    so X = 2^e * sum_t N_t 2^(-beta*t) + 2^e * rho_s,  |rho_s| <= 2^(-beta*s - 1)
    and |N_1| <= 2^beta, |N_t| <= 2^(beta-1) for t >= 2.

  product of one tile pair (A tile: e_A, NA_p;  B tile: e_B, NB_q):
    S_d = sum_{p+q=d} NA_p NB_q           (integer matrices, d = 2..s+1; pairs with
                                           p+q > s+1 are dropped)
    T   = sum_d S_d * 2^(beta*(s+1-d))    (an exact integer)
    contribution = T * 2^(e_A + e_B - beta*(s+1))

  accumulation, exact, then one rounding:
    each C element of tile (i, j) is the exact sum over its k blocks of
      T_k * 2^(E_k),  E_k = e_A(i,k) + e_B(k,j) - beta*(s+1),
    formed here as one Python integer in units of 2^(min_k E_k) (every term enters
    with its full value: nothing below any unit is dropped); that exact value is
    rounded once to the output format (round to nearest, ties to even, subnormal
    results rounded directly on the subnormal grid) and the epilogue is
    C_ij = fl(alpha*acc) + fl(beta*C_ij) as in the FP64 oracle.

Because the sum is exact before its single rounding, the value does not depend on
the order in which tile pairs, slice pairs or k blocks are added.

Row/column scaling (scaling="rows"): the same slicing with one exponent per row of an
A tile and per column of a B tile (e_A(i,k)[ii], e_B(k,j)[jj]); an all-zero row or
column has exponent 0 and zero slices. The contribution of a tile pair to element
(ii, jj) is T[ii,jj] * 2^(e_A[ii] + e_B[jj] - beta*(s+1)); the exact sum and its single
rounding are as above.

Complex elements (complex128 arenas, real alpha and beta): one exponent per tile (per
row of A and column of B with row/column scaling) over the real and imaginary parts
together; both parts sliced with it; per tile pair
the exact integers T_re = T(Ar,Br) - T(Ai,Bi) and T_im = T(Ar,Bi) + T(Ai,Br) (the complex
product's definition), accumulated and rounded like a real element, each part on its own;
the epilogue applies alpha and beta to each part.

Float32 elements (a float32 C arena; A and B may be float32 as well): the slicing and the
exact sum are the same (float32 values are exact in float64); the sum is rounded once to
binary32 (24-bit significand, subnormals on their own grid, ties to even) and the epilogue
runs in float32: C = fl32(fl32(alpha*acc) + fl32(beta*C)). With float64 C the exact sum is
rounded once to binary64 by Python's correctly rounded integer division, the epilogue in
float64.

All integer matrix products below go through a float64 matmul: every entry is an
integer of magnitude below 2^53, so the library routine returns it exactly in
any summation order.
"""
from __future__ import annotations

import math

import numpy as np

BETA_BITS = 7


def tile_exponent(x: np.ndarray) -> int:
    """Smallest integer e with max|x| < 2^e (0 for an all-zero or empty tile)."""
    if x.size == 0:
        return 0
    mu = float(np.max(np.abs(x)))
    if mu == 0.0:
        return 0
    _, e = np.frexp(mu)
    return int(e)


def slice_tile(x: np.ndarray, s: int, beta: int = BETA_BITS, e=None):
    """Error-free slicing of one tile (with its own exponent, or the given one). Returns
    (e, [N_1..N_s] as float64 integer matrices, rho_s residual in units of 2^e)."""
    e = tile_exponent(x) if e is None else e
    rho = np.ldexp(np.asarray(x, np.float64), -e)
    slices = []
    for t in range(1, s + 1):
        n_t = np.rint(np.ldexp(rho, beta * t))
        rho = rho - np.ldexp(n_t, -beta * t)
        slices.append(n_t)
    return e, slices, rho


def slice_rows(x: np.ndarray, s: int, beta: int = BETA_BITS, e=None):
    """Error-free slicing with one exponent per row (its own, or the given ones). Returns
    (e per row, nonzero-row flags, [N_1..N_s], rho_s residual in units of 2^e per row); an
    all-zero row has e = 0 and zero slices."""
    x = np.asarray(x, np.float64)
    if e is None:
        e = np.array([tile_exponent(row) for row in x], np.int64) if x.shape[0] else np.zeros(0, np.int64)
    nz = np.array([bool(np.any(row != 0)) for row in x], bool) if x.shape[0] else np.zeros(0, bool)
    rho = np.ldexp(x, -e[:, None]) if x.size else x.copy()
    slices = []
    for t in range(1, s + 1):
        n_t = np.rint(np.ldexp(rho, beta * t))
        rho = rho - np.ldexp(n_t, -beta * t)
        slices.append(n_t)
    return e, nz, slices, rho


def pair_integer(na, nb, s: int, beta: int = BETA_BITS) -> np.ndarray:
    """T = sum_d S_d 2^(beta(s+1-d)) for one tile pair: an int64 matrix, or a matrix of
    Python integers when the tile pair's inner depth n could take |T| beyond int64.

    |N_p N_q| <= 2^(2 beta), so |S_d| <= (d-1) n 2^(2 beta): each S_d is exact in the
    float64 matmul while s n 2^(2 beta) < 2^53 (checked), and |T| < 2 s n 2^(2 beta)
    2^(beta(s-1))."""
    r = na[0].shape[0]
    c = nb[0].shape[1]
    n = na[0].shape[1]
    if s * n * 2.0 ** (2 * beta) >= 2.0 ** 53:
        raise ValueError(f"pair_integer: inner depth {n} is beyond exact float64 slice sums")
    big = 2 * s * n * 2 ** (2 * beta + beta * (s - 1)) >= 2 ** 63
    T = np.zeros((r, c), object if big else np.int64)
    if r == 0 or c == 0:
        return T
    for d in range(2, s + 2):
        Sd = np.zeros((r, c), np.float64)
        for p in range(1, d):
            q = d - p
            if p > s or q > s:
                continue
            Sd += na[p - 1] @ nb[q - 1]
        if big:
            T += Sd.astype(np.int64).astype(object) * (1 << (beta * (s + 1 - d)))
        else:
            T += Sd.astype(np.int64) << np.int64(beta * (s + 1 - d))
    return T


def round_significand(v: int, bits: int) -> int:
    """The integer v rounded to ``bits`` significant bits, ties to even."""
    if v == 0:
        return 0
    a = abs(v)
    n = a.bit_length()
    if n <= bits:
        return v
    sh = n - bits
    q, rem, half = a >> sh, a & ((1 << sh) - 1), 1 << (sh - 1)
    if rem > half or (rem == half and (q & 1)):
        q += 1
    return (q << sh) if v > 0 else -(q << sh)


def round_binary32(v: int, L: int) -> np.float32:
    """v * 2^L rounded once to binary32: the last place of a normal result is 2^(E-23) for
    a value in [2^E, 2^(E+1)), of a subnormal one 2^-149; ties to even; overflow to inf."""
    if v == 0:
        return np.float32(0.0)
    a = abs(v)
    E = a.bit_length() - 1 + L
    Q = max(E - 23, -149)              # exponent of the last place
    sh = Q - L
    if sh <= 0:
        m = a << (-sh)
    else:
        m, rem, half = a >> sh, a & ((1 << sh) - 1), 1 << (sh - 1)
        if rem > half or (rem == half and (m & 1)):
            m += 1
    if m.bit_length() + Q > 128:       # |result| >= 2^128
        out = math.inf
    else:
        out = math.ldexp(float(m), Q)  # m <= 2^24: exact
    return np.float32(out if v > 0 else -out)


def round_binary64(v: int, L: int) -> float:
    """v * 2^L rounded once to binary64 (Python's int-to-float conversion and int / int
    division are correctly rounded, ties to even, subnormals included); overflow to inf."""
    try:
        return float(v << L) if L >= 0 else v / (1 << -L)
    except OverflowError:
        return math.copysign(math.inf, v)


def _finish(exact, L, ct, alpha: float, bet: float):
    """ct (a C tile, float64 or float32) = alpha*acc + beta*ct, acc = the exact integers
    times 2^L (L a scalar or per element) rounded once to ct's precision."""
    Ls = np.broadcast_to(np.asarray(L, dtype=object), exact.shape)
    if ct.dtype == np.float32:
        acc = np.array([round_binary32(int(v), int(l)) for v, l in zip(exact.reshape(-1), Ls.reshape(-1))],
                       np.float32).reshape(exact.shape)
        u = np.float32(alpha) * acc
        ct[...] = (u + np.float32(bet) * ct) if bet != 0.0 else u
    else:
        acc = np.array([round_binary64(int(v), int(l)) for v, l in zip(exact.reshape(-1), Ls.reshape(-1))],
                       np.float64).reshape(exact.shape)
        u = alpha * acc
        ct[...] = (u + bet * ct) if bet != 0.0 else u


def bsmm_split(prob_like, c_struct, C, c_off, s: int, beta: int = BETA_BITS, tiles=None, scaling: str = "tile"):
    """Split-mode product in place on the C arena (numpy arrays). ``prob_like``
    carries row_sizes, col_sizes, inner_sizes, a_mask, b_mask, a_off, b_off, A, B,
    alpha, beta. ``tiles`` restricts the work to a list of (i, j) C tiles; ``scaling``
    is "tile" (one exponent per tile) or "rows" (per row of A, per column of B)."""
    if scaling == "rows":
        return _bsmm_split_rows(prob_like, c_struct, C, c_off, s, beta, tiles)
    assert scaling == "tile", scaling
    r = np.asarray(prob_like.row_sizes, np.int64)
    c = np.asarray(prob_like.col_sizes, np.int64)
    q = np.asarray(prob_like.inner_sizes, np.int64)
    M, N, K = len(r), len(c), len(q)
    # transposed storage (see the generator's Problem): masks and offsets in (i,k) / (k,j)
    # indexing, tiles read back to their r_i x q_k / q_k x c_j shape
    ta, tb = bool(getattr(prob_like, "transa", False)), bool(getattr(prob_like, "transb", False))
    am = prob_like.a_mask.T if ta else prob_like.a_mask
    bm = prob_like.b_mask.T if tb else prob_like.b_mask
    a_off = prob_like.a_off.T if ta else prob_like.a_off
    b_off = prob_like.b_off.T if tb else prob_like.b_off
    cacheA, cacheB = {}, {}
    cplx = np.iscomplexobj(prob_like.A)

    def sl(x):  # (e, slices) or, for complex tiles, (e, (slices of re, slices of im))
        if not cplx:
            e, sl_, _ = slice_tile(x, s, beta)
            return e, sl_
        e = tile_exponent(np.concatenate([x.real.ravel(), x.imag.ravel()]))
        return e, (slice_tile(x.real, s, beta, e)[1], slice_tile(x.imag, s, beta, e)[1])

    def a_sl(i, k):
        if (i, k) not in cacheA:
            o = int(a_off[i, k])
            x = (prob_like.A[o:o + r[i] * q[k]].reshape(q[k], r[i]).T if ta
                 else prob_like.A[o:o + r[i] * q[k]].reshape(r[i], q[k]))
            cacheA[(i, k)] = sl(x)
        return cacheA[(i, k)]

    def b_sl(k, j):
        if (k, j) not in cacheB:
            o = int(b_off[k, j])
            x = (prob_like.B[o:o + q[k] * c[j]].reshape(c[j], q[k]).T if tb
                 else prob_like.B[o:o + q[k] * c[j]].reshape(q[k], c[j]))
            cacheB[(k, j)] = sl(x)
        return cacheB[(k, j)]

    todo = tiles if tiles is not None else [(i, j) for i in range(M) for j in range(N) if c_struct[i, j]]
    alpha, bet = float(prob_like.alpha), float(prob_like.beta)
    for (i, j) in todo:
        # every term of the exact sum: (T per part, its binary position E_k)
        terms = []
        for k in range(K):
            if not (am[i, k] and bm[k, j]):
                continue
            eA, na = a_sl(i, k)
            eB, nb = b_sl(k, j)
            if cplx:
                (ar, ai), (br, bi) = na, nb
                Ts = [pair_integer(ar, br, s, beta).astype(object) - pair_integer(ai, bi, s, beta).astype(object),
                      pair_integer(ar, bi, s, beta).astype(object) + pair_integer(ai, br, s, beta).astype(object)]
            else:
                Ts = [pair_integer(na, nb, s, beta).astype(object)]
            terms.append((Ts, eA + eB - beta * (s + 1)))
        L = min((E for _, E in terms), default=0)  # the unit of the exact sum: every shift below is >= 0
        parts = [np.zeros((r[i], c[j]), dtype=object) for _ in range(2 if cplx else 1)]
        for ex in parts:
            ex[...] = 0
        for Ts, E in terms:
            for t, T in enumerate(Ts):
                parts[t] = parts[t] + T * (1 << (E - L))
        o = int(c_off[i, j])
        ct = C[o:o + r[i] * c[j]].reshape(r[i], c[j])
        if cplx:
            _finish(parts[0], L, ct.real, alpha, bet)
            _finish(parts[1], L, ct.imag, alpha, bet)
        else:
            _finish(parts[0], L, ct, alpha, bet)
    return C


def _bsmm_split_rows(prob_like, c_struct, C, c_off, s, beta, tiles):
    """bsmm_split with one exponent per row of A and per column of B. Complex elements:
    one exponent per row (column) over the real and imaginary parts together, both parts
    sliced with it, the parts of the product as in tile mode."""
    cplx = np.iscomplexobj(prob_like.A)
    r = np.asarray(prob_like.row_sizes, np.int64)
    c = np.asarray(prob_like.col_sizes, np.int64)
    q = np.asarray(prob_like.inner_sizes, np.int64)
    M, N, K = len(r), len(c), len(q)
    ta, tb = bool(getattr(prob_like, "transa", False)), bool(getattr(prob_like, "transb", False))
    am = prob_like.a_mask.T if ta else prob_like.a_mask
    bm = prob_like.b_mask.T if tb else prob_like.b_mask
    a_off = prob_like.a_off.T if ta else prob_like.a_off
    b_off = prob_like.b_off.T if tb else prob_like.b_off
    cacheA, cacheB = {}, {}

    def lines(x):  # per row of x: (e, nonzero, slices) or, complex, (e, nonzero, (re slices, im slices))
        if not cplx:
            e, nz, sl, _ = slice_rows(x, s, beta)
            return e, nz, sl
        both = np.concatenate([x.real, x.imag], axis=1)  # one exponent over both parts of a row
        e, nz, _, _ = slice_rows(both, s, beta)
        return e, nz, (slice_rows(x.real, s, beta, e)[2], slice_rows(x.imag, s, beta, e)[2])

    def a_sl(i, k):  # per row of A_ik: (e[r_i], nonzero[r_i], slices)
        if (i, k) not in cacheA:
            o = int(a_off[i, k])
            x = (prob_like.A[o:o + r[i] * q[k]].reshape(q[k], r[i]).T if ta
                 else prob_like.A[o:o + r[i] * q[k]].reshape(r[i], q[k]))
            cacheA[(i, k)] = lines(x)
        return cacheA[(i, k)]

    def b_sl(k, j):  # per column of B_kj: slicing of the transpose, slices turned back
        if (k, j) not in cacheB:
            o = int(b_off[k, j])
            x = (prob_like.B[o:o + q[k] * c[j]].reshape(c[j], q[k]).T if tb
                 else prob_like.B[o:o + q[k] * c[j]].reshape(q[k], c[j]))
            e, nz, sl = lines(x.T)
            back = (lambda v: [t.T for t in v])
            cacheB[(k, j)] = (e, nz, (back(sl[0]), back(sl[1])) if cplx else back(sl))
        return cacheB[(k, j)]

    todo = tiles if tiles is not None else [(i, j) for i in range(M) for j in range(N) if c_struct[i, j]]
    alpha, bet = float(prob_like.alpha), float(prob_like.beta)
    for (i, j) in todo:
        terms = []  # (T per part, per-element binary position E_k[ii, jj])
        for k in range(K):
            if not (am[i, k] and bm[k, j]):
                continue
            eA, _, na = a_sl(i, k)
            eB, _, nb = b_sl(k, j)
            if cplx:
                (ar, ai), (br, bi) = na, nb
                Ts = [pair_integer(ar, br, s, beta).astype(object) - pair_integer(ai, bi, s, beta).astype(object),
                      pair_integer(ar, bi, s, beta).astype(object) + pair_integer(ai, br, s, beta).astype(object)]
            else:
                Ts = [pair_integer(na, nb, s, beta).astype(object)]
            terms.append((Ts, eA[:, None] + eB[None, :] - beta * (s + 1)))
        # per element, the unit of the exact sum: the lowest position of its terms
        L = np.zeros((r[i], c[j]), np.int64)
        if terms:
            L = np.minimum.reduce([E for _, E in terms])
        parts = [np.zeros((r[i], c[j]), dtype=object) for _ in range(2 if cplx else 1)]
        for ex in parts:
            ex[...] = 0
        for Ts, E in terms:
            sh = np.left_shift(np.ones_like(E, dtype=object), (E - L).astype(object))
            for t, T in enumerate(Ts):
                if T.size:
                    parts[t] = parts[t] + T * sh
        o = int(c_off[i, j])
        ct = C[o:o + r[i] * c[j]].reshape(r[i], c[j])
        if cplx:
            _finish(parts[0], L, ct.real, alpha, bet)
            _finish(parts[1], L, ct.imag, alpha, bet)
        else:
            _finish(parts[0], L, ct, alpha, bet)
    return C
