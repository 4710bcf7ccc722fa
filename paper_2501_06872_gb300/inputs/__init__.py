"""Seeded synthetic inputs (CSR graphs) for tests and benchmarks.

This module holds no transposition arithmetic.  It makes graphs; both the
CUDA path and the oracle consume what it makes.  Two back ends:

* numpy (this file) for the small cases the CPU tests need: the R-MAT edge list
  is drawn edge by edge and turned into CSR by a stable library sort by source
  (so rows keep generation order);
* CUDA (``gen.cu`` via :mod:`.gpu`) for the large cases: R-MAT and uniform
  graphs are drawn directly in CSR order (see that module).

Randomness is counter based: ``draw(key, i)`` is the SplitMix64 output
function (Steele, Lea, Flood, OOPSLA 2014) applied to ``key + i*golden``, so
any element of any stream can be computed independently.  The seeded vertex
permutation is a 4-round Feistel network over the next even power of two with
cycle walking, which is a bijection on [0, n).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1

# Stream identifiers (shared with gen.cu so both back ends name streams alike).
S_RMAT = 1
S_PERM = 2
S_VALS = 3
S_ER = 4
S_DEG = 5
S_BATCH = 6
S_SAMPLE = 7


def mix64(x):
    """SplitMix64 finaliser on a uint64 numpy array (wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = x ^ (x >> np.uint64(30))
        x = x * _M1
        x = x ^ (x >> np.uint64(27))
        x = x * _M2
        x = x ^ (x >> np.uint64(31))
    return x


def mix64_int(x: int) -> int:
    x &= MASK64
    x ^= x >> 30
    x = (x * 0xBF58476D1CE4E5B9) & MASK64
    x ^= x >> 27
    x = (x * 0x94D049BB133111EB) & MASK64
    x ^= x >> 31
    return x


def stream_key(seed: int, *ids: int) -> int:
    """Key of a named stream: seed folded with stream ids."""
    k = mix64_int(seed)
    for i in ids:
        k = mix64_int(k ^ ((i + 0x9E3779B97F4A7C15) & MASK64))
    return k


def draw(key: int, ctr):
    """uint64 random values for counters ``ctr`` of stream ``key``."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + (ctr + np.uint64(1)) * GOLDEN)


def threshold32(p: float) -> int:
    """Integer threshold t with P(u32 < t) = p, rounded down."""
    return min(int(math.floor(p * 4294967296.0)), 0xFFFFFFFF)


# ----------------------------------------------------------------------------
# Vertex permutations
# ----------------------------------------------------------------------------

def _feistel_params(n: int):
    bits = max(2, (max(n, 2) - 1).bit_length())
    if bits % 2:
        bits += 1
    return bits // 2


def feistel_perm(n: int, seed: int, x=None) -> np.ndarray:
    """Seeded bijection on [0, n); returns perm[x] (for all x when x is None)."""
    half = _feistel_params(n)
    hmask = np.uint64((1 << half) - 1)
    keys = [np.uint64(stream_key(seed, S_PERM, r)) for r in range(4)]
    if x is None:
        x = np.arange(n, dtype=np.uint64)
    else:
        x = np.asarray(x, dtype=np.uint64).copy()
    out = x.copy()
    todo = np.ones(out.shape, dtype=bool)
    h = np.uint64(half)
    while True:
        cur = out[todo]
        left = cur >> h
        right = cur & hmask
        for k in keys:
            f = mix64(right ^ k) & hmask
            left, right = right, left ^ f
        cur = (left << h) | right
        out[todo] = cur
        still = np.zeros(out.shape, dtype=bool)
        still[todo] = cur >= np.uint64(n)
        if not still.any():
            break
        todo = still
    return out.astype(np.uint64)


def degree_sort_perm(n: int, dst: np.ndarray) -> np.ndarray:
    """perm[v] = rank of v by (in-degree descending, vertex ID ascending)."""
    deg = np.bincount(dst.astype(np.int64), minlength=n)
    order = np.lexsort((np.arange(n), -deg))  # last key primary
    perm = np.empty(n, dtype=np.uint64)
    perm[order] = np.arange(n, dtype=np.uint64)
    return perm


# ----------------------------------------------------------------------------
# Edge lists and CSR assembly
# ----------------------------------------------------------------------------

def rmat_edges(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed=1):
    """R-MAT edge list (Chakrabarti, Zhan, Faloutsos 2004): every edge picks one
    quadrant per level with probabilities (a, b, c, d), level 0 deciding the
    most significant bit.  Self-loops and duplicates are kept."""
    m = edge_factor << scale
    key = stream_key(seed, S_RMAT)
    ta = threshold32(a)
    tab = threshold32(a + b)
    tabc = threshold32(a + b + c)
    src = np.zeros(m, dtype=np.uint64)
    dst = np.zeros(m, dtype=np.uint64)
    e = np.arange(m, dtype=np.uint64)
    for lvl in range(scale):
        r = draw(key, e * np.uint64(scale) + np.uint64(lvl)) >> np.uint64(32)
        sbit = (r >= np.uint64(tab)).astype(np.uint64)
        dbit = (((r >= np.uint64(ta)) & (r < np.uint64(tab))) | (r >= np.uint64(tabc))).astype(np.uint64)
        shift = np.uint64(scale - 1 - lvl)
        src |= sbit << shift
        dst |= dbit << shift
    return src.astype(np.uint32), dst.astype(np.uint32)


def er_edges(n: int, m: int, seed=1):
    """G(n, m) with replacement: both endpoints i.i.d. uniform on [0, n)."""
    key = stream_key(seed, S_ER)
    e = np.arange(m, dtype=np.uint64)
    r = draw(key, e)
    src = ((r >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    dst = ((r & np.uint64(0xFFFFFFFF)) * np.uint64(n)) >> np.uint64(32)
    return src.astype(np.uint32), dst.astype(np.uint32)


def uniform_vals(m: int, seed: int, lo=0.0, hi=1.0, stream=S_VALS):
    """f32 values U(lo, hi) drawn from 24 random bits per edge."""
    key = stream_key(seed, stream)
    r = draw(key, np.arange(m, dtype=np.uint64)) >> np.uint64(40)
    u = r.astype(np.float64) * (1.0 / 16777216.0)
    return (lo + (hi - lo) * u).astype(np.float32)


def csr_from_edges(n: int, src, dst, vals=None):
    """CSR whose rows keep the order of the edge list (stable sort by source)."""
    src = np.asarray(src, dtype=np.uint32)
    dst = np.asarray(dst, dtype=np.uint32)
    order = np.argsort(src, kind="stable")
    counts = np.bincount(src.astype(np.int64), minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = dst[order]
    v = None if vals is None else np.asarray(vals, dtype=np.float32)[order]
    return row_ptr, np.ascontiguousarray(col_idx), v


def relabel(src, dst, perm):
    perm = np.asarray(perm)
    return perm[src].astype(np.uint32), perm[dst].astype(np.uint32)


def rmat_csr(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1, order="natural",
             weighted=False, sorted_rows=False):
    """R-MAT graph in CSR form.

    order: "natural" (generated IDs), "random" (seeded Feistel permutation of
    both endpoints) or "degree" (relabelled by descending in-degree, ties by
    ID).  sorted_rows sorts each row's destinations (stable)."""
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor, a, b, c, seed)
    if order == "random":
        src, dst = relabel(src, dst, feistel_perm(n, seed))
    elif order == "degree":
        src, dst = relabel(src, dst, degree_sort_perm(n, dst))
    elif order != "natural":
        raise ValueError(order)
    vals = uniform_vals(src.shape[0], seed) if weighted else None
    if sorted_rows:
        o = np.lexsort((dst, src))
        src, dst = src[o], dst[o]
        vals = None if vals is None else vals[o]
    return (n,) + csr_from_edges(n, src, dst, vals)


def er_csr(n, m, seed=1, weighted=False, order="random"):
    src, dst = er_edges(n, m, seed)
    if order == "random":
        src, dst = relabel(src, dst, feistel_perm(n, seed))
    vals = uniform_vals(m, seed) if weighted else None
    return (n,) + csr_from_edges(n, src, dst, vals)


def random_csr(n, m, seed=1, weighted=True, hot=0, hot_frac=0.0, n_cols=None):
    """Small uniform graph for edge-case tests; optionally a fraction of the
    edges goes to ``hot`` distinct high-in-degree vertices.  With n_cols, an
    n x n_cols matrix (destinations drawn from [0, n_cols))."""
    nc = n if n_cols is None else n_cols
    key = stream_key(seed, 99)
    r = draw(key, np.arange(2 * m + 1, dtype=np.uint64))
    src = ((r[:m] >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    dst = ((r[m:2 * m] >> np.uint64(32)) * np.uint64(nc)) >> np.uint64(32)
    if hot and hot_frac > 0:
        pick = (r[m:2 * m] & np.uint64(0xFFFF)) < np.uint64(int(hot_frac * 65536))
        dst = np.where(pick, (r[m:2 * m] >> np.uint64(16)) % np.uint64(min(hot, nc)), dst)
    vals = uniform_vals(m, seed, -1.0, 1.0) if weighted else None
    return (n,) + csr_from_edges(n, src.astype(np.uint32), dst.astype(np.uint32), vals)


def fold_rect(row_ptr, col_idx, row_shift: int, col_shift: int):
    """Rectangular matrix from a square CSR by relabelling: rows u become
    u >> row_shift (2^row_shift consecutive rows merge, keeping their edges in
    CSR order) and columns v become v >> col_shift.  For a graph with
    n = 2^s vertices the result is 2^(s - row_shift) x 2^(s - col_shift).
    Returns (n_rows, n_cols, row_ptr, col_idx)."""
    row_ptr = np.asarray(row_ptr, dtype=np.uint64)
    n = row_ptr.shape[0] - 1
    if n & ((1 << row_shift) - 1) or n & ((1 << col_shift) - 1):
        raise ValueError("the vertex count must be a multiple of both folds")
    rp = np.ascontiguousarray(row_ptr[::1 << row_shift])
    ci = (np.asarray(col_idx, dtype=np.uint32) >> np.uint32(col_shift)).astype(np.uint32)
    return n >> row_shift, n >> col_shift, rp, ci


# ----------------------------------------------------------------------------
# Batched Zipf-degree matrices (small numpy version, for CPU tests)
# ----------------------------------------------------------------------------

def zipf_mean(s: float, n: int) -> float:
    k = np.arange(1, n + 1, dtype=np.float64)
    w = k ** (-s)
    return float((k * w).sum() / w.sum())


def zipf_sample(u: np.ndarray, s: float, n: int) -> np.ndarray:
    """Inverse-CDF Zipf(s) on {1..n} for uniforms u in [0,1)."""
    k = np.arange(1, n + 1, dtype=np.float64)
    cdf = np.cumsum(k ** (-s))
    cdf /= cdf[-1]
    return np.minimum(np.searchsorted(cdf, u, side="right") + 1, n)


def zipf_matrix(n: int, mean_deg: float, seed: int, idx: int, s_out=2.0, s_in=1.5,
                lo=-1.0, hi=1.0):
    """One square sparse matrix: Zipf(s_out) out-degrees scaled to mean_deg
    (clamped to [1, n]), destinations Zipf(s_in) over a seeded permutation."""
    key = stream_key(seed, S_BATCH, idx)
    mu = zipf_mean(s_out, n)
    u = (draw(key, np.arange(n, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    z = zipf_sample(u, s_out, n)
    deg = np.clip(np.rint(z * (mean_deg / mu)), 1, n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(deg, out=row_ptr[1:])
    m = int(row_ptr[-1])
    key2 = stream_key(seed, S_BATCH, idx, 1)
    u2 = (draw(key2, np.arange(m, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    ranks = zipf_sample(u2, s_in, n) - 1
    col_idx = feistel_perm(n, stream_key(seed, S_BATCH, idx, 2), ranks).astype(np.uint32)
    vals = uniform_vals(m, stream_key(seed, S_BATCH, idx, 3), lo, hi)
    return n, row_ptr, col_idx, vals
