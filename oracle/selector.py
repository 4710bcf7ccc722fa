"""Oracle for the configuration-search side of the library: graph features
and the selector MLP (forward, backward, masked MSE, Adam), in float64 numpy.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s baseline legs may import it.  It shares nothing with
``paper_2501_06872_gb300``: the SplitMix64 generator below is written from
its published definition (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), the features from their stated definitions,
the network from the textbook equations of a fully connected ReLU network
and Adam (Kingma & Ba, ICLR 2015).

Nothing here is from the paper: the paper prints no selector.  What pins it:
the published SplitMix64 outputs, closed forms on structured graphs, brute
force (plain sort / unique) against the histogram walks the kernels use, and
central finite differences for every gradient (parity of the GPU f32 kernels
against this fp64 code is therefore within f32 tolerance, not bit-exact).
"""
from __future__ import annotations

import math

import numpy as np

N_FEATURES = 41
GRID = 12
HIDDEN = 64
M64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(state: int) -> int:
    """Output function of SplitMix64 applied to a 64-bit state."""
    z = state & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def stream(seed: int, count: int):
    """Outputs 1..count of the SplitMix64 sequence started at `seed`
    (state_j = seed + j * golden gamma)."""
    return [splitmix64(seed + j * GOLDEN_GAMMA) for j in range(1, count + 1)]


def scaled(r: int, bound: int) -> int:
    """floor(r * bound / 2^64): maps a 64-bit output onto [0, bound)."""
    return (r * bound) >> 64


def sample_count(n: int, m: int) -> int:
    if m == 0:
        return 0
    return min(max((n + 99) // 100, 1024), 1 << 20)


def features(n: int, m: int, row_ptr, col_idx, has_vals: bool, seed: int, n_cols=None) -> np.ndarray:
    """The GT_N_FEATURES graph features, by their definitions (float64, then
    rounded to float32 as the library stores them).  For an n x n_cols
    matrix, n counts rows (degree bins, top rows, sampled rows) and n_cols
    sets feature 32 and the sample count; n_cols defaults to n."""
    nc = n if n_cols is None else int(n_cols)
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    f = np.zeros(N_FEATURES, dtype=np.float64)
    deg = np.diff(row_ptr)
    bins = np.zeros(deg.shape, dtype=np.int64)
    nz = deg > 0
    # bin = bit length of the degree (1 + floor(log2 d)), exact through frexp
    bins[nz] = np.minimum(31, np.frexp(deg[nz].astype(np.float64))[1].astype(np.int64))
    vcnt = np.bincount(bins, minlength=32)[:32]
    esum = np.bincount(bins, weights=deg.astype(np.float64), minlength=32)[:32]
    f[:32] = vcnt / float(n)
    f[32] = math.log2(nc) / 32.0
    f[33] = math.log2(m + 1.0) / 32.0
    f[34] = math.log2(float(deg.max() if n else 0) + 1.0) / 32.0
    take, got = float((n + 99) // 100), 0.0
    for b in range(31, -1, -1):
        if take <= 0.0:
            break
        c = float(vcnt[b])
        if c == 0.0:
            continue
        if c <= take:
            got += float(esum[b])
            take -= c
        else:
            got += float(esum[b]) * (take / c)
            take = 0.0
    f[35] = got / m if m else 0.0
    ns = sample_count(nc, m)
    if ns:
        pos = [scaled(r, m) for r in stream(seed, ns)]
        dst = col_idx[np.array(pos, dtype=np.int64)]
        _, counts = np.unique(dst, return_counts=True)
        counts = np.sort(counts)[::-1]
        f[36] = float(counts[:512].sum()) / ns
        f[37] = math.log2(float(counts[0]) * m / ns + 1.0) / 32.0
        total, pairs, same = 0.0, 0, 0
        for r in stream(seed ^ 0x4C4F43, 4096):
            u = scaled(r, n)
            beg, end = int(row_ptr[u]), int(row_ptr[u + 1])
            if end > m or beg > end or end - beg < 2:
                continue
            for i in range(min(end - beg - 1, 32)):
                a, b = int(col_idx[beg + i]), int(col_idx[beg + i + 1])
                total += math.log2(abs(a - b) + 1.0)
                pairs += 1
                same += (a >> 5) == (b >> 5)
        if pairs:
            f[38] = total / pairs / 32.0
            f[39] = same / pairs
    f[40] = 1.0 if has_vals else 0.0
    return f.astype(np.float32)


# ---- selector network ---------------------------------------------------------

def layout(F: int = N_FEATURES, H: int = HIDDEN, K: int = GRID):
    """Offsets of mu, sd, lo, hi, W1, b1, W2, b2, W3, b3 in the flat parameter
    vector (lo, hi: the training feature range, unused by the network)."""
    sizes = [("mu", F), ("sd", F), ("lo", F), ("hi", F), ("W1", H * F), ("b1", H), ("W2", H * H), ("b2", H),
             ("W3", K * H), ("b3", K)]
    out, off = {}, 0
    for name, size in sizes:
        out[name] = (off, size)
        off += size
    out["total"] = off
    return out


def unpack(p, F=N_FEATURES, H=HIDDEN, K=GRID):
    lo = layout(F, H, K)
    p = np.asarray(p, dtype=np.float64)

    def g(name, shape):
        o, s = lo[name]
        return p[o:o + s].reshape(shape)
    return (g("mu", (F,)), g("sd", (F,)), g("W1", (H, F)), g("b1", (H,)), g("W2", (H, H)), g("b2", (H,)),
            g("W3", (K, H)), g("b3", (K,)))


def forward(p, X, F=N_FEATURES, H=HIDDEN, K=GRID):
    """y = W3 relu(W2 relu(W1 x' + b1) + b2) + b3 with x' = (x - mu) / sd."""
    mu, sd, W1, b1, W2, b2, W3, b3 = unpack(p, F, H, K)
    X = np.asarray(X, dtype=np.float64)
    xn = (X - mu) / sd
    a1 = xn @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ W3.T + b3
    return y, (xn, a1, h1, a2, h2)


def loss(p, X, T, M, F=N_FEATURES, H=HIDDEN, K=GRID):
    """Masked mean squared error: sum M (y - T)^2 / max(1, sum M)."""
    y, _ = forward(p, X, F, H, K)
    M = np.asarray(M, dtype=np.float64)
    return float((M * (y - T) ** 2).sum() / max(1.0, M.sum()))


def backward(p, X, T, M, F=N_FEATURES, H=HIDDEN, K=GRID):
    """(loss, gradient vector in the parameter layout; mu, sd, lo, hi get 0).
    The ReLU derivative is taken as 1 where the pre-activation is > 0."""
    mu, sd, W1, b1, W2, b2, W3, b3 = unpack(p, F, H, K)
    y, (xn, a1, h1, a2, h2) = forward(p, X, F, H, K)
    T = np.asarray(T, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    den = max(1.0, M.sum())
    L = float((M * (y - T) ** 2).sum() / den)
    dy = 2.0 * M * (y - T) / den
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3
    da2 = dh2 * (a2 > 0)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * (a1 > 0)
    gW1 = da1.T @ xn
    gb1 = da1.sum(axis=0)
    lo = layout(F, H, K)
    g = np.zeros(lo["total"], dtype=np.float64)
    for name, arr in (("W1", gW1), ("b1", gb1), ("W2", gW2), ("b2", gb2), ("W3", gW3), ("b3", gb3)):
        o, s = lo[name]
        g[o:o + s] = arr.reshape(-1)
    return L, g


def adam(p, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8, first=None, wd=0.0):
    """Adam step t (1-based) on entries [first, end) (all when first is None),
    with an L2 penalty wd/2 |p|^2: the moments see g + wd * p."""
    p, g, m1, m2 = (np.array(a, dtype=np.float64) for a in (p, g, m1, m2))
    lo = 0 if first is None else first
    gw = g[lo:] + wd * p[lo:]
    m1[lo:] = b1 * m1[lo:] + (1.0 - b1) * gw
    m2[lo:] = b2 * m2[lo:] + (1.0 - b2) * gw ** 2
    mh = m1[lo:] / (1.0 - b1 ** t)
    vh = m2[lo:] / (1.0 - b2 ** t)
    p[lo:] = p[lo:] - lr * mh / (np.sqrt(vh) + eps)
    return p, m1, m2
