"""GPU back end of the seeded input generators (libgtgen.so via ctypes).

Graphs are drawn directly in CSR order (see gen.cu); PyTorch provides the
device memory, a prefix sum for row_ptr and, for the degree-sorted order, a
stable sort of the in-degrees.  Nothing here transposes anything.
"""
from __future__ import annotations

import ctypes
import os

import torch

import math

import numpy as np

from . import S_BATCH, S_DEG, S_RMAT, S_VALS, stream_key

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(os.path.dirname(_HERE), "_build", "libgtgen.so")
_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build with __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, u32, u64, d = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    lib.gtgen_split_degrees.argtypes = [u32, u64, d, u64, P, P, P]
    lib.gtgen_permute_degrees.argtypes = [u32, P, P, P, P]
    lib.gtgen_fill.argtypes = [u32, u32, P, P, P, P, u64, d, d, d, ctypes.c_int, P]
    lib.gtgen_feistel.argtypes = [u32, u64, P, P, P]
    lib.gtgen_invert.argtypes = [u32, P, P, P]
    lib.gtgen_histogram.argtypes = [P, u64, P, P]
    lib.gtgen_vals.argtypes = [u64, u64, ctypes.c_float, ctypes.c_float, P, P]
    lib.gtgen_zipf_degrees.argtypes = [u32, P, P, P, d, u64, P, P]
    lib.gtgen_batch_rowptr.argtypes = [u32, P, P, P, P]
    lib.gtgen_zipf_dst.argtypes = [u32, P, P, d, u64, u64, P, P]
    for f in ["gtgen_split_degrees", "gtgen_permute_degrees", "gtgen_fill", "gtgen_feistel",
              "gtgen_invert", "gtgen_histogram", "gtgen_vals", "gtgen_zipf_degrees", "gtgen_batch_rowptr",
              "gtgen_zipf_dst"]:
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with CUDA error {rc}")


def feistel_perm(n: int, seed: int, device="cuda"):
    perm = torch.empty(n, dtype=torch.int32, device=device)
    inv = torch.empty(n, dtype=torch.int32, device=device)
    _ok(load().gtgen_feistel(n, seed, _p(perm), _p(inv), _s()), "gtgen_feistel")
    return perm, inv


def _row_ptr_from(deg_perm):
    n = deg_perm.numel()
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=deg_perm.device)
    torch.cumsum(deg_perm, 0, out=row_ptr[1:])
    return row_ptr


def _split_degrees(scale, m, p0, key, device):
    n = 1 << scale
    deg = torch.empty(n, dtype=torch.int64, device=device)
    tmp = torch.empty(n, dtype=torch.int64, device=device)
    _ok(load().gtgen_split_degrees(scale, m, p0, key, _p(deg), _p(tmp), _s()), "gtgen_split_degrees")
    del tmp
    return deg


def _fill(n, scale, deg, perm, inv, key, a, b, c, uniform, device):
    lib = load()
    if perm is not None:
        dp = torch.empty_like(deg)
        _ok(lib.gtgen_permute_degrees(n, _p(deg), _p(perm), _p(dp), _s()), "gtgen_permute_degrees")
    else:
        dp = deg
    row_ptr = _row_ptr_from(dp)
    del dp
    m = int(row_ptr[-1].item())
    col_idx = torch.empty(m, dtype=torch.int32, device=device)
    _ok(lib.gtgen_fill(n, scale, _p(inv), _p(perm), _p(row_ptr), _p(col_idx), key, a, b, c, int(uniform), _s()),
        "gtgen_fill")
    return row_ptr, col_idx


def graph(scale: int, edge_factor: int = 16, kind: str = "rmat", a=0.57, b=0.19, c=0.19, seed: int = 1,
          order: str = "natural", weighted: bool = False, val_range=(0.0, 1.0), device="cuda"):
    """Seeded R-MAT ("rmat") or uniform ("er") graph on the GPU.

    order: "natural", "random" (seeded Feistel relabelling of both endpoints)
    or "degree" (relabelled by descending in-degree, ties by ID).
    Returns (n, row_ptr int64[n+1], col_idx int32[m], vals float32[m] | None)."""
    n = 1 << scale
    m = edge_factor << scale
    uniform = kind == "er"
    p0 = 0.5 if uniform else (a + b)
    deg = _split_degrees(scale, m, p0, stream_key(seed, S_DEG), device)
    key = stream_key(seed, S_RMAT)
    perm = inv = None
    if order == "random":
        perm, inv = feistel_perm(n, seed, device)
    elif order == "degree":
        rp0, ci0 = _fill(n, scale, deg, None, None, key, a, b, c, uniform, device)
        counts = torch.zeros(n, dtype=torch.int32, device=device)
        _ok(load().gtgen_histogram(_p(ci0), ci0.numel(), _p(counts), _s()), "gtgen_histogram")
        del rp0, ci0
        order_ids = torch.sort(counts.to(torch.int64), descending=True, stable=True).indices
        del counts
        perm = torch.empty(n, dtype=torch.int32, device=device)
        perm[order_ids] = torch.arange(n, dtype=torch.int32, device=device)
        inv = order_ids.to(torch.int32)
        del order_ids
    elif order != "natural":
        raise ValueError(order)
    row_ptr, col_idx = _fill(n, scale, deg, perm, inv, key, a, b, c, uniform, device)
    del deg, perm, inv
    vals = None
    if weighted:
        vals = torch.empty(col_idx.numel(), dtype=torch.float32, device=device)
        _ok(load().gtgen_vals(col_idx.numel(), stream_key(seed, S_VALS), float(val_range[0]),
                              float(val_range[1]), _p(vals), _s()), "gtgen_vals")
    torch.cuda.synchronize()
    return n, row_ptr, col_idx, vals


def fold_rect(row_ptr, col_idx, row_shift: int, col_shift: int):
    """Rectangular matrix from a square CSR by relabelling (as inputs.fold_rect):
    rows u -> u >> row_shift (consecutive rows merge, edges keep CSR order),
    columns v -> v >> col_shift, in place on col_idx.  Returns (n_rows,
    n_cols, row_ptr, col_idx)."""
    n = row_ptr.numel() - 1
    if n & ((1 << row_shift) - 1) or n & ((1 << col_shift) - 1):
        raise ValueError("the vertex count must be a multiple of both folds")
    rp = row_ptr[::1 << row_shift].contiguous() if row_shift else row_ptr
    if col_shift:
        col_idx.bitwise_right_shift_(col_shift)  # IDs < 2^31: the sign bit is clear
    torch.cuda.synchronize()
    return n >> row_shift, n >> col_shift, rp, col_idx


def _zipf_mean(s: float, n: int) -> float:
    """Mean of Zipf(s) truncated to {1..n}: ratio of generalised harmonic
    numbers, by direct sum for small n and Euler-Maclaurin tails otherwise."""
    def gh(p, n):
        if n <= 20000:
            k = np.arange(1, n + 1, dtype=np.float64)
            return float(np.sum(k ** (-p)))
        k = np.arange(1, 20001, dtype=np.float64)
        head = float(np.sum(k ** (-p)))
        a, b = 20000.5, n + 0.5
        if abs(p - 1.0) < 1e-12:
            return head + math.log(b / a)
        return head + (b ** (1 - p) - a ** (1 - p)) / (1 - p)
    return gh(s - 1.0, n) / gh(s, n)


def batch(n_graphs: int = 4096, seed: int = 0x5EED0004, n_min: int = 1024, n_max: int = 262144,
          mean_lo: float = 8.0, mean_hi: float = 32.0, s_out: float = 2.0, s_in: float = 1.5,
          weighted: bool = True, device="cuda"):
    """Batch of square sparse matrices: sizes log-uniform in [n_min, n_max],
    per-row out-degree round(Z * mean / mu) with Z ~ Zipf(s_out) and mean ~
    U[mean_lo, mean_hi] (clamped to [1, n]), destinations Zipf(s_in) ranks
    over a seeded permutation, values U(-1, 1).  All matrices live in union
    buffers; returns a dict with the buffers, offsets and per-graph sizes."""
    rng = np.random.default_rng(stream_key(seed, S_BATCH) & 0xFFFFFFFFFFFF)
    nv = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_graphs))).astype(np.int64)
    nv = np.clip(nv, n_min, n_max)
    means = rng.uniform(mean_lo, mean_hi, size=n_graphs)
    scale = np.array([means[i] / _zipf_mean(s_out, int(nv[i])) for i in range(n_graphs)], dtype=np.float64)
    voff = np.zeros(n_graphs + 1, dtype=np.int64)
    np.cumsum(nv, out=voff[1:])
    lib = load()
    d_nv = torch.from_numpy(nv.astype(np.int32)).to(device)
    d_voff = torch.from_numpy(voff).to(device)
    d_scale = torch.from_numpy(scale).to(device)
    total_v = int(voff[-1])
    deg = torch.empty(total_v, dtype=torch.int64, device=device)
    _ok(lib.gtgen_zipf_degrees(n_graphs, _p(d_voff), _p(d_nv), _p(d_scale), s_out, stream_key(seed, S_BATCH, 1),
                               _p(deg), _s()), "gtgen_zipf_degrees")
    ex = torch.zeros(total_v + 1, dtype=torch.int64, device=device)
    torch.cumsum(deg, 0, out=ex[1:])
    del deg
    rp = torch.empty(total_v + n_graphs, dtype=torch.int64, device=device)
    _ok(lib.gtgen_batch_rowptr(n_graphs, _p(d_voff), _p(ex), _p(rp), _s()), "gtgen_batch_rowptr")
    d_eoff = ex[d_voff].contiguous()
    del ex
    total_m = int(d_eoff[-1].item())
    col = torch.empty(total_m, dtype=torch.int32, device=device)
    _ok(lib.gtgen_zipf_dst(n_graphs, _p(d_eoff), _p(d_nv), s_in, stream_key(seed, S_BATCH, 2),
                           stream_key(seed, S_BATCH, 3), _p(col), _s()), "gtgen_zipf_dst")
    vals = None
    if weighted:
        vals = torch.empty(total_m, dtype=torch.float32, device=device)
        _ok(lib.gtgen_vals(total_m, stream_key(seed, S_BATCH, 4), -1.0, 1.0, _p(vals), _s()), "gtgen_vals")
    torch.cuda.synchronize()
    eoff = d_eoff.cpu().numpy()
    return {"n": nv, "m": np.diff(eoff), "voff": voff, "eoff": eoff, "row_ptr": rp, "col_idx": col, "vals": vals,
            "n_graphs": n_graphs, "total_m": total_m, "total_v": total_v}


def batch_graphs(b, col_ptr, row_idx, vals_out):
    """Per-graph descriptor dicts over union buffers (inputs of b, outputs given)."""
    out = []
    rp, ci, vv = b["row_ptr"], b["col_idx"], b["vals"]
    for g in range(b["n_graphs"]):
        n, m = int(b["n"][g]), int(b["m"][g])
        r0 = int(b["voff"][g]) + g
        e0 = int(b["eoff"][g])
        out.append({"n": n, "m": m,
                    "row_ptr": rp.data_ptr() + 8 * r0, "col_idx": ci.data_ptr() + 4 * e0,
                    "vals": None if vv is None else vv.data_ptr() + 4 * e0,
                    "col_ptr": col_ptr.data_ptr() + 8 * r0, "row_idx": row_idx.data_ptr() + 4 * e0,
                    "vals_out": None if vals_out is None else vals_out.data_ptr() + 4 * e0})
    return out
