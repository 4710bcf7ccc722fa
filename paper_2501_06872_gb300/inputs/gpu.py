"""GPU back end of the seeded input generators (libgtgen.so via ctypes).

Graphs are drawn directly in CSR order (see gen.cu); PyTorch provides the
device memory, a prefix sum for row_ptr and, for the degree-sorted order, a
stable sort of the in-degrees.  Nothing here transposes anything.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import S_DEG, S_RMAT, S_VALS, stream_key

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
    for f in ["gtgen_split_degrees", "gtgen_permute_degrees", "gtgen_fill", "gtgen_feistel",
              "gtgen_invert", "gtgen_histogram", "gtgen_vals"]:
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
