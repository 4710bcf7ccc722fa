"""Oracle for the graph-transposition hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It is independent of the CUDA path: it shares no source, header,
constant or helper with ``paper_2501_06872_gb300``, and neither imports the
other.

``transpose`` follows Algorithm 1 (Atomic GT, Sec. II-B) executed by a single
thread, which turns it into a stable counting sort of the CSR edge sequence by
destination (see ``gt_oracle.c``).  The result is the CSC of Sec. II-A with
every in-list in ascending source order and duplicate edges in CSR order.
Rectangular matrices (``n_cols`` columns, ``len(row_ptr) - 1`` rows) follow
the same definition; the default is the square case of a graph.
``transpose64`` is the same definition with 64-bit vertex IDs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

ERRORS = {0: "ok", 1: "invalid argument", 2: "col_idx out of range", 3: "bad row_ptr",
          4: "out of memory", 5: "degree overflow"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, '?')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile gt_oracle.c with gcc (plain -O2, no vendor or arch flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    lib.oracle_transpose.argtypes = [ctypes.c_uint32, ctypes.c_uint64, P, P, P, P, P, P]
    lib.oracle_transpose.restype = ctypes.c_int
    lib.oracle_transpose_rect.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, P, P, P, P, P, P]
    lib.oracle_transpose_rect.restype = ctypes.c_int
    lib.oracle_transpose_range.argtypes = [ctypes.c_uint32, ctypes.c_uint64, P, P, P,
                                           ctypes.c_uint32, ctypes.c_uint32, P, P, P]
    lib.oracle_transpose_range.restype = ctypes.c_int
    lib.oracle_columns.argtypes = [ctypes.c_uint32, ctypes.c_uint64, P, P, P, P, ctypes.c_uint64,
                                   P, P, P, P, ctypes.c_uint64]
    lib.oracle_columns.restype = ctypes.c_int
    lib.oracle_columns_rect.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, P, P, P, P,
                                        ctypes.c_uint64, P, P, P, P, ctypes.c_uint64]
    lib.oracle_columns_rect.restype = ctypes.c_int
    lib.oracle_transpose64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, P, P, P, P, P, P]
    lib.oracle_transpose64.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _inputs(row_ptr, col_idx, vals):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.uint32)
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.float32)
        if vals.shape != col_idx.shape:
            raise ValueError("vals must have one entry per edge")
    n = row_ptr.shape[0] - 1
    if n < 0 or n > 0xFFFFFFFF:
        raise ValueError("row_ptr must have n+1 entries with n < 2^32")
    return n, row_ptr, col_idx, vals


def _cols(n, n_cols):
    n_cols = n if n_cols is None else int(n_cols)
    if n_cols < 0 or n_cols > 0xFFFFFFFF:
        raise ValueError("n_cols must lie in [0, 2^32)")
    return n_cols


def transpose(row_ptr, col_idx, vals=None, n_cols=None):
    """CSR -> CSC.  Returns (col_ptr u64[n_cols+1], row_idx u32[m], vals_out
    f32[m] or None); n_cols defaults to the row count (a graph)."""
    n, row_ptr, col_idx, vals = _inputs(row_ptr, col_idx, vals)
    nc = _cols(n, n_cols)
    m = col_idx.shape[0]
    col_ptr = np.empty(nc + 1, dtype=np.uint64)
    row_idx = np.empty(m, dtype=np.uint32)
    vals_out = np.empty(m, dtype=np.float32) if vals is not None else None
    rc = _load().oracle_transpose_rect(n, nc, m, _ptr(row_ptr), _ptr(col_idx), _ptr(vals),
                                       _ptr(col_ptr), _ptr(row_idx), _ptr(vals_out))
    if rc:
        raise OracleError(rc)
    return col_ptr, row_idx, vals_out


def transpose64(row_ptr, col_idx, vals=None, n_cols=None):
    """CSR -> CSC with 64-bit vertex IDs: row_ptr u64[n_rows+1], col_idx
    u64[m] (< n_cols, default n_rows).  Returns (col_ptr u64[n_cols+1],
    row_idx u64[m], vals_out f32[m] or None)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.uint64)
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.float32)
        if vals.shape != col_idx.shape:
            raise ValueError("vals must have one entry per edge")
    n_rows = row_ptr.shape[0] - 1
    if n_rows < 0:
        raise ValueError("row_ptr must have n_rows + 1 entries")
    nc = n_rows if n_cols is None else int(n_cols)
    m = col_idx.shape[0]
    col_ptr = np.empty(nc + 1, dtype=np.uint64)
    row_idx = np.empty(m, dtype=np.uint64)
    vals_out = np.empty(m, dtype=np.float32) if vals is not None else None
    rc = _load().oracle_transpose64(n_rows, nc, m, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(col_ptr),
                                    _ptr(row_idx), _ptr(vals_out))
    if rc:
        raise OracleError(rc)
    return col_ptr, row_idx, vals_out


def transpose_range(row_ptr, col_idx, vals, v_lo, v_hi):
    """Destinations [v_lo, v_hi) only: (col_ptr[v_lo..v_hi], rows, vals) with
    global offsets.  A first call of the C routine gives the sizes, a second
    one the lists.  The C call releases the GIL (ctypes), so ranges may run in
    parallel threads; the arrays must not change meanwhile."""
    n, row_ptr, col_idx, vals = _inputs(row_ptr, col_idx, vals)
    m = col_idx.shape[0]
    lib = _load()
    col_ptr = np.empty(v_hi - v_lo + 1, dtype=np.uint64)
    rc = lib.oracle_transpose_range(n, m, _ptr(row_ptr), _ptr(col_idx), None, v_lo, v_hi, _ptr(col_ptr),
                                    None, None)
    if rc:
        raise OracleError(rc)
    cnt = int(col_ptr[-1] - col_ptr[0])
    rows = np.empty(max(cnt, 1), dtype=np.uint32)
    vo = np.empty(max(cnt, 1), dtype=np.float32) if vals is not None else None
    rc = lib.oracle_transpose_range(n, m, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), v_lo, v_hi,
                                    _ptr(col_ptr), _ptr(rows), _ptr(vo))
    if rc:
        raise OracleError(rc)
    return col_ptr, rows[:cnt], (vo[:cnt] if vo is not None else None)


def columns(row_ptr, col_idx, vals, cols, n_cols=None):
    """Sampled columns: (col_start u64[k], deg u64[k], rows concat u32, vals concat f32|None)."""
    n, row_ptr, col_idx, vals = _inputs(row_ptr, col_idx, vals)
    nc = _cols(n, n_cols)
    m = col_idx.shape[0]
    cols = np.ascontiguousarray(np.unique(np.asarray(cols, dtype=np.uint32)))
    k = cols.shape[0]
    start = np.empty(k, dtype=np.uint64)
    deg = np.empty(k, dtype=np.uint64)
    lib = _load()
    rc = lib.oracle_columns_rect(n, nc, m, _ptr(row_ptr), _ptr(col_idx), None, _ptr(cols), k,
                                 _ptr(start), _ptr(deg), None, None, 0)
    if rc:
        raise OracleError(rc)
    cap = int(deg.sum())
    rows = np.empty(max(cap, 1), dtype=np.uint32)
    vo = np.empty(max(cap, 1), dtype=np.float32) if vals is not None else None
    rc = lib.oracle_columns_rect(n, nc, m, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(cols), k,
                                 _ptr(start), _ptr(deg), _ptr(rows), _ptr(vo), cap)
    if rc:
        raise OracleError(rc)
    return cols, start, deg, rows[:cap], (vo[:cap] if vo is not None else None)


def timed_transpose(row_ptr, col_idx, vals=None, n_cols=None):
    """Run ``transpose`` once and return (outputs, wall seconds)."""
    t0 = time.perf_counter()
    out = transpose(row_ptr, col_idx, vals, n_cols)
    return out, time.perf_counter() - t0
