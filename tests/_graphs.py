"""Helpers shared by tests: brute-force definition of the transpose and
graph enumeration.  Nothing here is used by the CUDA path or the oracle."""
import itertools

import numpy as np


def brute_transpose(row_ptr, col_idx, vals=None, n_cols=None):
    """CSC by definition: list (v, u, e) for every edge and sort lexicographically
    (numpy lexsort), then compress the destinations into offsets (n_cols + 1
    of them; n_cols defaults to the row count)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    n = row_ptr.shape[0] - 1
    nc = n if n_cols is None else n_cols
    m = col_idx.shape[0]
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    e = np.arange(m, dtype=np.int64)
    order = np.lexsort((e, src, col_idx))  # last key is primary: (v, u, e)
    col_ptr = np.zeros(nc + 1, dtype=np.uint64)
    for v in col_idx:
        col_ptr[v + 1] += 1
    col_ptr = np.cumsum(col_ptr).astype(np.uint64)
    row_idx = src[order].astype(np.uint32)
    vo = None if vals is None else np.asarray(vals, dtype=np.float32)[order]
    return col_ptr, row_idx, vo


def csr_from_rows(n, rows):
    """rows: list of lists of destinations -> (row_ptr, col_idx)."""
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    for u, r in enumerate(rows):
        row_ptr[u + 1] = row_ptr[u] + len(r)
    col_idx = np.array([v for r in rows for v in r], dtype=np.uint32)
    return row_ptr, col_idx


def all_tiny_rect(max_rows=3, max_cols=3, max_m=3):
    """Every CSR of an n_rows x n_cols matrix with n_rows != n_cols (both <=
    the maxima) and m <= max_m entries, rows in any order, duplicates kept."""
    for nr in range(1, max_rows + 1):
        for nc in range(1, max_cols + 1):
            if nr == nc:
                continue
            pairs = [(u, v) for u in range(nr) for v in range(nc)]
            for m in range(0, max_m + 1):
                for seq in itertools.product(pairs, repeat=m):
                    if any(seq[i][0] > seq[i + 1][0] for i in range(m - 1)):
                        continue
                    rows = [[] for _ in range(nr)]
                    for u, v in seq:
                        rows[u].append(v)
                    yield nr, nc, rows


def all_tiny_graphs(max_n=3, max_m=4):
    """Every CSR with n <= max_n vertices and m <= max_m edges (rows in any
    order, duplicates and self-loops included)."""
    for n in range(1, max_n + 1):
        pairs = [(u, v) for u in range(n) for v in range(n)]
        for m in range(0, max_m + 1):
            for seq in itertools.product(pairs, repeat=m):
                if any(seq[i][0] > seq[i + 1][0] for i in range(m - 1)):
                    continue  # CSR order: sources non-decreasing
                rows = [[] for _ in range(n)]
                for u, v in seq:
                    rows[u].append(v)
                yield n, rows
