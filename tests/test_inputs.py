"""Generators: determinism by seed, bijective permutations, R-MAT marginals."""
import numpy as np

from paper_2501_06872_gb300 import inputs


def test_feistel_is_bijection():
    for n in [1, 2, 3, 5, 1000, 1 << 12, 12345]:
        p = inputs.feistel_perm(n, seed=7)
        assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint64))
    assert not np.array_equal(inputs.feistel_perm(4096, 1), inputs.feistel_perm(4096, 2))


def test_deterministic_by_seed():
    a = inputs.rmat_csr(10, 8, seed=3, weighted=True)
    b = inputs.rmat_csr(10, 8, seed=3, weighted=True)
    c = inputs.rmat_csr(10, 8, seed=4, weighted=True)
    assert all(np.array_equal(x, y) for x, y in zip(a[1:], b[1:]))
    assert not np.array_equal(a[2], c[2])


def test_rmat_marginals():
    # P(source bit = 0) = a + b and P(destination bit = 0) = a + c at every level
    src, dst = inputs.rmat_edges(12, 16, seed=2)
    for bit in [0, 5, 11]:
        s0 = np.mean(((src >> bit) & 1) == 0)
        d0 = np.mean(((dst >> bit) & 1) == 0)
        assert abs(s0 - 0.76) < 0.01 and abs(d0 - 0.76) < 0.01


def test_degree_order_is_sorted():
    n, row_ptr, col_idx, _ = inputs.rmat_csr(10, 16, seed=1, order="degree")
    deg = np.bincount(col_idx, minlength=n)
    assert np.all(np.diff(deg) <= 0)


def test_zipf_matrix_shape():
    n, row_ptr, col_idx, vals = inputs.zipf_matrix(1500, 12.0, seed=1, idx=3)
    assert row_ptr[0] == 0 and row_ptr[-1] == col_idx.size == vals.size
    assert col_idx.max() < n and np.all(np.diff(row_ptr.astype(np.int64)) >= 1)
    assert -1.0 <= vals.min() and vals.max() < 1.0
    assert 8.0 < col_idx.size / n < 16.0


def test_fold_rect_relabels_rows_and_columns():
    n, row_ptr, col_idx, _ = inputs.rmat_csr(8, 4, seed=3)
    nr, nc, rp, ci = inputs.fold_rect(row_ptr, col_idx, 2, 5)
    assert (nr, nc) == (64, 8) and rp.shape == (65,) and ci.shape == col_idx.shape
    src = np.repeat(np.arange(n), np.diff(row_ptr.astype(np.int64)))
    src_f = np.repeat(np.arange(nr), np.diff(rp.astype(np.int64)))
    assert np.array_equal(src_f, src >> 2)  # same edge sequence, rows merged by 4
    assert np.array_equal(ci, col_idx >> 5)
