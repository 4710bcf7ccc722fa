"""Pins for the oracle against what the paper and the mathematics fix (CPU only).

* Fig. 1 (Sec. II-A): the offsets/edges values stated in the text.
* The definition (Sec. II-A): CSC lists = CSR edges stably sorted by
  destination -> brute force by lexicographic sort, exhaustively on tiny graphs.
* Involution (Sec. II-A: the transpose of the transpose is the original).
* Degree preservation and offsets semantics (Algorithm 1 Steps 1-2).
* Undirected graphs have identical CSR and CSC (Sec. II-A).
* Weights ride along unchanged (Sec. II-A).
* Rectangular n_rows x n_cols matrices: the same definition with n_cols + 1
  offsets, pinned by brute force (exhaustively on tiny shapes), by scipy's
  CSR -> CSC conversion (a library routine), by the involution with the
  shapes swapped, and by the range check against n_cols, not n_rows.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2501_06872_gb300 import inputs
from tests._graphs import all_tiny_graphs, all_tiny_rect, brute_transpose, csr_from_rows

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_pins.txt")


def _read_golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *vs = line.split()
            out[k] = [int(x) for x in vs]
    return out


def test_fig1_pins():
    g = _read_golden()
    n = g["reconstruction_n"][0]
    ed = g["reconstruction_edges"]
    rows = [[] for _ in range(n)]
    for i in range(0, len(ed), 2):
        rows[ed[i]].append(ed[i + 1])
    row_ptr, col_idx = csr_from_rows(n, rows)
    # the reconstruction agrees with the CSR values stated in the text
    assert list(row_ptr[:2]) == g["csr_offsets_prefix"]
    assert list(col_idx[row_ptr[0]:row_ptr[1]]) == g["csr_vertex0_out"]
    col_ptr, row_idx, _ = oracle.transpose(row_ptr, col_idx)
    assert list(col_ptr[:2]) == g["csc_offsets_prefix"]
    assert list(row_idx[:1]) == g["csc_edges_prefix"]


def test_exhaustive_tiny_vs_definition():
    count = 0
    for n, rows in all_tiny_graphs(3, 4):
        row_ptr, col_idx = csr_from_rows(n, rows)
        m = col_idx.shape[0]
        vals = np.arange(m, dtype=np.float32) + 0.5  # distinct: exposes the duplicate order
        got = oracle.transpose(row_ptr, col_idx, vals)
        exp = brute_transpose(row_ptr, col_idx, vals)
        assert np.array_equal(got[0], exp[0])
        assert np.array_equal(got[1], exp[1])
        assert np.array_equal(got[2], exp[2])
        count += 1
    assert count == 1683  # every CSR with n <= 3 and m <= 4


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("n,m", [(1, 5), (7, 0), (17, 200), (300, 5000), (1000, 777)])
def test_random_vs_definition(seed, n, m):
    n, row_ptr, col_idx, vals = inputs.random_csr(n, m, seed=seed, hot=3, hot_frac=0.3)
    got = oracle.transpose(row_ptr, col_idx, vals)
    exp = brute_transpose(row_ptr, col_idx, vals)
    for a, b in zip(got, exp):
        assert np.array_equal(a, b)


def test_rmat_small_vs_definition():
    n, row_ptr, col_idx, vals = inputs.rmat_csr(10, 8, seed=5, weighted=True)
    got = oracle.transpose(row_ptr, col_idx, vals)
    exp = brute_transpose(row_ptr, col_idx, vals)
    for a, b in zip(got, exp):
        assert np.array_equal(a, b)


def test_invariants_degrees_offsets():
    n, row_ptr, col_idx, vals = inputs.rmat_csr(11, 16, seed=9, order="random", weighted=True)
    col_ptr, row_idx, vo = oracle.transpose(row_ptr, col_idx, vals)
    m = col_idx.shape[0]
    assert col_ptr[0] == 0 and col_ptr[-1] == m
    assert np.all(np.diff(col_ptr.astype(np.int64)) >= 0)
    # in-degree of CSR = out-degree of CSC; out-degree of CSR = in-degree of CSC
    assert np.array_equal(np.diff(col_ptr.astype(np.int64)), np.bincount(col_idx, minlength=n))
    assert np.array_equal(np.bincount(row_idx, minlength=n), np.diff(row_ptr.astype(np.int64)))
    # the multiset of (u, v, w) triples is preserved
    src = np.repeat(np.arange(n), np.diff(row_ptr.astype(np.int64)))
    dst_t = np.repeat(np.arange(n), np.diff(col_ptr.astype(np.int64)))
    a = np.lexsort((vals.view(np.uint32), col_idx, src))
    b = np.lexsort((vo.view(np.uint32), dst_t, row_idx))
    assert np.array_equal(src[a], row_idx[b])
    assert np.array_equal(col_idx[a], dst_t[b])
    assert np.array_equal(vals[a].view(np.uint32), vo[b].view(np.uint32))
    # every list ascending in source
    for v in range(0, n, 37):
        seg = row_idx[col_ptr[v]:col_ptr[v + 1]]
        assert np.all(np.diff(seg.astype(np.int64)) >= 0)


def test_involution_sorted_rows():
    n, row_ptr, col_idx, vals = inputs.rmat_csr(9, 8, seed=3, weighted=True, sorted_rows=True)
    c1 = oracle.transpose(row_ptr, col_idx, vals)
    c2 = oracle.transpose(c1[0], c1[1], c1[2])
    assert np.array_equal(c2[0], row_ptr)
    assert np.array_equal(c2[1], col_idx)
    assert np.array_equal(c2[2].view(np.uint32), vals.view(np.uint32))


def test_involution_unsorted_rows_up_to_row_order():
    n, row_ptr, col_idx, _ = inputs.rmat_csr(9, 8, seed=4)
    c1 = oracle.transpose(row_ptr, col_idx)
    c2 = oracle.transpose(c1[0], c1[1])
    assert np.array_equal(c2[0], row_ptr)
    for u in range(n):
        a, b = int(row_ptr[u]), int(row_ptr[u + 1])
        assert np.array_equal(np.sort(c2[1][a:b]), np.sort(col_idx[a:b]))


def test_undirected_graph_is_its_own_transpose():
    src, dst = inputs.er_edges(200, 1500, seed=2)
    s2 = np.concatenate([src, dst])
    d2 = np.concatenate([dst, src])
    o = np.lexsort((d2, s2))
    row_ptr, col_idx, _ = inputs.csr_from_edges(200, s2[o], d2[o])
    col_ptr, row_idx, _ = oracle.transpose(row_ptr, col_idx)
    assert np.array_equal(col_ptr, row_ptr)
    assert np.array_equal(row_idx, col_idx)


def test_degenerate_cases():
    # no edges
    col_ptr, row_idx, _ = oracle.transpose(np.zeros(6, np.uint64), np.zeros(0, np.uint32))
    assert np.array_equal(col_ptr, np.zeros(6, np.uint64)) and row_idx.size == 0
    # one vertex with self-loops, weights kept in CSR order
    col_ptr, row_idx, vo = oracle.transpose(np.array([0, 3], np.uint64), np.zeros(3, np.uint32),
                                            np.array([3.0, 1.0, 2.0], np.float32))
    assert list(col_ptr) == [0, 3] and list(row_idx) == [0, 0, 0] and list(vo) == [3.0, 1.0, 2.0]
    # all edges into the last vertex
    n = 50
    row_ptr = np.arange(n + 1, dtype=np.uint64)
    col_idx = np.full(n, n - 1, np.uint32)
    col_ptr, row_idx, _ = oracle.transpose(row_ptr, col_idx)
    assert col_ptr[n - 1] == 0 and col_ptr[n] == n and np.array_equal(row_idx, np.arange(n))


def test_errors():
    with pytest.raises(oracle.OracleError) as ei:
        oracle.transpose(np.array([0, 1], np.uint64), np.array([1], np.uint32))
    assert ei.value.code == 2
    with pytest.raises(oracle.OracleError) as ei:
        oracle.transpose(np.array([0, 2, 1], np.uint64), np.array([0], np.uint32))
    assert ei.value.code == 3


def test_range_chunks_reassemble_full():
    n, row_ptr, col_idx, vals = inputs.rmat_csr(10, 16, seed=8, order="random", weighted=True)
    full = oracle.transpose(row_ptr, col_idx, vals)
    cuts = [0, 1, 100, 513, 900, n]
    rows, vs = [], []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        cp, r, v = oracle.transpose_range(row_ptr, col_idx, vals, lo, hi)
        assert np.array_equal(cp, full[0][lo:hi + 1])
        rows.append(r)
        vs.append(v)
    assert np.array_equal(np.concatenate(rows), full[1])
    assert np.array_equal(np.concatenate(vs), full[2])


def test_sampled_columns_match_full():
    n, row_ptr, col_idx, vals = inputs.rmat_csr(10, 16, seed=6, order="degree", weighted=True)
    full = oracle.transpose(row_ptr, col_idx, vals)
    cols = np.array([0, 1, 2, 17, 400, 1023], dtype=np.uint32)
    c, start, deg, rows, vo = oracle.columns(row_ptr, col_idx, vals, cols)
    off = 0
    for i, v in enumerate(c):
        assert start[i] == full[0][v]
        assert deg[i] == full[0][v + 1] - full[0][v]
        d = int(deg[i])
        assert np.array_equal(rows[off:off + d], full[1][full[0][v]:full[0][v + 1]])
        assert np.array_equal(vo[off:off + d], full[2][full[0][v]:full[0][v + 1]])
        off += d


def test_brute_force_detects_planted_mistakes():
    """The pins must fail on plausible mistakes: here they are planted in a copy
    of the oracle's output (dropped edge, swapped order, off-by-one offset)."""
    n, row_ptr, col_idx, vals = inputs.random_csr(40, 300, seed=11)
    good = oracle.transpose(row_ptr, col_idx, vals)
    exp = brute_transpose(row_ptr, col_idx, vals)
    assert all(np.array_equal(a, b) for a, b in zip(good, exp))
    bad_ptr = good[0].copy()
    bad_ptr[5] += 1
    assert not np.array_equal(bad_ptr, exp[0])
    bad_rows = good[1].copy()
    j = int(np.argmax(np.diff(bad_rows.astype(np.int64)) > 0))
    bad_rows[j], bad_rows[j + 1] = bad_rows[j + 1], bad_rows[j]
    assert not np.array_equal(bad_rows, exp[1])


# ---- rectangular matrices ------------------------------------------------------

def test_rect_exhaustive_tiny_vs_definition():
    count = 0
    for nr, nc, rows in all_tiny_rect(3, 3, 3):
        row_ptr, col_idx = csr_from_rows(nr, rows)
        m = col_idx.shape[0]
        vals = np.arange(m, dtype=np.float32) + 0.25
        got = oracle.transpose(row_ptr, col_idx, vals, n_cols=nc)
        exp = brute_transpose(row_ptr, col_idx, vals, n_cols=nc)
        assert got[0].shape == (nc + 1,)
        for a, b in zip(got, exp):
            assert np.array_equal(a, b)
        count += 1
    # per shape: C(m + r - 1, r - 1) ways to split m entries over r rows, c^m destination sequences
    assert count == sum(math.comb(m + r - 1, r - 1) * c ** m for r in range(1, 4) for c in range(1, 4) if r != c
                        for m in range(4)) == 338


@pytest.mark.parametrize("nr,nc,m", [(1, 50, 200), (50, 1, 200), (300, 7, 4000), (7, 300, 4000),
                                     (1000, 3, 777), (3, 1000, 777)])
def test_rect_random_vs_definition(nr, nc, m):
    n, row_ptr, col_idx, vals = inputs.random_csr(nr, m, seed=nr + nc, hot=2, hot_frac=0.3, n_cols=nc)
    assert int(col_idx.max()) < nc
    got = oracle.transpose(row_ptr, col_idx, vals, n_cols=nc)
    exp = brute_transpose(row_ptr, col_idx, vals, n_cols=nc)
    for a, b in zip(got, exp):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("rs,cs", [(0, 3), (3, 0), (2, 5)])
def test_rect_matches_scipy(rs, cs):
    sp = pytest.importorskip("scipy.sparse")
    n, row_ptr, col_idx, vals = inputs.rmat_csr(10, 8, seed=21, order="random", weighted=True)
    nr, nc, rp, ci = inputs.fold_rect(row_ptr, col_idx, rs, cs)
    a = sp.csr_matrix((vals, ci.astype(np.int64), rp.astype(np.int64)), shape=(nr, nc))
    t = a.tocsc()  # scipy's conversion: a stable counting sort by column, duplicates kept
    cp, ri, vo = oracle.transpose(rp, ci, vals, n_cols=nc)
    assert np.array_equal(cp.astype(np.int64), t.indptr.astype(np.int64))
    assert np.array_equal(ri.astype(np.int64), t.indices.astype(np.int64))
    assert np.array_equal(vo.view(np.uint32), np.asarray(t.data, dtype=np.float32).view(np.uint32))


def test_rect_involution_swaps_shape():
    n, row_ptr, col_idx, vals = inputs.rmat_csr(9, 8, seed=13, weighted=True, sorted_rows=True)
    nr, nc, rp, ci = inputs.fold_rect(row_ptr, col_idx, 3, 0)  # 64 x 512; merged rows stay sorted per source
    o = np.lexsort((ci, np.repeat(np.arange(nr), np.diff(rp.astype(np.int64)))))
    ci, vals = ci[o], vals[o]
    c1 = oracle.transpose(rp, ci, vals, n_cols=nc)
    assert c1[0].shape == (nc + 1,) and int(c1[1].max()) < nr
    c2 = oracle.transpose(c1[0], c1[1], c1[2], n_cols=nr)
    assert np.array_equal(c2[0], rp)
    assert np.array_equal(c2[1], ci)
    assert np.array_equal(c2[2].view(np.uint32), vals.view(np.uint32))


def test_rect_degenerate_and_errors():
    # one row: every column holds that row once per entry, values in CSR order
    cp, ri, vo = oracle.transpose(np.array([0, 4], np.uint64), np.array([2, 0, 2, 5], np.uint32),
                                  np.array([1.0, 2.0, 3.0, 4.0], np.float32), n_cols=6)
    assert list(cp) == [0, 1, 1, 3, 3, 3, 4] and list(ri) == [0, 0, 0, 0] and list(vo) == [2.0, 1.0, 3.0, 4.0]
    # one column: the rows of the entries in CSR order
    cp, ri, _ = oracle.transpose(np.array([0, 2, 2, 3], np.uint64), np.zeros(3, np.uint32), n_cols=1)
    assert list(cp) == [0, 3] and list(ri) == [0, 0, 2]
    # zero columns and no entries
    cp, ri, _ = oracle.transpose(np.zeros(4, np.uint64), np.zeros(0, np.uint32), n_cols=0)
    assert list(cp) == [0] and ri.size == 0
    # a tall matrix: a column index below n_rows but not below n_cols is out of range
    with pytest.raises(oracle.OracleError) as ei:
        oracle.transpose(np.array([0, 1, 1, 1], np.uint64), np.array([1], np.uint32), n_cols=1)
    assert ei.value.code == 2
    # a wide matrix: a column index above n_rows is fine
    cp, ri, _ = oracle.transpose(np.array([0, 1], np.uint64), np.array([9], np.uint32), n_cols=10)
    assert cp[9] == 0 and cp[10] == 1


def test_rect_sampled_columns_match_full():
    n, row_ptr, col_idx, vals = inputs.rmat_csr(10, 16, seed=6, order="degree", weighted=True)
    nr, nc, rp, ci = inputs.fold_rect(row_ptr, col_idx, 4, 1)
    full = oracle.transpose(rp, ci, vals, n_cols=nc)
    cols = np.array([0, 3, 100, nc - 1], dtype=np.uint32)
    c, start, deg, rows, vo = oracle.columns(rp, ci, vals, cols, n_cols=nc)
    off = 0
    for i, v in enumerate(c):
        assert start[i] == full[0][v] and deg[i] == full[0][v + 1] - full[0][v]
        d = int(deg[i])
        assert np.array_equal(rows[off:off + d], full[1][full[0][v]:full[0][v + 1]])
        off += d


def test_property_random_shapes_vs_definition():
    """Arbitrary small CSR matrices (any shape, duplicates, empty rows and
    columns, weighted or not) against the brute-force definition."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=300, deadline=None, derandomize=True)
    @hyp.given(st.integers(1, 12), st.integers(1, 12), st.data(), st.booleans())
    def check(nr, nc, data, weighted):
        rows = [data.draw(st.lists(st.integers(0, nc - 1), max_size=6)) for _ in range(nr)]
        row_ptr, col_idx = csr_from_rows(nr, rows)
        vals = (np.arange(col_idx.size, dtype=np.float32) * 0.5 - 3.0) if weighted else None
        got = oracle.transpose(row_ptr, col_idx, vals, n_cols=nc)
        exp = brute_transpose(row_ptr, col_idx, vals, n_cols=nc)
        assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
        if weighted:
            assert np.array_equal(got[2].view(np.uint32), exp[2].view(np.uint32))

    check()


def test_oracle64_matches_brute_force_and_the_32_bit_oracle():
    """The 64-bit-ID routine against the definition (lexicographic sort of the
    (v, u, e) triples) on random rectangular matrices with duplicates and
    values, and against the 32-bit routine where IDs fit 32 bits."""
    from tests._graphs import brute_transpose
    rng = np.random.default_rng(64)
    for trial in range(40):
        nr, nc = int(rng.integers(1, 60)), int(rng.integers(1, 60))
        deg = rng.integers(0, 6, nr)
        rp = np.zeros(nr + 1, np.uint64)
        np.cumsum(deg, out=rp[1:])
        m = int(rp[-1])
        ci = rng.integers(0, nc, m).astype(np.uint64)
        vv = rng.standard_normal(m).astype(np.float32)
        got = oracle.transpose64(rp, ci, vv, n_cols=nc)
        exp = brute_transpose(rp, ci, vv, n_cols=nc)
        assert np.array_equal(got[0], exp[0])
        assert np.array_equal(got[1], exp[1].astype(np.uint64))
        assert np.array_equal(got[2].view(np.uint32), exp[2].view(np.uint32))
        o32 = oracle.transpose(rp, ci.astype(np.uint32), vv, n_cols=nc)
        assert np.array_equal(got[0], o32[0]) and np.array_equal(got[1], o32[1].astype(np.uint64))


def test_oracle64_errors_and_degenerate_shapes():
    rp = np.array([0, 2, 3], np.uint64)
    with pytest.raises(oracle.OracleError) as e:
        oracle.transpose64(rp, np.array([0, 5, 1], np.uint64), n_cols=5)  # 5 >= n_cols
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.transpose64(np.array([0, 2, 1], np.uint64), np.array([0, 1], np.uint64), n_cols=4)
    assert e.value.code == 3
    cp, ri, vo = oracle.transpose64(np.zeros(4, np.uint64), np.zeros(0, np.uint64), n_cols=7)
    assert np.array_equal(cp, np.zeros(8, np.uint64)) and ri.size == 0 and vo is None
