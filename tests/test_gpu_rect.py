"""GPU parity for rectangular sparse matrices (n_rows x n_cols), bit-exact
against the oracle through the C ABI: every method and configuration, the
batch path with mixed shapes, the host paths, sub-shapes on one plan, the
search and the error reports.  Rows and columns are counted separately
everywhere (row_ptr has n_rows + 1 entries, col_ptr n_cols + 1), so the
shapes below are chosen far from square in both directions."""
import numpy as np
import pytest

import oracle
from oracle import selector as so
from paper_2501_06872_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _dev(row_ptr, col_idx, vals):
    d = torch.device("cuda:0")
    rp = torch.from_numpy(np.ascontiguousarray(row_ptr).view(np.int64)).to(d)
    ci = torch.from_numpy(np.ascontiguousarray(col_idx, dtype=np.uint32).view(np.int32)).to(d)
    vv = None if vals is None else torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float32)).to(d)
    return rp, ci, vv


def config(**kw):
    from paper_2501_06872_gb300 import binding
    base = dict(hdv_k=0, table_log2=0, block_threads=256, ctas_per_sm=4, warp_edges=256, stage_edges=0,
                sample_permille=10, flags=1, method=0, radix_tile=0, seed=7)
    base.update(kw)
    if base["hdv_k"] and not base["table_log2"]:
        base["table_log2"] = max(1, (2 * base["hdv_k"] - 1).bit_length())
    return binding.Config.from_dict(base)


CONFIGS = {
    "atomic": dict(hdv_k=0),
    "hdv64": dict(hdv_k=64, warp_edges=128),
    "hdv512_staged": dict(hdv_k=512, stage_edges=256, warp_edges=512),
    "noagg_staged": dict(hdv_k=16, flags=0, stage_edges=128),
    "big_blocks": dict(hdv_k=128, block_threads=1024, ctas_per_sm=1, warp_edges=64),
    "radix": dict(method=1),
    "radix4096": dict(method=1, radix_tile=4096, ctas_per_sm=3),
    "radix2048": dict(method=1, radix_tile=2048, ctas_per_sm=6),
    "part_hdv64": dict(hdv_k=64, warp_edges=128, partition_bits=6),
}


def gpu_rect(row_ptr, col_idx, vals, n_cols, cfg=None, check=True):
    from paper_2501_06872_gb300 import binding
    rp, ci, vv = _dev(row_ptr, col_idx, vals)
    out = binding.transpose(rp, ci, vv, config=cfg, check=check, n_cols=n_cols)
    torch.cuda.synchronize()
    return (out[0].cpu().numpy().view(np.uint64), out[1].cpu().numpy().view(np.uint32),
            None if out[2] is None else out[2].cpu().numpy())


def assert_same(got, exp):
    assert got[0].shape == exp[0].shape, "col_ptr length differs"
    assert np.array_equal(got[0], exp[0]), "col_ptr differs"
    if not np.array_equal(got[1], exp[1]):
        bad = np.nonzero(got[1] != exp[1])[0]
        raise AssertionError(f"row_idx differs at {bad.size} slots, first {bad[:8]}")
    if exp[2] is not None:
        assert np.array_equal(got[2].view(np.uint32), exp[2].view(np.uint32)), "vals differ"


SHAPES = {  # (rows, cols, entries)
    "tall": (60000, 300, 250000),
    "wide": (300, 60000, 250000),
}


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("shape", sorted(SHAPES))
def test_rect_all_configs(name, shape):
    nr, nc, m = SHAPES[shape]
    _, rp, ci, vv = inputs.random_csr(nr, m, seed=nr % 97 + 3, weighted=True, hot=9, hot_frac=0.3, n_cols=nc)
    cfg = config(**CONFIGS[name])
    assert_same(gpu_rect(rp, ci, vv, nc, cfg), oracle.transpose(rp, ci, vv, n_cols=nc))
    assert_same(gpu_rect(rp, ci, None, nc, cfg), oracle.transpose(rp, ci, None, n_cols=nc))


@pytest.mark.parametrize("nr,nc,m", [(1 << 20, 17, 1 << 20), (17, 1 << 20, 1 << 20), (1, 5000, 30000),
                                     (5000, 1, 30000), (3, 2, 7)])
def test_rect_extreme_shapes(nr, nc, m):
    _, rp, ci, vv = inputs.random_csr(nr, m, seed=11, weighted=True, n_cols=nc)
    exp = oracle.transpose(rp, ci, vv, n_cols=nc)
    for name in ["atomic", "hdv64", "radix", "radix2048"]:
        assert_same(gpu_rect(rp, ci, vv, nc, config(**CONFIGS[name])), exp)
    assert_same(gpu_rect(rp, ci, vv, nc), exp)  # default configuration


@pytest.mark.parametrize("order", ["natural", "random", "degree"])
@pytest.mark.parametrize("rs,cs", [(6, 0), (0, 6), (3, 9)])
def test_rect_folded_rmat(order, rs, cs):
    n, rp0, ci0, vv = inputs.rmat_csr(16, 16, seed=4, order=order, weighted=True)
    nr, nc, rp, ci = inputs.fold_rect(rp0, ci0, rs, cs)
    exp = oracle.transpose(rp, ci, vv, n_cols=nc)
    for name in ["hdv512_staged", "big_blocks", "radix", "radix4096"]:
        assert_same(gpu_rect(rp, ci, vv, nc, config(**CONFIGS[name])), exp)
    assert_same(gpu_rect(rp, ci, vv, nc), exp)


def test_rect_involution_on_gpu():
    """A^T^T = A with the shapes swapped (rows sorted, so the CSR is the CSC of its CSC)."""
    n, rp0, ci0, vv0 = inputs.rmat_csr(14, 8, seed=8, order="random", weighted=True, sorted_rows=True)
    nr, nc, rp, ci = inputs.fold_rect(rp0, ci0, 4, 0)
    src = np.repeat(np.arange(nr), np.diff(rp.astype(np.int64)))
    o = np.lexsort((ci, src))
    ci, vv = ci[o], vv0[o]
    for name in ["atomic", "radix"]:
        t = gpu_rect(rp, ci, vv, nc, config(**CONFIGS[name]))
        tt = gpu_rect(t[0], t[1], t[2], nr, config(**CONFIGS[name]))
        assert_same(tt, (rp, ci, vv))


@pytest.mark.parametrize("name", ["atomic", "hdv64", "radix", "radix4096"])
def test_rect_errors_are_reported(name):
    from paper_2501_06872_gb300 import binding
    cfg = config(**CONFIGS[name])
    # tall 6 x 2: an index < n_rows but >= n_cols is out of range
    with pytest.raises(binding.GtError) as ei:
        gpu_rect(np.array([0, 1, 2, 2, 2, 2, 3], np.uint64), np.array([0, 1, 4], np.uint32), None, 2, cfg)
    assert ei.value.code == 2
    # tall: row_ptr decreases at a row index beyond the column count
    n_rows, n_cols = 20000, 3
    rp = np.arange(n_rows + 1, dtype=np.uint64)
    rp[15000] = 14990  # rp[14999] = 14999 > rp[15000]
    with pytest.raises(binding.GtError) as ei:
        gpu_rect(rp, np.zeros(n_rows, np.uint32), None, n_cols, cfg)
    assert ei.value.code == 3
    # row_ptr[n_rows] != m
    with pytest.raises(binding.GtError) as ei:
        gpu_rect(np.array([0, 1, 1], np.uint64), np.array([0, 5], np.uint32), None, 9, cfg)
    assert ei.value.code == 3
    # a wide matrix accepts an index above n_rows
    got = gpu_rect(np.array([0, 1], np.uint64), np.array([8], np.uint32), None, 9, cfg)
    assert list(got[0]) == [0] * 9 + [1]


def test_rect_zero_rows_or_columns():
    from paper_2501_06872_gb300 import binding
    got = gpu_rect(np.zeros(1, np.uint64), np.zeros(0, np.uint32), None, 5)  # 0 x 5
    assert np.array_equal(got[0], np.zeros(6, np.uint64))
    got = gpu_rect(np.zeros(4, np.uint64), np.zeros(0, np.uint32), None, 0)  # 3 x 0
    assert np.array_equal(got[0], np.zeros(1, np.uint64))
    with pytest.raises(binding.GtError) as ei:
        binding.Plan(0, 5, False, n_cols=4)
    assert ei.value.code == 1


@pytest.mark.parametrize("name", ["atomic", "hdv64", "hdv512_staged"])
def test_rect_unsorted_mode_multisets(name):
    from paper_2501_06872_gb300 import binding
    nr, nc, m = 40000, 700, 200000
    _, rp, ci, vv = inputs.random_csr(nr, m, seed=5, weighted=True, hot=5, hot_frac=0.5, n_cols=nc)
    exp = oracle.transpose(rp, ci, vv, n_cols=nc)
    c = dict(CONFIGS[name])
    c["flags"] = c.get("flags", 1) | binding.FLAG_UNSORTED
    got = gpu_rect(rp, ci, vv, nc, config(**c))
    assert np.array_equal(got[0], exp[0])

    def ms(cp, ri, vo):
        cols = np.repeat(np.arange(nc, dtype=np.int64), np.diff(cp.astype(np.int64)))
        o = np.lexsort((vo.view(np.uint32), ri, cols))
        return cols[o], ri[o], vo.view(np.uint32)[o]
    for x, y in zip(ms(*got), ms(*exp)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("name", ["hdv64", "radix"])
def test_rect_sub_shapes_on_one_plan(name):
    """One plan (the largest rows, columns and entries) serves smaller shapes of both orientations."""
    from paper_2501_06872_gb300 import binding
    plan = binding.Plan(50000, 400000, True, config(**CONFIGS[name]), n_cols=50000)
    assert plan.shape() == (50000, 50000, 400000)
    for nr, nc, m in [(50000, 37, 400000), (37, 50000, 300000), (1000, 1000, 5000), (50000, 50000, 0)]:
        _, rp, ci, vv = inputs.random_csr(nr, m, seed=nr + nc, weighted=m > 0, n_cols=nc)
        d_rp, d_ci, d_vv = _dev(rp, ci, vv)
        cp = torch.full((nc + 1,), -1, dtype=torch.int64, device="cuda")
        ri = torch.full((max(m, 1),), -1, dtype=torch.int32, device="cuda")
        vo = torch.full((m,), -1.0, dtype=torch.float32, device="cuda") if m else None
        plan.transpose_sub(nr, m, d_rp, d_ci, d_vv, cp, ri, vo, n_cols=nc)
        plan.check()
        exp = oracle.transpose(rp, ci, vv, n_cols=nc)
        assert_same((cp.cpu().numpy().view(np.uint64), ri.cpu().numpy().view(np.uint32)[:m],
                     None if vo is None else vo.cpu().numpy()), exp)
    with pytest.raises(binding.GtError):  # more columns than the plan holds
        plan.transpose_sub(10, 5, d_rp, d_ci, d_vv, cp, ri, vo, n_cols=50001)
    plan.close()


def test_rect_host_paths():
    from paper_2501_06872_gb300 import binding
    nr, nc, m = 70000, 900, 300000
    _, rp, ci, vv = inputs.random_csr(nr, m, seed=12, weighted=True, n_cols=nc)
    exp = oracle.transpose(rp, ci, vv, n_cols=nc)
    for name in ["hdv64", "radix"]:
        plan = binding.Plan(nr, m, True, config(**CONFIGS[name]), n_cols=nc)
        cp = np.empty(nc + 1, np.uint64)
        ri = np.empty(m, np.uint32)
        vo = np.empty(m, np.float32)
        plan.transpose_host(rp, ci, vv, cp, ri, vo)
        assert_same((cp, ri, vo), exp)
        h = [torch.from_numpy(x).pin_memory() for x in (rp.view(np.int64), ci.view(np.int32), vv)]
        outs = (torch.empty(nc + 1, dtype=torch.int64).pin_memory(), torch.empty(m, dtype=torch.int32).pin_memory(),
                torch.empty(m, dtype=torch.float32).pin_memory())
        plan.transpose_host_async(*h, *outs)
        plan.host_wait()
        assert_same((outs[0].numpy().view(np.uint64), outs[1].numpy().view(np.uint32), outs[2].numpy()), exp)
        plan.close()


def test_rect_batch_mixed_shapes():
    """Square graphs, tall and wide matrices in one batch plan (two sub-batches
    forced by a small edge cap are covered by the square tests)."""
    from paper_2501_06872_gb300 import binding
    shapes = [(5000, 5000, 40000), (20000, 33, 60000), (33, 20000, 60000), (1, 3000, 4000), (3000, 1, 4000),
              (777, 0, 9000)]  # n_cols = 0: square
    graphs, keep, exps = [], [], []
    for i, (nr, nc, m) in enumerate(shapes):
        ncols = nc if nc else nr
        _, rp, ci, vv = inputs.random_csr(nr, m, seed=40 + i, weighted=True, hot=3, hot_frac=0.2, n_cols=ncols)
        d_rp, d_ci, d_vv = _dev(rp, ci, vv)
        cp = torch.full((ncols + 1,), -1, dtype=torch.int64, device="cuda")
        ri = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        vo = torch.full((m,), -1.0, dtype=torch.float32, device="cuda")
        keep.append((d_rp, d_ci, d_vv, cp, ri, vo))
        graphs.append(dict(n=nr, n_cols=nc, m=m, row_ptr=d_rp, col_idx=d_ci, vals=d_vv, col_ptr=cp, row_idx=ri,
                           vals_out=vo))
        exps.append(oracle.transpose(rp, ci, vv, n_cols=ncols))
    plan = binding.BatchPlan(graphs, True)
    plan.transpose()
    plan.check()
    plan.close()
    for (d_rp, d_ci, d_vv, cp, ri, vo), exp in zip(keep, exps):
        assert_same((cp.cpu().numpy().view(np.uint64), ri.cpu().numpy().view(np.uint32), vo.cpu().numpy()), exp)


def test_rect_batch_many_sub_batches(monkeypatch):
    """Tall and wide matrices split over several sub-batches (small edge cap)."""
    from paper_2501_06872_gb300 import binding
    monkeypatch.setenv("GT_BATCH_MAX_EDGES", "30000")
    graphs, keep, exps = [], [], []
    for i in range(10):
        nr, nc = (3000, 17) if i % 2 else (17, 3000)
        m = 9000 + 500 * i
        _, rp, ci, vv = inputs.random_csr(nr, m, seed=60 + i, weighted=True, n_cols=nc)
        d_rp, d_ci, d_vv = _dev(rp, ci, vv)
        cp = torch.full((nc + 1,), -1, dtype=torch.int64, device="cuda")
        ri = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        vo = torch.full((m,), -1.0, dtype=torch.float32, device="cuda")
        keep.append((d_rp, d_ci, d_vv, cp, ri, vo))
        graphs.append(dict(n=nr, n_cols=nc, m=m, row_ptr=d_rp, col_idx=d_ci, vals=d_vv, col_ptr=cp, row_idx=ri,
                           vals_out=vo))
        exps.append(oracle.transpose(rp, ci, vv, n_cols=nc))
    plan = binding.BatchPlan(graphs, True)
    plan.transpose()
    plan.check()
    assert plan.info()["sub_batches"] > 3
    plan.close()
    for (d_rp, d_ci, d_vv, cp, ri, vo), exp in zip(keep, exps):
        assert_same((cp.cpu().numpy().view(np.uint64), ri.cpu().numpy().view(np.uint32), vo.cpu().numpy()), exp)


def test_rect_batch_reports_column_out_of_range():
    from paper_2501_06872_gb300 import binding
    _, rp, ci, vv = inputs.random_csr(5000, 20000, seed=3, weighted=False, n_cols=40)
    ci = ci.copy()
    ci[777] = 40  # < n_rows, == n_cols
    d_rp, d_ci, _ = _dev(rp, ci, None)
    cp = torch.empty(41, dtype=torch.int64, device="cuda")
    ri = torch.empty(20000, dtype=torch.int32, device="cuda")
    plan = binding.BatchPlan([dict(n=5000, n_cols=40, m=20000, row_ptr=d_rp, col_idx=d_ci, col_ptr=cp,
                                   row_idx=ri)], False)
    plan.transpose()
    assert plan.status() == 2
    plan.close()


@pytest.mark.parametrize("rs,cs", [(5, 0), (0, 5)])
def test_rect_features_match_oracle(rs, cs):
    from paper_2501_06872_gb300 import binding
    n, rp0, ci0, _ = inputs.rmat_csr(15, 8, seed=17, order="random")
    nr, nc, rp, ci = inputs.fold_rect(rp0, ci0, rs, cs)
    d_rp, d_ci, _ = _dev(rp, ci, None)
    got = binding.graph_features(d_rp, d_ci, False, seed=99, n_cols=nc).cpu().numpy()
    exp = so.features(nr, len(ci), rp.astype(np.int64), ci.astype(np.int64), False, 99, n_cols=nc)
    np.testing.assert_allclose(got, exp, rtol=2e-6, atol=1e-7)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_rect_tune_keeps_bytes(mode):
    from paper_2501_06872_gb300 import binding
    n, rp0, ci0, vv = inputs.rmat_csr(15, 12, seed=19, order="degree", weighted=True)
    nr, nc, rp, ci = inputs.fold_rect(rp0, ci0, 0, 4)
    exp = oracle.transpose(rp, ci, vv, n_cols=nc)
    d_rp, d_ci, d_vv = _dev(rp, ci, vv)
    m = len(ci)
    plan = binding.Plan(nr, m, True, n_cols=nc)
    cp = torch.empty(nc + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(m, dtype=torch.int32, device="cuda")
    vo = torch.empty(m, dtype=torch.float32, device="cuda")
    sel = binding.Selector.pretrained() if mode == 2 else None
    chosen, table = plan.tune(mode, d_rp, d_ci, d_vv, cp, ri, vo, selector=sel)
    assert 0 <= chosen < binding.TUNE_GRID
    if mode == 1:
        assert all(t["status"] == 0 for t in table)
    plan.transpose(d_rp, d_ci, d_vv, cp, ri, vo)
    plan.check()
    assert_same((cp.cpu().numpy().view(np.uint64), ri.cpu().numpy().view(np.uint32), vo.cpu().numpy()), exp)
    plan.close()
    if sel is not None:
        sel.close()
