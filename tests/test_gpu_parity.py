"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit-exact.

Integer outputs (col_ptr, row_idx) and the carried f32 value bits must be
identical; every configuration must give the same bytes.
"""
import numpy as np
import pytest

import oracle
from paper_2501_06872_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _to_dev(row_ptr, col_idx, vals):
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(np.ascontiguousarray(row_ptr).view(np.int64)).to(dev)
    ci = torch.from_numpy(np.ascontiguousarray(col_idx, dtype=np.uint32).view(np.int32)).to(dev)
    vv = None if vals is None else torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float32)).to(dev)
    return rp, ci, vv


def gpu_transpose(row_ptr, col_idx, vals=None, cfg=None, check=True):
    from paper_2501_06872_gb300 import binding
    rp, ci, vv = _to_dev(row_ptr, col_idx, vals)
    out = binding.transpose(rp, ci, vv, config=cfg, check=check)
    torch.cuda.synchronize()
    cp = out[0].cpu().numpy().view(np.uint64)
    ri = out[1].cpu().numpy().view(np.uint32)
    vo = None if out[2] is None else out[2].cpu().numpy()
    return cp, ri, vo


def assert_same(got, exp):
    assert np.array_equal(got[0], exp[0]), "col_ptr differs"
    if not np.array_equal(got[1], exp[1]):
        bad = np.nonzero(got[1] != exp[1])[0]
        raise AssertionError(f"row_idx differs at {bad.size} slots, first {bad[:8]}")
    if exp[2] is not None:
        assert np.array_equal(got[2].view(np.uint32), exp[2].view(np.uint32)), "vals differ"


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
    "hdv4096_w1024": dict(hdv_k=4096, table_log2=13, block_threads=128, ctas_per_sm=1, warp_edges=2048),
    "noagg_staged": dict(hdv_k=16, flags=0, stage_edges=128),
    "big_blocks": dict(hdv_k=128, block_threads=1024, ctas_per_sm=1, warp_edges=64),
    "steal": dict(hdv_k=512, flags=1 | 16, warp_edges=512),  # two-phase Step 3 (GT_FLAG_STEAL_TAILS)
    "steal_atomic": dict(hdv_k=0, flags=1 | 16, warp_edges=256),
    "radix": dict(method=1),  # bulk-copy staged downsweep
    "radix4096": dict(method=1, radix_tile=4096, ctas_per_sm=3),
    "radix2048": dict(method=1, radix_tile=2048, ctas_per_sm=6),
    # partitioned (two-level) form: bucket by the top destination bits first
    "part_atomic": dict(hdv_k=0, partition_bits=4),
    "part_hdv64": dict(hdv_k=64, partition_bits=8, warp_edges=128),
    "part_big": dict(hdv_k=512, partition_bits=2, block_threads=1024, ctas_per_sm=1, warp_edges=64),
    "part_noagg": dict(hdv_k=16, flags=0, partition_bits=6),
}


def test_fig1_reconstruction():
    row_ptr = np.array([0, 2, 3, 4, 6], np.uint64)
    col_idx = np.array([1, 2, 2, 3, 0, 1], np.uint32)
    assert_same(gpu_transpose(row_ptr, col_idx), oracle.transpose(row_ptr, col_idx))


def test_empty_and_degenerate():
    # no edges
    rp = np.zeros(9, np.uint64)
    got = gpu_transpose(rp, np.zeros(0, np.uint32))
    assert np.array_equal(got[0], np.zeros(9, np.uint64))
    # single vertex, weighted self-loops (order of parallel edges = CSR order)
    rp = np.array([0, 5], np.uint64)
    ci = np.zeros(5, np.uint32)
    vv = np.array([5, 4, 3, 2, 1], np.float32)
    assert_same(gpu_transpose(rp, ci, vv), oracle.transpose(rp, ci, vv))
    # all edges into the last vertex, long enough for the radix path
    n = 20000
    rp = np.arange(n + 1, dtype=np.uint64)
    ci = np.full(n, n - 1, np.uint32)
    vv = np.arange(n, dtype=np.float32)
    for name in ["atomic", "hdv64", "radix"]:
        assert_same(gpu_transpose(rp, ci, vv, config(**CONFIGS[name])), oracle.transpose(rp, ci, vv))


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("seed", [1, 2])
def test_random_graphs_all_configs(name, seed):
    n, rp, ci, vv = inputs.random_csr(5000, 77777, seed=seed, weighted=True, hot=20, hot_frac=0.4)
    assert_same(gpu_transpose(rp, ci, vv, config(**CONFIGS[name])), oracle.transpose(rp, ci, vv))
    assert_same(gpu_transpose(rp, ci, None, config(**CONFIGS[name])), oracle.transpose(rp, ci, None))


@pytest.mark.parametrize("order", ["natural", "random", "degree"])
def test_rmat_numpy_scale14(order):
    n, rp, ci, vv = inputs.rmat_csr(14, 16, seed=3, order=order, weighted=True)
    exp = oracle.transpose(rp, ci, vv)
    for name in ["atomic", "hdv512_staged", "big_blocks", "radix", "radix4096", "radix2048", "part_atomic",
                 "part_hdv64", "part_big"]:
        assert_same(gpu_transpose(rp, ci, vv, config(**CONFIGS[name])), exp)
    assert_same(gpu_transpose(rp, ci, vv), exp)  # default configuration


@pytest.mark.parametrize("m", [1, 4095, 4096, 4097, 8192 * 152 + 4096 * 3 + 17, 4096 * 700])
def test_radix_tile_boundaries(m):
    """Edge counts around the 4096-edge tile of the bulk-staged downsweep:
    one ragged tile, exactly one tile, a ragged last tile after full ones,
    uneven tiles per CTA, and a whole number of tiles."""
    n = 3000
    _, rp, ci, vv = inputs.random_csr(n, m, seed=m % 97, weighted=True, hot=5, hot_frac=0.3)
    exp = oracle.transpose(rp, ci, vv)
    assert_same(gpu_transpose(rp, ci, vv, config(**CONFIGS["radix"])), exp)
    assert_same(gpu_transpose(rp, ci, None, config(**CONFIGS["radix"])), oracle.transpose(rp, ci, None))


def test_long_parallel_edge_runs_in_split_rows():
    """A hub row split over many partitions sends 100,000 parallel edges into
    one long list and 3,000 into another: the tagged runs must come out in
    CSR order (long runs take the CTA sort paths, not a quadratic one)."""
    rng = np.random.default_rng(21)
    n = 6000
    rows = [np.concatenate([np.full(100000, 7), np.full(3000, 9), rng.integers(0, n, 50000)])]
    rows += [rng.integers(0, n, rng.integers(0, 40)) for _ in range(n - 1)]
    for r in rows[1:200]:
        r[:] = 7 if len(r) else r  # more sources into list 7
    rp = np.zeros(n + 1, np.uint64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.concatenate(rows).astype(np.uint32)
    vv = rng.standard_normal(len(ci)).astype(np.float32)
    exp = oracle.transpose(rp, ci, vv)
    for name in ["atomic", "hdv64", "noagg_staged", "radix", "steal", "steal_atomic", "part_atomic", "part_hdv64"]:
        assert_same(gpu_transpose(rp, ci, vv, config(**dict(CONFIGS[name], warp_edges=2048))), exp)


def test_radix_unaligned_arrays_fall_back():
    """Arrays that are not 16-byte aligned take the register downsweep."""
    from paper_2501_06872_gb300 import binding
    n, rp, ci, vv = inputs.rmat_csr(13, 8, seed=12, order="random", weighted=True)
    m = len(ci)
    exp = oracle.transpose(rp, ci, vv)
    d = torch.device("cuda:0")
    rpd = torch.from_numpy(rp.view(np.int64)).to(d)
    ci_big = torch.zeros(m + 1, dtype=torch.int32, device=d)
    ci_big[1:] = torch.from_numpy(ci.view(np.int32)).to(d)
    vv_big = torch.zeros(m + 1, dtype=torch.float32, device=d)
    vv_big[1:] = torch.from_numpy(vv).to(d)
    cp = torch.empty(n + 1, dtype=torch.int64, device=d)
    ri_big = torch.empty(m + 1, dtype=torch.int32, device=d)
    vo_big = torch.empty(m + 1, dtype=torch.float32, device=d)
    plan = binding.Plan(n, m, True, config(**CONFIGS["radix"]))
    plan.transpose(rpd, ci_big[1:], vv_big[1:], cp, ri_big[1:], vo_big[1:])
    plan.check()
    plan.close()
    got = (cp.cpu().numpy().view(np.uint64), ri_big[1:].cpu().numpy().view(np.uint32), vo_big[1:].cpu().numpy())
    assert_same(got, exp)


def test_split_rows_with_parallel_edges():
    """Hub rows much longer than a partition, with many parallel edges into
    LDV lists of all lengths: partitions split the rows, and parallel edges
    must keep CSR order."""
    rng = np.random.default_rng(5)
    n = 3000
    rows = []
    for u in range(n):
        if u in (0, 7, 1500):
            d = rng.integers(0, 40, size=30000)  # few destinations, many repeats
            d = np.where(rng.random(30000) < 0.5, d, rng.integers(0, n, size=30000))
        else:
            d = rng.integers(0, n, size=rng.integers(0, 6))
        rows.append(d.astype(np.uint32))
    rp = np.zeros(n + 1, np.uint64)
    rp[1:] = np.cumsum([r.size for r in rows])
    ci = np.concatenate(rows).astype(np.uint32)
    vv = rng.standard_normal(ci.size).astype(np.float32)
    exp = oracle.transpose(rp, ci, vv)
    for cfg in [config(hdv_k=0, warp_edges=64), config(hdv_k=8, warp_edges=128, stage_edges=128),
                config(hdv_k=0, warp_edges=4096, block_threads=64), config(method=1),
                config(hdv_k=0, warp_edges=64, partition_bits=5), config(hdv_k=8, warp_edges=128, partition_bits=8)]:
        assert_same(gpu_transpose(rp, ci, vv, cfg), exp)


def test_split_hub_rows_into_radix_lists():
    """Two hub rows of 120,000 edges into 10 destinations each (lists > 8192
    entries take the radix path) split across many partitions, weighted."""
    rng = np.random.default_rng(9)
    n = 500
    rows = [rng.integers(0, 10, size=120000) if u in (3, 250) else rng.integers(0, n, size=rng.integers(0, 4))
            for u in range(n)]
    rp = np.zeros(n + 1, np.uint64)
    rp[1:] = np.cumsum([r.size for r in rows])
    ci = np.concatenate(rows).astype(np.uint32)
    vv = rng.standard_normal(ci.size).astype(np.float32)
    exp = oracle.transpose(rp, ci, vv)
    for cfg in [config(hdv_k=0, warp_edges=256), config(hdv_k=4, warp_edges=512, stage_edges=256), config(method=1),
                config(hdv_k=0, warp_edges=256, partition_bits=3), config(hdv_k=4, warp_edges=512, partition_bits=8)]:
        assert_same(gpu_transpose(rp, ci, vv, cfg), exp)
    assert_same(gpu_transpose(rp, ci, None, config(hdv_k=0, warp_edges=256)), oracle.transpose(rp, ci, None))


def test_ragged_edge_counts_and_empty_rows():
    for m in [1, 3, 5, 31, 33, 129, 1023, 4097]:
        n = 257
        key = np.random.default_rng(m)
        src = np.sort(key.integers(0, n, size=m) // 3 * 3)  # two thirds of rows empty
        dst = key.integers(0, n, size=m)
        rp, ci, _ = inputs.csr_from_edges(n, src.astype(np.uint32), dst.astype(np.uint32))
        vv = key.standard_normal(m).astype(np.float32)
        exp = oracle.transpose(rp, ci, vv)
        for name in ["atomic", "noagg_staged", "hdv512_staged", "radix", "part_atomic", "part_hdv64"]:
            assert_same(gpu_transpose(rp, ci, vv, config(**CONFIGS[name])), exp)


@pytest.mark.parametrize("name", ["atomic", "hdv64", "radix", "radix4096", "part_atomic", "part_hdv64"])
def test_errors_are_reported_not_faulted(name):
    from paper_2501_06872_gb300 import binding
    cfg = config(**CONFIGS[name])
    cases = [
        (np.array([0, 2, 3, 4], np.uint64), np.array([1, 2, 3, 0], np.uint32), 2),  # 3 >= n
        (np.array([0, 3, 2, 4], np.uint64), np.array([1, 2, 0, 0], np.uint32), 3),  # decreasing
        (np.array([0, 1, 2, 3], np.uint64), np.array([1, 2, 0, 0], np.uint32), 3),  # row_ptr[n] != m
        (np.array([1, 2, 3, 4], np.uint64), np.array([1, 2, 0, 0], np.uint32), 3),  # row_ptr[0] != 0
        (np.array([0, 0, 1, 1], np.uint64), np.zeros(0, np.uint32), 3),             # m = 0, row_ptr not zero
    ]
    for rp, ci, code in cases:
        with pytest.raises(binding.GtError) as ei:
            gpu_transpose(rp, ci, None, cfg)
        assert ei.value.code == code, (rp, ci)


def test_host_path_matches_device_path():
    from paper_2501_06872_gb300 import binding
    n, rp, ci, vv = inputs.rmat_csr(12, 8, seed=4, order="random", weighted=True)
    m = ci.size
    plan = binding.Plan(n, m, True, config(hdv_k=64))
    cp = np.empty(n + 1, np.uint64)
    ri = np.empty(m, np.uint32)
    vo = np.empty(m, np.float32)
    for _ in range(2):
        plan.transpose_host(rp, ci, vv, cp, ri, vo)
        assert_same((cp, ri, vo), oracle.transpose(rp, ci, vv))
    plan.close()


def _column_multisets(cp, ri, vo, n):
    """(destination, source, value bits) triples sorted: the CSC as a multiset per list."""
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(cp.astype(np.int64)))
    vb = np.zeros_like(ri) if vo is None else vo.view(np.uint32)
    o = np.lexsort((vb, ri, cols))
    return cols[o], ri[o], vb[o]


@pytest.mark.parametrize("name", ["atomic", "hdv64", "hdv512_staged", "noagg_staged", "steal", "part_atomic",
                                  "part_hdv64"])
def test_unsorted_mode_keeps_every_list_as_a_multiset(name):
    """GT_FLAG_UNSORTED (the paper's output, no LDV sort): col_ptr is exact and
    every list holds the oracle's (source, value) multiset."""
    from paper_2501_06872_gb300 import binding
    graphs = [inputs.rmat_csr(13, 16, seed=5, order="random", weighted=True),
              inputs.random_csr(4000, 90001, seed=3, weighted=True, hot=7, hot_frac=0.5)]
    for n, rp, ci, vv in graphs:
        for vals in (vv, None):
            exp = oracle.transpose(rp, ci, vals)
            c = dict(CONFIGS[name])
            c["flags"] = c.get("flags", 1) | binding.FLAG_UNSORTED
            got = gpu_transpose(rp, ci, vals, config(**c))
            assert np.array_equal(got[0], exp[0])
            for x, y in zip(_column_multisets(got[0], got[1], got[2], n), _column_multisets(exp[0], exp[1], exp[2], n)):
                assert np.array_equal(x, y)


def test_unsorted_mode_split_hub_rows():
    """Hub rows split over partitions with many parallel edges: still the right multisets."""
    from paper_2501_06872_gb300 import binding
    rng = np.random.default_rng(31)
    n = 3000
    rows = [np.concatenate([np.full(20000, 7), rng.integers(0, n, 30000)])] + \
           [rng.integers(0, n, rng.integers(0, 30)) for _ in range(n - 1)]
    rp = np.zeros(n + 1, np.uint64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.concatenate(rows).astype(np.uint32)
    vv = rng.standard_normal(len(ci)).astype(np.float32)
    exp = oracle.transpose(rp, ci, vv)
    got = gpu_transpose(rp, ci, vv, config(hdv_k=0, warp_edges=2048, flags=1 | binding.FLAG_UNSORTED))
    assert np.array_equal(got[0], exp[0])
    for x, y in zip(_column_multisets(got[0], got[1], got[2], n), _column_multisets(exp[0], exp[1], exp[2], n)):
        assert np.array_equal(x, y)


def test_host_async_pipeline():
    """Three overlapped host calls with different values, each into its own
    pinned output buffers, all equal to the oracle."""
    from paper_2501_06872_gb300 import binding
    n, rp, ci, vv = inputs.rmat_csr(13, 16, seed=7, order="random", weighted=True)
    m = len(ci)
    plan = binding.Plan(n, m, True, config(**CONFIGS["radix"]))
    h_rp = torch.from_numpy(rp.view(np.int64)).pin_memory()
    h_ci = torch.from_numpy(ci.view(np.int32)).pin_memory()
    vals = [vv, vv * 2 + 1, -vv]
    h_vv = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).pin_memory() for x in vals]
    outs = [(torch.empty(n + 1, dtype=torch.int64).pin_memory(), torch.empty(m, dtype=torch.int32).pin_memory(),
             torch.empty(m, dtype=torch.float32).pin_memory()) for _ in vals]
    for k in range(3):
        plan.transpose_host_async(h_rp, h_ci, h_vv[k], *outs[k])
    plan.host_wait()
    for k in range(3):
        exp = oracle.transpose(rp, ci, vals[k].astype(np.float32))
        got = (outs[k][0].numpy().view(np.uint64), outs[k][1].numpy().view(np.uint32), outs[k][2].numpy())
        assert_same(got, exp)
    plan.close()


@pytest.mark.parametrize("name,sets", [("radix", 2), ("hdv64", 2), ("atomic", 2), ("radix", 1), ("hdv64", 1)])
def test_host_async_pipeline_different_graphs(name, sets, monkeypatch):
    """Four overlapped host calls on three different graphs of one shape: the
    next call's input copies start once the previous transposition stopped
    reading its inputs, and the two device output sets alternate; every call
    must still give its own graph's CSC."""
    from paper_2501_06872_gb300 import binding
    monkeypatch.setenv("GT_HOST_SETS", str(sets))  # 1: the one-set fallback of a plan short of memory
    n, m = 6000, 120000
    graphs = [inputs.random_csr(n, m, seed=70 + k, weighted=True, hot=5, hot_frac=0.3) for k in range(3)]
    order = [0, 1, 2, 1]
    plan = binding.Plan(n, m, True, config(**CONFIGS[name]))
    hin = [[torch.from_numpy(np.ascontiguousarray(x).view(t)).pin_memory()
            for x, t in ((g[1], np.int64), (g[2], np.int32), (g[3], np.float32))] for g in graphs]
    outs = [(torch.empty(n + 1, dtype=torch.int64).pin_memory(), torch.empty(m, dtype=torch.int32).pin_memory(),
             torch.empty(m, dtype=torch.float32).pin_memory()) for _ in order]
    for k, gi in enumerate(order):
        plan.transpose_host_async(*hin[gi], *outs[k])
    plan.host_wait()
    for k, gi in enumerate(order):
        _, rp, ci, vv = graphs[gi]
        got = (outs[k][0].numpy().view(np.uint64), outs[k][1].numpy().view(np.uint32), outs[k][2].numpy())
        assert_same(got, oracle.transpose(rp, ci, vv))
    plan.close()


def test_plan_reuse_and_stats():
    from paper_2501_06872_gb300 import binding
    n, rp, ci, vv = inputs.rmat_csr(13, 16, seed=2, order="degree", weighted=True)
    exp = oracle.transpose(rp, ci, vv)
    d_rp, d_ci, d_vv = _to_dev(rp, ci, vv)
    m = ci.size
    plan = binding.Plan(n, m, True, config(hdv_k=256, warp_edges=512))
    cp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(m, dtype=torch.int32, device="cuda")
    vo = torch.empty(m, dtype=torch.float32, device="cuda")
    plan.enable_timing(True)
    for _ in range(3):
        plan.transpose(d_rp, d_ci, d_vv, cp, ri, vo)
        plan.check()
        assert_same((cp.cpu().numpy().view(np.uint64), ri.cpu().numpy().view(np.uint32), vo.cpu().numpy()), exp)
    st = plan.stats()
    t = plan.timing()
    assert st["hdv_selected"] > 0 and 0 < st["hdv_edges"] < m and st["kernel_launches"] >= 8
    assert t["calls"] == 3 and t["total_ms"] > 0
    # every list of an HDV is long: coverage is the fraction of edges into them
    plan.set_config(config(hdv_k=0))
    plan.transpose(d_rp, d_ci, d_vv, cp, ri, vo)
    plan.check()
    assert plan.stats()["hdv_edges"] == 0
    plan.close()


@pytest.mark.parametrize("kind,order,weighted", [("rmat", "natural", False), ("rmat", "degree", True),
                                                  ("er", "random", True)])
def test_gpu_generated_scale16(kind, order, weighted):
    """R-MAT scale 16 (65,536 vertices, 1,048,576 edges) and a uniform graph of
    the same size, generated on the GPU, against the oracle."""
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    n, rp, ci, vv = ggen.graph(16, 16, kind=kind, seed=0x5EED0001, order=order, weighted=weighted)
    h_rp = rp.cpu().numpy().view(np.uint64)
    h_ci = ci.cpu().numpy().view(np.uint32)
    h_vv = None if vv is None else vv.cpu().numpy()
    exp = oracle.transpose(h_rp, h_ci, h_vv)
    out = binding.transpose(rp, ci, vv)
    got = (out[0].cpu().numpy().view(np.uint64), out[1].cpu().numpy().view(np.uint32),
           None if vv is None else out[2].cpu().numpy())
    assert_same(got, exp)


def test_step3_partition_times_are_recorded_and_change_no_byte():
    """GT_FLAG_PARTITION_TIMES records each warp partition's Step 3 (the
    scatter) start and end; the output stays the oracle's."""
    from paper_2501_06872_gb300 import binding
    n, rp, ci, vv = inputs.rmat_csr(17, 16, seed=5, order="random", weighted=True)
    exp = oracle.transpose(rp, ci, vv)
    rpd, cid, vvd = _to_dev(rp, ci, vv)
    m = len(ci)
    cfg = config(hdv_k=512, warp_edges=2048, flags=binding.FLAG_AGGREGATE | binding.FLAG_PARTITION_TIMES)
    plan = binding.Plan(n, m, True, cfg)
    cp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(m, dtype=torch.int32, device="cuda")
    vo = torch.empty(m, dtype=torch.float32, device="cuda")
    plan.transpose(rpd, cid, vvd, cp, ri, vo)
    plan.check()
    t = np.array(plan.partition_times())
    assert t.size == plan.stats()["partitions"] and (t >= 0).all() and t.max() > 0
    assert_same((cp.cpu().numpy().view(np.uint64), ri.cpu().numpy().view(np.uint32), vo.cpu().numpy()), exp)
    plan.close()
    plan = binding.Plan(n, m, True, config(hdv_k=512))
    with pytest.raises(binding.GtError) as e:
        plan.partition_times()
    assert e.value.code == 1
    plan.close()


@pytest.mark.parametrize("weighted", [True, False])
def test_two_phase_step3_on_skewed_graphs(weighted):
    """Two-phase Step 3 (heads by their own warps, tails claimed by free
    warps) on R-MAT graphs in all vertex orders, with HDVs and without:
    bit-exact, and its busy times are recorded per warp."""
    from paper_2501_06872_gb300 import binding
    for order in ("natural", "degree", "random"):
        n, rp, ci, vv = inputs.rmat_csr(16, 16, seed=31, order=order, weighted=weighted)
        exp = oracle.transpose(rp, ci, vv if weighted else None)
        for k in (0, 512):
            cfg = config(hdv_k=k, warp_edges=1024, flags=binding.FLAG_AGGREGATE | binding.FLAG_STEAL_TAILS)
            assert_same(gpu_transpose(rp, ci, vv if weighted else None, cfg), exp)


def test_two_phase_step3_rejects_staging():
    from paper_2501_06872_gb300 import binding
    with pytest.raises(binding.GtError) as e:
        binding.Plan(1000, 20000, True, config(hdv_k=64, stage_edges=256, flags=1 | 16))
    assert e.value.code == 1


def test_partitioned_form_rejects_staging_and_steal():
    from paper_2501_06872_gb300 import binding
    for bad in (dict(hdv_k=64, partition_bits=4, stage_edges=256), dict(hdv_k=64, partition_bits=4, flags=1 | 16),
                dict(hdv_k=0, partition_bits=9)):
        with pytest.raises(binding.GtError) as e:
            binding.Plan(1000, 20000, True, config(**bad))
        assert e.value.code == 1


@pytest.mark.parametrize("weighted", [True, False])
def test_partitioned_form_across_bucket_widths(weighted):
    """The two-level form (bucket by the top destination bits, then Steps
    0-3 over the bucketed list in ranges taken in order) on R-MAT graphs in
    every vertex order, for every bucket width up to all the key bits: the
    oracle's bytes, the bucketing time reported apart, and as many
    partitions as ranges of warp_edges edges."""
    from paper_2501_06872_gb300 import binding
    for order in ("natural", "degree", "random"):
        n, rp, ci, vv = inputs.rmat_csr(15, 16, seed=41, order=order, weighted=weighted)
        vals = vv if weighted else None
        exp = oracle.transpose(rp, ci, vals)
        m = ci.size
        for bits in (1, 5, 8):
            for k in (0, 256):
                cfg = config(hdv_k=k, warp_edges=512, partition_bits=bits)
                assert_same(gpu_transpose(rp, ci, vals, cfg), exp)
        # the timing split and the partition count through a plan
        rpd, cid, vvd = _to_dev(rp, ci, vals)
        plan = binding.Plan(n, m, weighted, config(hdv_k=256, warp_edges=512, partition_bits=8))
        cp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        ri = torch.empty(m, dtype=torch.int32, device="cuda")
        vo = torch.empty(m, dtype=torch.float32, device="cuda") if weighted else None
        plan.enable_timing(True)
        plan.transpose(rpd, cid, vvd, cp, ri, vo)
        plan.check()
        t = plan.timing()
        st = plan.stats()
        plan.close()
        assert t["partition_ms"] > 0 and t["total_ms"] >= t["partition_ms"]
        assert st["partitions"] >= m // 512  # one partition per range of warp_edges edges
        assert_same((cp.cpu().numpy().view(np.uint64), ri.cpu().numpy().view(np.uint32),
                     None if vo is None else vo.cpu().numpy()), exp)


@pytest.mark.parametrize("steal", [False, True])
def test_hdv_insertion_points_over_many_partitions(steal):
    """More than 32 K warp partitions (the partitioned form's ranges of
    warp_edges edges, or many small unpartitioned ones): the HDV insertion
    points are scanned in slices of partitions, with the same bytes."""
    from paper_2501_06872_gb300 import binding
    n, rp, ci, vv = inputs.rmat_csr(16, 32, seed=43, order="degree", weighted=True)
    exp = oracle.transpose(rp, ci, vv)
    if steal:  # unpartitioned: 32 CTAs of 32 warps per SM, two ranges per warp
        cfg = config(hdv_k=256, warp_edges=32, block_threads=1024, ctas_per_sm=32,
                     flags=binding.FLAG_AGGREGATE | binding.FLAG_STEAL_TAILS)
    else:
        cfg = config(hdv_k=256, warp_edges=32, partition_bits=6)
    from paper_2501_06872_gb300 import binding as b
    plan = b.Plan(n, ci.size, True, cfg)
    P = plan.stats()["partitions"]
    plan.close()
    assert P > 32768
    assert_same(gpu_transpose(rp, ci, vv, cfg), exp)


def test_long_tagged_runs_in_lists_sorted_by_three_radix_passes():
    """More than 2^16 rows, so the longest lists take three radix passes on the
    source and end in the caller's arrays rather than in the scratch: a hub row
    split over many partitions sends 80,000 parallel edges into one list (a
    tagged run far longer than 64) and 5,000 into another."""
    rng = np.random.default_rng(47)
    n = 70000
    rows = [np.concatenate([np.full(80000, 11), np.full(5000, 13), rng.integers(0, n, 20000)])]
    rows += [rng.integers(0, n, rng.integers(0, 6)) for _ in range(n - 1)]
    for r in rows[1:3000]:
        if len(r):
            r[0] = 11  # more sources into list 11, around the tagged run
    rp = np.zeros(n + 1, np.uint64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.concatenate(rows).astype(np.uint32)
    vv = rng.standard_normal(len(ci)).astype(np.float32)
    exp = oracle.transpose(rp, ci, vv)
    for cfg in [config(hdv_k=0, warp_edges=2048), config(hdv_k=4, warp_edges=1024),
                config(hdv_k=0, warp_edges=2048, partition_bits=6)]:
        assert_same(gpu_transpose(rp, ci, vv, cfg), exp)
