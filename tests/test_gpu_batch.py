"""Batched transposition (one CUDA-graph launch sequence over many graphs)
against the oracle per graph, and against the single-graph path."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _run_batch(b, weighted, cfg=None, calls=1, stream=None):
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    cp = torch.full((b["total_v"] + b["n_graphs"],), -1, dtype=torch.int64, device="cuda")
    ri = torch.full((b["total_m"],), -1, dtype=torch.int32, device="cuda")
    vo = torch.full((b["total_m"],), float("nan"), dtype=torch.float32, device="cuda") if weighted else None
    plan = binding.BatchPlan(ggen.batch_graphs(b, cp, ri, vo), weighted, cfg)
    s = stream or torch.cuda.Stream()
    for _ in range(calls):
        plan.transpose(s)
    plan.check()
    info = plan.info()
    plan.close()
    return cp, ri, vo, info


def _check_against_oracle(b, cp, ri, vo, weighted, graphs):
    rp_all = b["row_ptr"].cpu().numpy().view(np.uint64)
    ci_all = b["col_idx"].cpu().numpy().view(np.uint32)
    vv_all = b["vals"].cpu().numpy() if weighted else None
    cp_all = cp.cpu().numpy().view(np.uint64)
    ri_all = ri.cpu().numpy().view(np.uint32)
    vo_all = vo.cpu().numpy() if weighted else None
    for g in graphs:
        n, m = int(b["n"][g]), int(b["m"][g])
        r0, e0 = int(b["voff"][g]) + g, int(b["eoff"][g])
        exp = oracle.transpose(rp_all[r0:r0 + n + 1], ci_all[e0:e0 + m],
                               None if vv_all is None else vv_all[e0:e0 + m])
        assert np.array_equal(cp_all[r0:r0 + n + 1], exp[0]), f"col_ptr of graph {g}"
        assert np.array_equal(ri_all[e0:e0 + m], exp[1]), f"row_idx of graph {g}"
        if weighted:
            assert np.array_equal(vo_all[e0:e0 + m].view(np.uint32), exp[2].view(np.uint32)), f"vals of graph {g}"


@pytest.mark.parametrize("weighted", [True, False])
def test_batch_vs_oracle_graph_mode(weighted):
    from paper_2501_06872_gb300.inputs import gpu as ggen
    b = ggen.batch(n_graphs=48, seed=11, n_min=1024, n_max=6000, weighted=weighted)
    cp, ri, vo, info = _run_batch(b, weighted, calls=2)
    assert info["n_graphs"] == 48 and info["n_edges"] == b["total_m"] and info["kernel_launches"] > 0
    _check_against_oracle(b, cp, ri, vo, weighted, range(48))


def test_batch_no_graph_flag_and_key_widths():
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    b = ggen.batch(n_graphs=20, seed=12, n_min=1024, n_max=3000)
    for key_bits, flags in [(28, 2), (32, 0), (16, 0)]:  # 2 = GT_FLAG_NO_GRAPH
        cfg = binding.default_config(1 << 20, 1 << 24)
        cfg.method, cfg.flags, cfg.batch_key_bits = 1, flags, key_bits
        cp, ri, vo, info = _run_batch(b, True, cfg)
        _check_against_oracle(b, cp, ri, vo, True, range(20))
    # 16-bit keys hold 12 column bits and 4 graph bits: 16 graphs per sub-batch
    assert info["key_bits"] == 16 and info["sub_batches"] >= 2


def test_batch_many_sub_batches(monkeypatch):
    from paper_2501_06872_gb300.inputs import gpu as ggen
    monkeypatch.setenv("GT_BATCH_MAX_EDGES", "50000")
    b = ggen.batch(n_graphs=30, seed=13, n_min=1024, n_max=2048)
    cp, ri, vo, info = _run_batch(b, True)
    assert info["sub_batches"] > 3
    _check_against_oracle(b, cp, ri, vo, True, range(30))


def test_batch_matches_single_graph_path():
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    b = ggen.batch(n_graphs=12, seed=14, n_min=2000, n_max=20000)
    cp, ri, vo, _ = _run_batch(b, True)
    nmax, mmax = int(b["n"].max()), int(b["m"].max())
    plan = binding.Plan(nmax, mmax, True)
    for g in range(12):
        n, m = int(b["n"][g]), int(b["m"][g])
        r0, e0 = int(b["voff"][g]) + g, int(b["eoff"][g])
        c2 = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        r2 = torch.empty(m, dtype=torch.int32, device="cuda")
        v2 = torch.empty(m, dtype=torch.float32, device="cuda")
        plan.transpose_sub(n, m, b["row_ptr"][r0:r0 + n + 1], b["col_idx"][e0:e0 + m], b["vals"][e0:e0 + m],
                           c2, r2, v2)
        plan.check()
        assert torch.equal(c2, cp[r0:r0 + n + 1]) and torch.equal(r2, ri[e0:e0 + m])
        assert torch.equal(v2.view(torch.int32), vo[e0:e0 + m].view(torch.int32))
    plan.close()


def test_batch_reports_out_of_range():
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    b = ggen.batch(n_graphs=5, seed=15, n_min=1024, n_max=1500)
    e0 = int(b["eoff"][3])
    b["col_idx"][e0 + 7] = int(b["n"][3])  # == n: out of range
    with pytest.raises(binding.GtError) as ei:
        _run_batch(b, True)
    assert ei.value.code == 2


def _descs_tensor(graphs):
    """Device copy of a descriptor list (the bytes of gt_graph_desc[])."""
    import ctypes
    from paper_2501_06872_gb300 import binding
    arr = (binding.GraphDesc * len(graphs))()
    for i, g in enumerate(graphs):
        arr[i] = binding.GraphDesc(int(g["n"]), int(g.get("n_cols", 0)), int(g["m"]), g["row_ptr"], g["col_idx"],
                                   g.get("vals"), g["col_ptr"], g["row_idx"], g.get("vals_out"))
    return torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).cuda()


def _outputs(b, weighted):
    cp = torch.full((b["total_v"] + b["n_graphs"],), -1, dtype=torch.int64, device="cuda")
    ri = torch.full((b["total_m"],), -1, dtype=torch.int32, device="cuda")
    vo = torch.full((b["total_m"],), float("nan"), dtype=torch.float32, device="cuda") if weighted else None
    return cp, ri, vo


def test_two_batches_through_one_plan_and_one_captured_graph():
    """A plan sized by limits takes two different batches (device descriptor
    arrays passed per call) on the same stream: the second call replays the
    CUDA graph captured by the first with the new descriptors."""
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    ba = ggen.batch(n_graphs=30, seed=31, n_min=1024, n_max=8000)
    bb = ggen.batch(n_graphs=45, seed=32, n_min=1500, n_max=5000)
    limits = {"max_graphs": 64, "max_cols": 8192, "max_graph_edges": 1 << 20,
              "max_edges": max(ba["total_m"], bb["total_m"]) + 1000,
              "max_cols_total": max(ba["total_v"], bb["total_v"]) + 1000}
    plan = binding.BatchPlan([], True, limits=limits)
    s = torch.cuda.Stream()
    for b in (ba, bb, ba):
        cp, ri, vo = _outputs(b, True)
        graphs = ggen.batch_graphs(b, cp, ri, vo)
        d = _descs_tensor(graphs)
        st = torch.full((len(graphs),), -7, dtype=torch.int32, device="cuda")
        plan.transpose_descs(len(graphs), d, st, s)
        plan.check()
        assert st.cpu().tolist() == [0] * len(graphs)
        info = plan.info()
        assert info["n_graphs"] == b["n_graphs"] and info["n_edges"] == b["total_m"]
        _check_against_oracle(b, cp, ri, vo, True, range(b["n_graphs"]))
    plan.close()


def test_per_graph_status_reports_each_graphs_own_error():
    """Graph 1: a destination out of range; graph 3: row_ptr[n] != m; graph 4:
    no vertices; graph 6: more columns than the plan's limit.  Each gets its
    own code, the others are transposed bit-exactly."""
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    b = ggen.batch(n_graphs=8, seed=33, n_min=1024, n_max=3000)
    cp, ri, vo = _outputs(b, True)
    graphs = ggen.batch_graphs(b, cp, ri, vo)
    e1 = int(b["eoff"][1])
    b["col_idx"][e1 + 3] = int(b["n"][1]) + 5                      # out of range
    r3 = int(b["voff"][3]) + 3
    graphs[3] = dict(graphs[3], m=int(b["m"][3]) + 1)               # row_ptr[n] != m
    graphs[4] = dict(graphs[4], n=0)                                # no vertices
    graphs[6] = dict(graphs[6], n_cols=1 << 20)                     # wider than the limit
    limits = {"max_graphs": 8, "max_cols": 4096, "max_graph_edges": int(b["m"].max()) + 10,
              "max_edges": b["total_m"] + 10, "max_cols_total": b["total_v"] + (1 << 20)}
    plan = binding.BatchPlan(graphs, True, limits=limits)
    plan.transpose()
    codes = plan.graph_status()
    assert codes == [0, 2, 0, 3, 1, 0, 7, 0], codes
    assert plan.status() != 0
    plan.close()
    # the other graphs are exact (graph 3's row_ptr and values were not touched, its descriptor was)
    _check_against_oracle(b, cp, ri, vo, True, [0, 2, 5, 7])
    del r3


def test_batch_autotuner_picks_a_grid_point_and_keeps_bytes():
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    b = ggen.batch(n_graphs=40, seed=34, n_min=1024, n_max=20000)
    cp, ri, vo = _outputs(b, True)
    plan = binding.BatchPlan(ggen.batch_graphs(b, cp, ri, vo), True)
    chosen, table = plan.tune(reps=2)
    assert 0 <= chosen < binding.BATCH_TUNE_GRID
    assert table[chosen] > 0 and all(t < 0 or t >= table[chosen] for t in table)
    cfg = plan.config()
    ref = binding.batch_grid_config(chosen)
    assert (cfg.batch_key_bits, cfg.batch_edges_log2) == (ref.batch_key_bits, ref.batch_edges_log2)
    plan.check()
    _check_against_oracle(b, cp, ri, vo, True, range(40))
    cp.fill_(-1)
    plan.transpose()  # the installed configuration, replayed
    plan.check()
    _check_against_oracle(b, cp, ri, vo, True, range(40))
    plan.close()
