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


def test_batch_no_graph_flag_and_tile_2048():
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    b = ggen.batch(n_graphs=20, seed=12, n_min=1024, n_max=3000)
    cfg = binding.default_config(1 << 20, 1 << 24)
    cfg.method, cfg.radix_tile, cfg.ctas_per_sm, cfg.flags = 1, 2048, 3, 2  # GT_FLAG_NO_GRAPH
    cp, ri, vo, info = _run_batch(b, True, cfg)
    _check_against_oracle(b, cp, ri, vo, True, range(20))


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
