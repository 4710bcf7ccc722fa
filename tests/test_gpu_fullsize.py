"""Parity at the full sizes the bench times, in the bench's launch
configuration (the library's default for the size):

* R-MAT scale 28, 2^32 weighted edges, degree-sorted: sampled columns
  against the oracle element by element (the heaviest lists, seeded random
  ones, the last ones), and over all 2^32 entries the properties any correct
  CSC has -- col_ptr[0] = 0, col_ptr[n] = m, col_ptr non-decreasing, in-degrees
  equal to a histogram of col_idx, the multiset sums of row IDs and value
  bits preserved, and sources ascending inside every column.
* The 4096-matrix batch (3.67 G edges): every matrix against the oracle.

Each test needs a GPU with more than 200 GB of memory and about 60 GB of
host memory, and runs for a minute or so."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    if torch.cuda.get_device_properties(0).total_memory < 200e9:
        pytest.skip("needs a GPU with more than 200 GB")
    avail = 0
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    if avail and avail < 80e9:
        pytest.skip("needs about 60 GB of free host memory for the oracle's inputs")
    import __graft_entry__
    __graft_entry__.build()


def test_rmat28_bench_workload_sampled_columns_and_properties():
    import bench
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    n, n_cols, rp, ci, vv = bench.make_workload("rmat28-degree", bench.SEED)
    m = ci.numel()
    assert (n, m) == (1 << 28, 1 << 32)
    plan = binding.Plan(n, m, True, binding.default_config(n, m))
    cp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(m, dtype=torch.int32, device="cuda")
    vo = torch.empty(m, dtype=torch.float32, device="cuda")
    plan.transpose(rp, ci, vv, cp, ri, vo)
    plan.check()
    assert plan.config().method == 1  # the radix method, as the bench runs it
    plan.close()
    torch.cuda.empty_cache()

    # properties over all entries
    assert int(cp[0]) == 0 and int(cp[n]) == m
    deg = cp[1:] - cp[:-1]
    assert bool((deg >= 0).all())
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    ggen._ok(ggen.load().gtgen_histogram(ggen._p(ci), m, ggen._p(counts), ggen._s()), "gtgen_histogram")
    assert torch.equal(deg, counts.to(torch.int64))
    del counts
    out_deg = rp[1:] - rp[:-1]
    rows = torch.arange(n, dtype=torch.int64, device="cuda")
    src_sum = int((rows * out_deg).sum().item())  # < 2^60: exact in int64
    del rows, out_deg
    assert int(ri.to(torch.int64).sum().item()) == src_sum
    vbits = lambda t: t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    assert int(vbits(vo).sum().item()) == int(vbits(vv).sum().item())
    start = torch.zeros(m, dtype=torch.bool, device="cuda")
    start[cp[:-1][deg > 0]] = True
    ok = (ri[1:] >= ri[:-1]) | start[1:]
    assert bool(ok.all())
    del start, ok, deg

    # sampled columns against the oracle
    rng = np.random.default_rng(28)
    cols = np.unique(np.concatenate([np.arange(8), rng.integers(0, n, 40), np.arange(n - 4, n)])).astype(np.uint32)
    rp_h = rp.cpu().numpy().view(np.uint64)
    ci_h = ci.cpu().numpy().view(np.uint32)
    vv_h = vv.cpu().numpy()
    c, start_o, deg_o, rows_o, vals_o = oracle.columns(rp_h, ci_h, vv_h, cols)
    cp_h = cp.cpu().numpy()
    off = 0
    for i, v in enumerate(c):
        a, b = int(cp_h[v]), int(cp_h[v + 1])
        assert a == int(start_o[i]) and b - a == int(deg_o[i]), f"col_ptr of column {v}"
        d = b - a
        assert np.array_equal(ri[a:b].cpu().numpy().view(np.uint32), rows_o[off:off + d]), f"rows of column {v}"
        assert np.array_equal(vo[a:b].cpu().numpy().view(np.uint32), vals_o[off:off + d].view(np.uint32)), \
            f"values of column {v}"
        off += d
    assert off > 1_000_000  # the heaviest lists are in the sample


def test_batch_4096_every_matrix():
    """The 4096-matrix batch (3.67 G edges) through one batch plan, every
    matrix compared with the oracle element by element (host threads, one
    matrix per task)."""
    import concurrent.futures as cf
    import os
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    b = ggen.batch(n_graphs=4096, seed=0x5EED0004)
    cp = torch.full((b["total_v"] + b["n_graphs"],), -1, dtype=torch.int64, device="cuda")
    ri = torch.full((b["total_m"],), -1, dtype=torch.int32, device="cuda")
    vo = torch.full((b["total_m"],), float("nan"), dtype=torch.float32, device="cuda")
    plan = binding.BatchPlan(ggen.batch_graphs(b, cp, ri, vo), True)
    plan.transpose()
    plan.check()
    assert plan.graph_status() == [0] * 4096
    plan.close()
    rp_all = b["row_ptr"].cpu().numpy().view(np.uint64)
    ci_all = b["col_idx"].cpu().numpy().view(np.uint32)
    vv_all = b["vals"].cpu().numpy()
    cp_all = cp.cpu().numpy().view(np.uint64)
    ri_all = ri.cpu().numpy().view(np.uint32)
    vo_all = vo.cpu().numpy().view(np.uint32)
    del cp, ri, vo
    ns, ms = b["n"].tolist(), b["m"].tolist()
    voff, eoff = b["voff"].tolist(), b["eoff"].tolist()

    def check(g):
        n, m = int(ns[g]), int(ms[g])
        r0, e0 = int(voff[g]) + g, int(eoff[g])
        exp = oracle.transpose(rp_all[r0:r0 + n + 1], ci_all[e0:e0 + m], vv_all[e0:e0 + m])
        ok = (np.array_equal(cp_all[r0:r0 + n + 1], exp[0]) and np.array_equal(ri_all[e0:e0 + m], exp[1]) and
              np.array_equal(vo_all[e0:e0 + m], exp[2].view(np.uint32)))
        return g, m, ok
    threads = max(1, min(16, len(os.sched_getaffinity(0))))
    covered = 0
    with cf.ThreadPoolExecutor(threads) as ex:
        for g, m, ok in ex.map(check, range(4096)):
            assert ok, f"matrix {g} differs from the oracle"
            covered += m
    assert covered == b["total_m"]
