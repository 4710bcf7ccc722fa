"""Whole-output parity at the full sizes of the stated workloads, element by
element against the oracle:

* R-MAT scale 24, random vertex order, unweighted (16.8 M vertices, 268 M
  edges), and the Erdos-Renyi graph of the same size, each through the radix
  method (the library's default at this size) and through PoTra's own method
  (Algorithm 2 with k = 512 HDVs);
* R-MAT scale 28 with f32 values (2^28 vertices, 2^32 edges) in the
  degree-sorted and in the random vertex order, through the default
  configuration the bench times.

The oracle runs on destination ranges [lo, hi) in parallel host threads
(``oracle.transpose_range``: the same counting sort restricted to a range,
with global offsets; together the ranges cover every destination once).  The
range bounds split the edges evenly, from a histogram of the input col_idx
made by the input generator library.  Each scale-28 case needs a GPU with
more than 200 GB and about 110 GB of host memory, and runs for a minute or
two."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _threads():
    return max(1, min(16, len(os.sched_getaffinity(0))))


def _bounds(ci, n, parts):
    """Destination bounds 0 = b_0 < ... < b_parts = n splitting the edges
    about evenly (in-degree histogram of the input, prefix sums, search)."""
    from paper_2501_06872_gb300.inputs import gpu as ggen
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    ggen._ok(ggen.load().gtgen_histogram(ggen._p(ci), ci.numel(), ggen._p(counts), ggen._s()), "gtgen_histogram")
    cum = torch.cumsum(counts.to(torch.int64), 0)
    del counts
    m = ci.numel()
    targets = torch.tensor([(k * m) // parts for k in range(1, parts)], dtype=torch.int64, device="cuda")
    inner = torch.searchsorted(cum, targets, right=True).cpu().numpy().tolist()
    del cum
    b = sorted(set([0] + [min(max(int(x), 1), n - 1) for x in inner] + [n]))
    return list(zip(b[:-1], b[1:]))


def _host(rp, ci, vv):
    rp_h = rp.cpu().numpy().view(np.uint64)
    ci_h = ci.cpu().numpy().view(np.uint32)
    vv_h = None if vv is None else vv.cpu().numpy()
    return rp_h, ci_h, vv_h


def _check_range(lo, hi, res, outs):
    """One oracle range against every GPU output in outs (col_ptr, row_idx, vals_out)."""
    cp_o, rows_o, vals_o = res
    a, b = int(cp_o[0]), int(cp_o[-1])
    for name, (cp, ri, vo) in outs.items():
        cp_g = cp[lo:hi + 1].cpu().numpy().view(np.uint64)
        if not np.array_equal(cp_g, cp_o):
            bad = np.nonzero(cp_g != cp_o)[0]
            raise AssertionError(f"{name}: col_ptr differs in [{lo},{hi}) at {bad.size} entries, first {lo + bad[0]}")
        ri_g = ri[a:b].cpu().numpy().view(np.uint32)
        if not np.array_equal(ri_g, rows_o):
            bad = np.nonzero(ri_g != rows_o)[0]
            raise AssertionError(f"{name}: row_idx differs in [{lo},{hi}) at {bad.size} slots, first {a + bad[0]}")
        if vals_o is not None:
            vo_g = vo[a:b].cpu().numpy().view(np.uint32)
            assert np.array_equal(vo_g, vals_o.view(np.uint32)), f"{name}: vals differ in [{lo},{hi})"


def _oracle_compare(rp_h, ci_h, vv_h, ranges, outs):
    """Runs the oracle over the ranges in parallel threads and compares each
    range with every GPU output as soon as it is done; returns the edges
    covered."""
    covered = 0
    with cf.ThreadPoolExecutor(_threads()) as ex:
        futs = {ex.submit(oracle.transpose_range, rp_h, ci_h, vv_h, lo, hi): (lo, hi) for lo, hi in ranges}
        for f in cf.as_completed(futs):
            lo, hi = futs[f]
            res = f.result()
            _check_range(lo, hi, res, outs)
            covered += int(res[0][-1] - res[0][0])
            del res
    return covered


def _run(rp, ci, vv, n, cfg):
    from paper_2501_06872_gb300 import binding
    m = ci.numel()
    plan = binding.Plan(n, m, vv is not None, cfg)
    cp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(m, dtype=torch.int32, device="cuda")
    vo = torch.empty(m, dtype=torch.float32, device="cuda") if vv is not None else None
    try:
        plan.transpose(rp, ci, vv, cp, ri, vo)
        plan.check()
        method = plan.config().method
    finally:
        plan.close()
    return (cp, ri, vo), method


def _hlh_config(n, m):
    from paper_2501_06872_gb300 import binding
    cfg = binding.default_config(n, m)
    cfg.method, cfg.hdv_k, cfg.table_log2 = 0, 512, 10
    return cfg


@pytest.mark.parametrize("workload", ["rmat24-random", "er24-random"])
def test_scale24_whole_output_radix_and_hlh(workload):
    import bench
    from paper_2501_06872_gb300 import binding
    n, n_cols, rp, ci, vv = bench.make_workload(workload, bench.SEED)
    m = ci.numel()
    assert (n, n_cols, m, vv) == (1 << 24, 1 << 24, 1 << 28, None)
    outs = {}
    outs["default"], method = _run(rp, ci, vv, n, binding.default_config(n, m))
    assert method == 1  # the radix method, as the bench runs this size
    outs["hlh_k512"], method = _run(rp, ci, vv, n, _hlh_config(n, m))
    assert method == 0
    ranges = _bounds(ci, n, 16)
    rp_h, ci_h, vv_h = _host(rp, ci, vv)
    assert _oracle_compare(rp_h, ci_h, vv_h, ranges, outs) == m


@pytest.mark.parametrize("workload", ["rmat28-degree", "rmat28-random"])
def test_scale28_weighted_whole_output(workload):
    import bench
    from paper_2501_06872_gb300 import binding
    if torch.cuda.get_device_properties(0).total_memory < 200e9:
        pytest.skip("needs a GPU with more than 200 GB")
    avail = _mem_available()
    if avail and avail < 120e9:
        pytest.skip("needs about 110 GB of free host memory for the inputs and the oracle's output")
    n, n_cols, rp, ci, vv = bench.make_workload(workload, bench.SEED)
    m = ci.numel()
    assert (n, n_cols, m) == (1 << 28, 1 << 28, 1 << 32) and vv is not None
    out, method = _run(rp, ci, vv, n, binding.default_config(n, m))
    assert method == 1
    torch.cuda.empty_cache()
    ranges = _bounds(ci, n, max(16, _threads()))
    rp_h, ci_h, vv_h = _host(rp, ci, vv)
    del rp, ci, vv
    torch.cuda.empty_cache()
    assert _oracle_compare(rp_h, ci_h, vv_h, ranges, {"default": out}) == m
