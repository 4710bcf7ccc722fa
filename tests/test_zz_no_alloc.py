"""gt_transpose_noalloc, the entry point for callers that cannot allocate
device memory on the call path (a host program whose pool owns all device
memory, or a loop that cannot take cudaMalloc's synchronisation).  Its output
must equal the oracle's and gt_transpose's, bit for bit, on consecutive calls
that reuse the shared fixed scratch array, including the degenerate graphs
(no vertices, no edges) and a graph whose workspace only just fits.
Collected last on purpose."""
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


def _dev(rp, ci, vv):
    d = torch.device("cuda:0")
    return (torch.from_numpy(rp.view(np.int64)).to(d), torch.from_numpy(ci.view(np.int32)).to(d),
            None if vv is None else torch.from_numpy(vv).to(d))


def _outs(n, m, weighted):
    return (torch.empty(n + 1, dtype=torch.int64, device="cuda"), torch.empty(m, dtype=torch.int32, device="cuda"),
            torch.empty(m, dtype=torch.float32, device="cuda") if weighted else None)


def _assert_oracle(out, exp):
    assert np.array_equal(out[0].cpu().numpy().view(np.uint64), exp[0]), "col_ptr differs from the oracle"
    assert np.array_equal(out[1].cpu().numpy().view(np.uint32), exp[1]), "row_idx differs from the oracle"
    if exp[2] is not None:
        assert np.array_equal(out[2].cpu().numpy().view(np.uint32), exp[2].view(np.uint32)), "vals differ"


@pytest.mark.parametrize("weighted", [True, False])
def test_noalloc_matches_oracle_and_gt_transpose_twice(weighted):
    from paper_2501_06872_gb300 import binding
    graphs = [inputs.rmat_csr(14, 16, seed=21, order="random", weighted=weighted),
              inputs.random_csr(3000, 50000, seed=22, weighted=weighted, hot=5, hot_frac=0.3)]
    for n, rp, ci, vv in graphs:
        exp = oracle.transpose(rp, ci, vv)
        rp_d, ci_d, vv_d = _dev(rp, ci, vv)
        ref = binding.transpose(rp_d, ci_d, vv_d)
        for _ in range(2):  # the second call starts from the first call's leftovers
            out = _outs(n, ci.size, weighted)
            binding.transpose_noalloc(rp_d, ci_d, vv_d, *out)
            torch.cuda.synchronize()
            _assert_oracle(out, exp)
            assert torch.equal(out[0], ref[0])
            assert torch.equal(out[1], ref[1])
            if weighted:
                assert torch.equal(out[2].view(torch.int32), ref[2].view(torch.int32))


@pytest.mark.parametrize("weighted", [True, False])
def test_noalloc_degenerate_graphs(weighted):
    from paper_2501_06872_gb300 import binding
    # no vertices (col_ptr = [0]), then vertices without edges (col_ptr all 0)
    for n in (0, 1, 5000):
        rp = np.zeros(n + 1, np.uint64)
        ci = np.zeros(0, np.uint32)
        vv = np.zeros(0, np.float32) if weighted else None
        exp = oracle.transpose(rp, ci, vv)
        rp_d = torch.from_numpy(rp.view(np.int64)).cuda()
        ci_d = torch.empty(0, dtype=torch.int32, device="cuda")
        vv_d = torch.empty(0, dtype=torch.float32, device="cuda") if weighted else None
        for _ in range(2):
            out = _outs(n, 0, weighted)
            out[0].fill_(-1)
            binding.transpose_noalloc(rp_d, ci_d, vv_d, *out)
            torch.cuda.synchronize()
            _assert_oracle(out, exp)


def _even_graph(n, m, seed):
    """n vertices, m edges spread evenly over the rows, uniform destinations."""
    rng = np.random.default_rng(seed)
    rp = (np.arange(n + 1, dtype=np.uint64) * np.uint64(m)) // np.uint64(n)
    ci = rng.integers(0, n, m, dtype=np.uint32)
    return rp, ci


def _fits(n, m, weighted):
    """Whether the entry point accepts an n-vertex, m-edge graph (a rejected
    call returns GT_ERR_UNSUPPORTED before it enqueues anything)."""
    from paper_2501_06872_gb300 import binding
    rp = (torch.arange(n + 1, dtype=torch.int64, device="cuda") * m) // n
    ci = torch.zeros(m, dtype=torch.int32, device="cuda")
    vv = torch.zeros(m, dtype=torch.float32, device="cuda") if weighted else None
    try:
        binding.transpose_noalloc(rp, ci, vv, *_outs(n, m, weighted))
        return True
    except binding.GtError as e:
        assert e.code == 7, f"unexpected status {e.code}"
        return False


@pytest.mark.parametrize("weighted", [True, False])
def test_noalloc_largest_graph_that_fits(weighted):
    """The largest edge count the fixed array takes for 2^20 vertices (found
    by bisection over the entry point's own accept/reject answer) transposes
    bit-exactly; one edge more is rejected."""
    from paper_2501_06872_gb300 import binding
    n = 1 << 20
    lo, hi = 1, 1 << 25  # lo fits, hi does not
    assert _fits(n, lo, weighted) and not _fits(n, hi, weighted)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if _fits(n, mid, weighted):
            lo = mid
        else:
            hi = mid
    m = lo
    assert m > (1 << 22)  # tens of MiB of edge workspace inside the 64 MiB array
    rp, ci = _even_graph(n, m, seed=64)
    vv = np.random.default_rng(65).random(m, dtype=np.float32) if weighted else None
    exp = oracle.transpose(rp, ci, vv)
    rp_d, ci_d, vv_d = _dev(rp, ci, vv)
    for _ in range(2):
        out = _outs(n, m, weighted)
        binding.transpose_noalloc(rp_d, ci_d, vv_d, *out)
        torch.cuda.synchronize()
        _assert_oracle(out, exp)
    assert not _fits(n, m + 1, weighted)


def test_noalloc_rejects_graphs_beyond_its_scratch():
    from paper_2501_06872_gb300 import binding
    n, m = 1 << 22, 1 << 24  # workspace well above 64 MiB
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(m, dtype=torch.int32, device="cuda")
    out = _outs(n, m, False)
    with pytest.raises(binding.GtError) as ei:
        binding.transpose_noalloc(rp, ci, None, *out)
    assert ei.value.code == 7  # GT_ERR_UNSUPPORTED
