"""gt_transpose_noalloc, the entry point for callers that cannot allocate
device memory on the call path (a host program whose pool owns all device
memory, or a loop that cannot take cudaMalloc's synchronisation).  Its output
must equal gt_transpose's, bit for bit, on consecutive calls that reuse the
shared fixed scratch array.  Collected last on purpose."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("weighted", [True, False])
def test_noalloc_matches_gt_transpose_twice(weighted):
    from paper_2501_06872_gb300 import binding
    graphs = [inputs.rmat_csr(14, 16, seed=21, order="random", weighted=weighted),
              inputs.random_csr(3000, 50000, seed=22, weighted=weighted, hot=5, hot_frac=0.3)]
    for n, rp, ci, vv in graphs:
        rp_d, ci_d, vv_d = _dev(rp, ci, vv)
        ref = binding.transpose(rp_d, ci_d, vv_d)
        for _ in range(2):  # the second call starts from the first call's leftovers
            out = _outs(n, ci.size, weighted)
            binding.transpose_noalloc(rp_d, ci_d, vv_d, *out)
            torch.cuda.synchronize()
            assert torch.equal(out[0], ref[0])
            assert torch.equal(out[1], ref[1])
            if weighted:
                assert torch.equal(out[2].view(torch.int32), ref[2].view(torch.int32))


def test_noalloc_rejects_graphs_beyond_its_scratch():
    from paper_2501_06872_gb300 import binding
    n, m = 1 << 22, 1 << 24  # workspace well above 64 MiB
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(m, dtype=torch.int32, device="cuda")
    out = _outs(n, m, False)
    with pytest.raises(binding.GtError) as ei:
        binding.transpose_noalloc(rp, ci, None, *out)
    assert ei.value.code == 7  # GT_ERR_UNSUPPORTED
