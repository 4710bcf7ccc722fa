"""64-bit vertex IDs (gt_transpose_u64) against the 64-bit oracle, element by
element: small rectangular matrices, a matrix with more than 2^32 columns
(33-bit destination keys) and one with more than 2^32 rows (33-bit source
IDs).  The two large cases hold 34 GB arrays on the GPU and on the host."""
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


def _dev64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _assert_same(got, exp):
    cp, ri, vo = got
    assert np.array_equal(cp.cpu().numpy().view(np.uint64), exp[0]), "col_ptr differs"
    assert np.array_equal(ri.cpu().numpy().view(np.uint64), exp[1]), "row_idx differs"
    if exp[2] is not None:
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), exp[2].view(np.uint32)), "vals differ"


@pytest.mark.parametrize("weighted", [True, False])
def test_u64_small_matrices_match_the_oracle(weighted):
    from paper_2501_06872_gb300 import binding
    rng = np.random.default_rng(640)
    for nr, nc, m in [(1, 1, 1), (7, 3, 40), (300, 5000, 70000), (5000, 300, 70000), (20000, 20000, 1 << 18)]:
        deg = rng.multinomial(m, np.ones(nr) / nr)
        rp = np.zeros(nr + 1, np.uint64)
        np.cumsum(deg, out=rp[1:])
        hot = rng.integers(0, nc, 4)
        ci = np.where(rng.random(m) < 0.3, hot[rng.integers(0, 4, m)], rng.integers(0, nc, m)).astype(np.uint64)
        vv = rng.standard_normal(m).astype(np.float32) if weighted else None
        exp = oracle.transpose64(rp, ci, vv, n_cols=nc)
        got = binding.transpose_u64(_dev64(rp), _dev64(ci), None if vv is None else torch.from_numpy(vv).cuda(),
                                    n_cols=nc)
        _assert_same(got, exp)


def test_u64_errors_and_empty():
    from paper_2501_06872_gb300 import binding
    rp = _dev64([0, 2, 3])
    with pytest.raises(binding.GtError) as e:
        binding.transpose_u64(rp, _dev64([0, 9, 1]), n_cols=9)  # 9 >= n_cols
    assert e.value.code == 2
    with pytest.raises(binding.GtError) as e:
        binding.transpose_u64(_dev64([0, 2, 1]), _dev64([0, 1]), n_cols=4)
    assert e.value.code == 3
    cp, ri, _ = binding.transpose_u64(_dev64([0, 0, 0]), _dev64([]), n_cols=5)
    assert cp.cpu().tolist() == [0] * 6 and ri.numel() == 0


def test_u64_more_than_2_32_columns():
    """2^20 rows, 2^32 + 2^20 + 7 columns: uniform destinations, a band around
    2^32 and hot columns above it; col_ptr (34 GB) is compared whole."""
    from paper_2501_06872_gb300 import binding
    if torch.cuda.get_device_properties(0).total_memory < 150e9:
        pytest.skip("needs a GPU with more than 150 GB")
    avail = _mem_available()
    if avail and avail < 110e9:
        pytest.skip("needs about 100 GB of free host memory")
    nr, nc, m = 1 << 20, (1 << 32) + (1 << 20) + 7, 1 << 22
    rng = np.random.default_rng(641)
    deg = rng.multinomial(m, np.ones(nr) / nr)
    rp = np.zeros(nr + 1, np.uint64)
    np.cumsum(deg, out=rp[1:])
    pick = rng.random(m)
    uni = rng.integers(0, nc, m, dtype=np.uint64)
    band = (1 << 32) - 1000 + rng.integers(0, 2000, m).astype(np.uint64)
    hot = np.array([(1 << 32) + 5, (1 << 32) + 123456, nc - 1], np.uint64)[rng.integers(0, 3, m)]
    ci = np.where(pick < 0.5, uni, np.where(pick < 0.75, band, hot)).astype(np.uint64)
    vv = rng.standard_normal(m).astype(np.float32)
    cp, ri, vo = binding.transpose_u64(_dev64(rp), _dev64(ci), torch.from_numpy(vv).cuda(), n_cols=nc)
    exp_cp, exp_ri, exp_vo = oracle.transpose64(rp, ci, vv, n_cols=nc)
    assert np.array_equal(ri.cpu().numpy().view(np.uint64), exp_ri)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), exp_vo.view(np.uint32))
    step = 1 << 27
    for a in range(0, nc + 1, step):
        b = min(a + step, nc + 1)
        assert np.array_equal(cp[a:b].cpu().numpy().view(np.uint64), exp_cp[a:b]), f"col_ptr [{a}, {b})"


def test_u64_more_than_2_32_rows():
    """2^32 + 2^20 + 3 rows (most of them empty), 2^20 columns: the source IDs
    of the edges in rows above 2^32 need 33 bits."""
    from paper_2501_06872_gb300 import binding
    if torch.cuda.get_device_properties(0).total_memory < 150e9:
        pytest.skip("needs a GPU with more than 150 GB")
    avail = _mem_available()
    if avail and avail < 80e9:
        pytest.skip("needs about 70 GB of free host memory")
    nr, nc, m = (1 << 32) + (1 << 20) + 3, 1 << 20, 1 << 22
    rng = np.random.default_rng(642)
    rows = np.unique(np.concatenate([rng.integers(0, nr, 200000, dtype=np.uint64),
                                     (1 << 32) - 2 + np.arange(8, dtype=np.uint64), np.array([nr - 1], np.uint64)]))
    counts = rng.multinomial(m, np.ones(rows.size) / rows.size).astype(np.int64)
    deg = torch.zeros(nr, dtype=torch.int64, device="cuda")
    deg[torch.from_numpy(rows.view(np.int64)).cuda()] = torch.from_numpy(counts).cuda()
    rp_d = torch.zeros(nr + 1, dtype=torch.int64, device="cuda")
    torch.cumsum(deg, 0, out=rp_d[1:])
    del deg
    ci = rng.integers(0, nc, m, dtype=np.uint64)
    cp, ri, _ = binding.transpose_u64(rp_d, _dev64(ci), None, n_cols=nc)
    rp = rp_d.cpu().numpy().view(np.uint64)
    del rp_d
    exp_cp, exp_ri, _ = oracle.transpose64(rp, ci, None, n_cols=nc)
    got_ri = ri.cpu().numpy().view(np.uint64)
    assert np.array_equal(cp.cpu().numpy().view(np.uint64), exp_cp)
    assert np.array_equal(got_ri, exp_ri)
    assert int(got_ri.max()) > (1 << 32)  # 33-bit sources were carried
