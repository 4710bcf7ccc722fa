"""GPU: graph features, selector MLP kernels and the autotuner against the
oracle.  Features and the MLP are f32 on the device against the fp64 oracle
(within f32 tolerance); every configuration the search can install must give
the oracle's CSC bit for bit."""
import os

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


def dev(rp, ci, vv=None):
    d = torch.device("cuda:0")
    return (torch.from_numpy(np.ascontiguousarray(rp).view(np.int64)).to(d),
            torch.from_numpy(np.ascontiguousarray(ci, dtype=np.uint32).view(np.int32)).to(d),
            None if vv is None else torch.from_numpy(np.ascontiguousarray(vv, dtype=np.float32)).to(d))


def graphs():
    out = []
    n, rp, ci, vv = inputs.rmat_csr(13, 16, seed=5, order="random", weighted=True)
    out.append(("rmat13-random", n, rp, ci, vv))
    n, rp, ci, vv = inputs.rmat_csr(12, 8, seed=6, order="degree", weighted=False)
    out.append(("rmat12-degree", n, rp, ci, None))
    n, rp, ci, vv = inputs.er_csr(5000, 60000, seed=2)
    out.append(("er", n, rp, ci, None))
    n = 1000
    out.append(("in-star", n, np.concatenate([[0, 0], np.arange(1, n)]).astype(np.uint64),
                np.zeros(n - 1, dtype=np.uint32), None))
    n = 300
    rows = [[u + 1, u + 2] if u + 2 < n else [] for u in range(n)]
    rp = np.zeros(n + 1, dtype=np.uint64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    out.append(("consecutive", n, rp, np.array([v for r in rows for v in r], dtype=np.uint32), None))
    out.append(("empty", 7, np.zeros(8, dtype=np.uint64), np.zeros(0, dtype=np.uint32), None))
    # 7 M vertices: ~70,000 samples all on vertex 0 (a frequency >= 2^16, listed exactly)
    n = 7_000_000
    rp = np.minimum(np.arange(n + 1, dtype=np.uint64), 1000).astype(np.uint64)
    out.append(("hub-7M", n, rp, np.zeros(1000, dtype=np.uint32), None))
    return out


@pytest.mark.parametrize("idx", range(7))
def test_features_match_oracle(idx):
    from paper_2501_06872_gb300 import binding
    name, n, rp, ci, vv = graphs()[idx]
    seed = 0x1234 + idx
    rpd, cid, _ = dev(rp, ci)
    got = binding.graph_features(rpd, cid, vv is not None, seed=seed).cpu().numpy()
    exp = so.features(n, len(ci), rp.astype(np.int64), ci.astype(np.int64), vv is not None, seed)
    np.testing.assert_allclose(got, exp, rtol=2e-6, atol=1e-7, err_msg=name)


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    lo = so.layout()
    p = rng.normal(scale=scale, size=lo["total"]).astype(np.float32)
    F = so.N_FEATURES
    p[F:2 * F] = rng.uniform(0.5, 2.0, size=F)
    return p


def test_forward_backward_adam_match_oracle():
    from paper_2501_06872_gb300 import binding
    rng = np.random.default_rng(3)
    B = 37
    p = random_params(1)
    X = rng.normal(size=(B, so.N_FEATURES)).astype(np.float32)
    T = rng.normal(size=(B, so.GRID)).astype(np.float32)
    M = (rng.random(size=(B, so.GRID)) < 0.85).astype(np.float32)
    sel = binding.Selector(p)
    assert sel.n_params == so.layout()["total"]
    Xd, Td, Md = (torch.from_numpy(a).cuda() for a in (X, T, M))
    y = sel.forward(Xd).cpu().numpy()
    ye, _ = so.forward(p, X)
    np.testing.assert_allclose(y, ye, rtol=1e-4, atol=1e-4 * np.abs(ye).max())
    loss = torch.zeros(1, device="cuda")
    g = torch.zeros(sel.n_params, device="cuda")
    sel.backward(Xd, Td, Md, loss=loss, grads=g)
    Le, ge = so.backward(p, X, T, M)
    assert float(loss.item()) == pytest.approx(Le, rel=1e-4)
    g = g.cpu().numpy()
    np.testing.assert_allclose(g, ge, rtol=1e-3, atol=1e-4 * np.abs(ge).max())
    # one Adam step from zero moments, then a second one
    lr = 1e-2
    sel.adam_step(lr=lr)
    first = so.layout()["W1"][0]
    pe, m1, m2 = so.adam(p, g, np.zeros_like(ge), np.zeros_like(ge), 1, lr, first=first)
    np.testing.assert_allclose(sel.params(), pe, rtol=1e-5, atol=1e-6)
    sel.backward(Xd, Td, Md, grads=(g2 := torch.zeros(sel.n_params, device="cuda")))
    sel.adam_step(lr=lr, weight_decay=0.05)  # the second step with an L2 penalty
    pe2, _, _ = so.adam(pe, g2.cpu().numpy(), m1, m2, 2, lr, first=first, wd=0.05)
    np.testing.assert_allclose(sel.params(), pe2, rtol=1e-5, atol=1e-5)
    sel.close()


def test_training_reduces_loss():
    from paper_2501_06872_gb300 import binding
    rng = np.random.default_rng(8)
    B = 128
    X = rng.normal(size=(B, so.N_FEATURES)).astype(np.float32)
    W = rng.normal(size=(so.N_FEATURES, so.GRID)).astype(np.float32) * 0.3
    T = np.maximum(X @ W, 0).astype(np.float32)
    M = np.ones_like(T)
    sel = binding.Selector(seed=5)
    Xd, Td, Md = (torch.from_numpy(a).cuda() for a in (X, T, M))
    loss = torch.zeros(1, device="cuda")
    sel.backward(Xd, Td, Md, loss=loss)
    l0 = float(loss.item())
    for _ in range(400):
        sel.backward(Xd, Td, Md, loss=loss)
        sel.adam_step(lr=3e-3)
    sel.backward(Xd, Td, Md, loss=loss)
    assert float(loss.item()) < 0.1 * l0
    sel.close()


def test_every_grid_point_gives_oracle_bytes():
    from paper_2501_06872_gb300 import binding
    n, rp, ci, vv = inputs.rmat_csr(14, 16, seed=9, order="random", weighted=True)
    exp = oracle.transpose(rp, ci, vv)
    rpd, cid, vvd = dev(rp, ci, vv)
    m = len(ci)
    plan = binding.Plan(n, m, True)
    for i in range(binding.TUNE_GRID):
        plan.set_config(binding.grid_config(i, n, m))
        cp = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
        ri = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        vo = torch.full((m,), -1.0, dtype=torch.float32, device="cuda")
        plan.transpose(rpd, cid, vvd, cp, ri, vo)
        plan.check()
        assert np.array_equal(cp.cpu().numpy().view(np.uint64), exp[0]), i
        assert np.array_equal(ri.cpu().numpy().view(np.uint32), exp[1]), i
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), exp[2].view(np.uint32)), i
    plan.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_tune_modes_install_a_config_and_keep_bytes(mode):
    from paper_2501_06872_gb300 import binding
    n, rp, ci, vv = inputs.rmat_csr(15, 12, seed=10, order="degree", weighted=True)
    exp = oracle.transpose(rp, ci, vv)
    rpd, cid, vvd = dev(rp, ci, vv)
    m = len(ci)
    cp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(m, dtype=torch.int32, device="cuda")
    vo = torch.empty(m, dtype=torch.float32, device="cuda")
    plan = binding.Plan(n, m, True)
    sel = binding.Selector(seed=3) if mode == binding.TUNE_LEARNED else None
    idx, table = plan.tune(mode, rpd, cid, vvd, cp, ri, vo, selector=sel, reps=2)
    assert 0 <= idx < binding.TUNE_GRID
    got = plan.config().as_dict()
    want = binding.grid_config(idx, n, m).as_dict()
    assert got == want
    if mode == binding.TUNE_EXHAUSTIVE:
        ms = np.array([t["ms"] for t in table])
        assert (ms > 0).all() and all(t["status"] == 0 for t in table)
        assert ms[idx] == ms.min()
    if mode == binding.TUNE_LEARNED:
        sc = np.array([t["score"] for t in table])
        assert idx == int(np.argmin(sc))
    plan.transpose(rpd, cid, vvd, cp, ri, vo)
    plan.check()
    assert np.array_equal(ri.cpu().numpy().view(np.uint32), exp[1])
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), exp[2].view(np.uint32))
    plan.close()
    if sel is not None:
        sel.close()


def test_tune_reports_bad_input():
    from paper_2501_06872_gb300 import binding
    n = 64
    rp = np.arange(0, 2 * n + 1, 2, dtype=np.uint64)
    ci = (np.arange(2 * n) % n).astype(np.uint32)
    ci[17] = n + 5
    rpd, cid, _ = dev(rp, ci)
    cp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(2 * n, dtype=torch.int32, device="cuda")
    plan = binding.Plan(n, 2 * n, False)
    with pytest.raises(binding.GtError) as e:
        plan.tune(binding.TUNE_EXHAUSTIVE, rpd, cid, None, cp, ri, None, reps=1)
    assert e.value.code == 2
    plan.close()


def _heldout():
    import json
    import paper_2501_06872_gb300 as pkg
    root = os.path.dirname(pkg.__file__)
    d = np.load(os.path.join(root, "selector_dataset.npz"), allow_pickle=False)
    rep = json.load(open(os.path.join(root, "selector_report.json")))
    meta = json.loads(str(d["meta"]))
    n_train = rep["n_train"]
    from paper_2501_06872_gb300 import selector_train as st
    times = st.merge_equivalent(d["times"], meta)  # points that run the same kernels share one time
    return d["features"][n_train:], times[n_train:], meta[n_train:], rep


def _regret(times, idx):
    best = np.where(times > 0, times, np.inf).min(axis=1)
    return times[np.arange(len(idx)), idx] / best


def test_trained_selector_gains_over_the_method_without_it():
    """On the 64 held-out graphs (timed by the exhaustive autotuner), the
    trained network's picks, run through the library's forward kernels, have
    a lower mean regret than the default configuration (the method without
    the selector) and than the analytic model."""
    from paper_2501_06872_gb300 import binding
    feats, times, meta, rep = _heldout()
    sel = binding.Selector.pretrained()
    scores = sel.forward(torch.from_numpy(feats.astype(np.float32)).cuda()).cpu().numpy()
    an = np.array([m["analytic"] for m in meta])
    pick = np.array([scores[i].argmin() if sel.in_range(feats[i]) else an[i] for i in range(len(feats))])
    sel.close()
    learned = _regret(times, pick).mean()
    default = _regret(times, np.array([m["default"] for m in meta])).mean()
    analytic = _regret(times, an).mean()
    assert learned == pytest.approx(rep["test"]["learned"]["mean"], rel=1e-6)
    assert learned < default
    assert learned < analytic
    # summed over the held-out graphs, the learned picks take less time than the analytic ones
    rows = np.arange(len(pick))
    assert times[rows, pick].sum() < times[rows, an].sum()
