"""Pins of the selector oracle (features, MLP, Adam) -- CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import selector as so

HERE = os.path.dirname(os.path.abspath(__file__))


def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) if l.startswith("0x")]
    assert so.stream(0, 3) == vals


def test_scaled_is_floor_of_product():
    for r in [0, 1, (1 << 64) - 1, 0x8000000000000000, 12345678901234567890]:
        for b in [1, 7, 1000, (1 << 32) + 3]:
            assert so.scaled(r, b) == (r * b) // (1 << 64)
            assert 0 <= so.scaled(r, b) < b


def star_in(n):
    # every vertex u >= 1 has one edge u -> 0
    row_ptr = np.concatenate([[0, 0], np.arange(1, n)]).astype(np.int64)
    col_idx = np.zeros(n - 1, dtype=np.int64)
    return row_ptr, col_idx


def test_features_in_star_closed_forms():
    n = 1000
    rp, ci = star_in(n)
    m = n - 1
    f = so.features(n, m, rp, ci, False, 5).astype(np.float64)
    assert f[0] == pytest.approx(1 / n) and f[1] == pytest.approx((n - 1) / n)
    assert f[2:32].sum() == 0
    assert f[32] == pytest.approx(math.log2(n) / 32)
    assert f[33] == pytest.approx(math.log2(m + 1) / 32)
    assert f[34] == pytest.approx(1 / 32)
    # 10 vertices of the 999 in bin 1 (one edge each): 10 edges of 999
    assert f[35] == pytest.approx(10 / m, rel=1e-6)
    assert f[36] == 1.0  # every sample lands on vertex 0
    assert f[37] == pytest.approx(math.log2(m + 1) / 32, rel=1e-6)
    assert f[38] == 0 and f[39] == 0  # no row has two edges
    assert f[40] == 0
    assert so.features(n, m, rp, ci, True, 5)[40] == 1


def test_features_rect_closed_forms():
    # tall: 1000 rows x 4 columns, row u -> column u % 4 (one entry per row)
    nr, nc = 1000, 4
    rp = np.arange(nr + 1, dtype=np.int64)
    ci = np.arange(nr, dtype=np.int64) % nc
    f = so.features(nr, nr, rp, ci, False, 3, n_cols=nc).astype(np.float64)
    assert f[1] == 1.0 and f[0] == 0  # every row has degree 1 (fractions of rows)
    assert f[32] == pytest.approx(math.log2(nc) / 32)  # the column space
    assert f[35] == pytest.approx(10 / nr)  # the ceil(1000/100) = 10 top rows hold 10 entries
    assert f[36] == 1.0  # 4 distinct destinations, all within the top 512
    assert so.sample_count(nc, nr) == 1024
    # wide: 4 rows x 10^6 columns: the sample count follows the columns
    assert so.sample_count(10 ** 6, 4000) == 10000
    rp = np.array([0, 1000, 2000, 3000, 4000], dtype=np.int64)
    ci = (np.arange(4000, dtype=np.int64) * 250) % 10 ** 6
    g = so.features(4, 4000, rp, ci, False, 3, n_cols=10 ** 6).astype(np.float64)
    assert g[32] == pytest.approx(math.log2(10 ** 6) / 32)
    assert g[10] == 1.0  # degree 1000 -> bin 10 for all 4 rows
    assert g[35] == pytest.approx(1000 / 4000)  # ceil(4/100) = 1 top row of 4


def test_features_consecutive_neighbours():
    # u -> u+1, u+2 while u+2 < n: every neighbour pair differs by one
    n = 5000
    rows = [[u + 1, u + 2] if u + 2 < n else [] for u in range(n)]
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([v for r in rows for v in r], dtype=np.int64)
    f = so.features(n, len(ci), rp, ci, False, 9)
    assert f[38] == pytest.approx(1 / 32)
    assert 0.9 < f[39] < 1.0
    assert f[2] == pytest.approx((n - 2) / n)  # degree 2 -> bin 2


def test_features_top_fraction_at_bin_edge():
    # 200 vertices: two of degree 100 (bin 7), 198 of degree 1 -> the top
    # ceil(200/100) = 2 vertices hold exactly 200 of 398 edges
    n = 200
    deg = np.array([100, 100] + [1] * 198)
    rp = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    ci = np.arange(rp[-1]) % n
    f = so.features(n, int(rp[-1]), rp, ci, False, 3)
    assert f[35] == pytest.approx(200 / 398, rel=1e-7)
    assert f[7] == pytest.approx(2 / n) and f[1] == pytest.approx(198 / n)


def test_coverage_matches_counter_brute_force():
    from collections import Counter
    rng = np.random.default_rng(4)
    n, m = 3000, 40000
    ci = (rng.zipf(1.6, size=m) % n).astype(np.int64)
    rp = np.sort(rng.integers(0, m + 1, size=n + 1))
    rp[0], rp[-1] = 0, m
    f = so.features(n, m, rp, ci, False, 11)
    ns = so.sample_count(n, m)
    c = Counter(int(ci[so.scaled(r, m)]) for r in so.stream(11, ns))
    top = sum(v for _, v in c.most_common(512))
    assert f[36] == pytest.approx(top / ns, rel=1e-6)
    assert f[37] == pytest.approx(math.log2(max(c.values()) * m / ns + 1) / 32, rel=1e-6)


def test_empty_graph_features():
    f = so.features(10, 0, np.zeros(11, dtype=np.int64), np.zeros(0, dtype=np.int64), False, 1)
    assert f[0] == 1.0 and f[33] == 0 and f[35] == 0 and f[36] == 0 and f[38] == 0


def small_net(seed, F=5, H=6, K=3, B=9):
    rng = np.random.default_rng(seed)
    lo = so.layout(F, H, K)
    p = rng.normal(size=lo["total"])
    p[lo["sd"][0]:lo["sd"][0] + F] = rng.uniform(0.5, 2.0, size=F)
    X = rng.normal(size=(B, F))
    T = rng.normal(size=(B, K))
    M = (rng.random(size=(B, K)) < 0.8).astype(np.float64)
    return p, X, T, M, lo


def fd_check(backward, seed=0, F=5, H=6, K=3):
    p, X, T, M, lo = small_net(seed, F, H, K)
    _, g = backward(p, X, T, M, F, H, K)
    worst = 0.0
    for i in range(lo["W1"][0], lo["total"]):
        num = five_point(p, i, lambda q: so.loss(q, X, T, M, F, H, K))
        worst = max(worst, abs(num - g[i]) / max(1e-2, abs(num) + abs(g[i])))
    return worst


def five_point(p, i, fn, h=1e-5):
    """Central difference of fourth order: (-f(+2h) + 8 f(+h) - 8 f(-h) + f(-2h)) / 12h."""
    vals = []
    for k in (2, 1, -1, -2):
        q = p.copy()
        q[i] += k * h
        vals.append(fn(q))
    return (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)


def test_backward_matches_central_differences():
    for seed in range(3):
        assert fd_check(so.backward, seed) < 1e-6


def test_full_size_backward_spot_check():
    rng = np.random.default_rng(1)
    lo = so.layout()
    p = rng.normal(scale=0.2, size=lo["total"])
    p[lo["sd"][0]:lo["sd"][0] + so.N_FEATURES] = 1.0
    X = rng.normal(size=(16, so.N_FEATURES))
    T = rng.normal(size=(16, so.GRID))
    M = np.ones((16, so.GRID))
    _, g = so.backward(p, X, T, M)
    for i in rng.choice(np.arange(lo["W1"][0], lo["total"]), size=60, replace=False):
        num = five_point(p, i, lambda q: so.loss(q, X, T, M))
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num))


def test_planted_mistake_is_caught():
    """A backward pass that drops the second ReLU mask fails the pin."""
    def bad_backward(p, X, T, M, F, H, K):
        mu, sd, W1, b1, W2, b2, W3, b3 = so.unpack(p, F, H, K)
        y, (xn, a1, h1, a2, h2) = so.forward(p, X, F, H, K)
        den = max(1.0, M.sum())
        dy = 2.0 * M * (y - T) / den
        da2 = dy @ W3  # mask dropped
        da1 = (da2 @ W2) * (a1 > 0)
        lo = so.layout(F, H, K)
        g = np.zeros(lo["total"])
        for name, arr in (("W1", da1.T @ xn), ("b1", da1.sum(0)), ("W2", da2.T @ h1), ("b2", da2.sum(0)),
                          ("W3", dy.T @ h2), ("b3", dy.sum(0))):
            o, s = lo[name]
            g[o:o + s] = arr.reshape(-1)
        return 0.0, g
    assert fd_check(bad_backward, 0) > 1e-2


def test_masked_entries_do_not_contribute():
    p, X, T, M, lo = small_net(2)
    T2 = T.copy()
    T2[M == 0] += 100.0
    assert so.loss(p, X, T, M, 5, 6, 3) == pytest.approx(so.loss(p, X, T2, M, 5, 6, 3))


def test_zero_weights_give_bias_and_bias_gradient():
    p, X, T, M, lo = small_net(3)
    p[lo["W3"][0]:lo["W3"][0] + lo["W3"][1]] = 0.0
    y, _ = so.forward(p, X, 5, 6, 3)
    b3 = p[lo["b3"][0]:lo["b3"][0] + 3]
    assert np.allclose(y, b3)
    _, g = so.backward(p, X, T, M, 5, 6, 3)
    expect = (2 * M * (b3 - T)).sum(0) / max(1.0, M.sum())
    assert np.allclose(g[lo["b3"][0]:lo["b3"][0] + 3], expect)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    z = np.zeros(50)
    lr, eps = 1e-2, 1e-8
    p1, m1, m2 = so.adam(p, g, z, z, 1, lr, eps=eps)
    # step 1: bias-corrected moments are g and g^2
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    p2, _, _ = so.adam(p, g, z, z, 1, lr, first=10)
    assert np.array_equal(p2[:10], p[:10])
    # with an L2 penalty the step-1 direction is that of g + wd * p
    wd = 0.3
    p3, _, _ = so.adam(p, g, z, z, 1, lr, eps=eps, wd=wd)
    gw = g + wd * p
    assert np.allclose(p3, p - lr * gw / (np.abs(gw) + eps), rtol=0, atol=1e-15)


def test_shipped_selector_report_reproduces_in_fp64():
    """The committed report's held-out regret follows from the committed
    parameters and dataset through the fp64 oracle forward pass."""
    import json
    import paper_2501_06872_gb300 as pkg
    root = os.path.dirname(pkg.__file__)
    d = np.load(os.path.join(root, "selector_dataset.npz"), allow_pickle=False)
    rep = json.load(open(os.path.join(root, "selector_report.json")))
    p = np.fromfile(os.path.join(root, "selector_params.f32"), dtype="<f4").astype(np.float64)
    assert p.size == so.layout()["total"]
    n_train = rep["n_train"]
    from paper_2501_06872_gb300 import selector_train as st
    t_all = st.merge_equivalent(d["times"], json.loads(str(d["meta"])))
    f, t = d["features"][n_train:].astype(np.float64), t_all[n_train:]
    y, _ = so.forward(p, f)
    idx = y.argmin(axis=1)
    # outside the trained range (widened by 5 % of its width) the analytic choice stands
    lo_o, hi_o = so.layout()["lo"][0], so.layout()["hi"][0]
    lo, hi = p[lo_o:lo_o + so.N_FEATURES], p[hi_o:hi_o + so.N_FEATURES]
    pad = 0.05 * (hi - lo) + 1e-6
    f32 = d["features"][n_train:]
    out = ((f32 < lo - pad) | (f32 > hi + pad)).any(axis=1)
    meta = json.loads(str(d["meta"]))[n_train:]
    idx = np.where(out, np.array([m["analytic"] for m in meta]), idx)
    best = np.where(t > 0, t, np.inf).min(axis=1)
    reg = t[np.arange(len(idx)), idx] / best
    assert reg.mean() == pytest.approx(rep["test"]["learned"]["mean"], rel=1e-6)


def test_trainer_targets_and_regret_helpers():
    """Log-regret targets are 0 at the best grid point and ln(t/t_best)
    elsewhere, masked where a point was not timed; regret is t_pick/t_best."""
    from paper_2501_06872_gb300 import selector_train as st
    times = np.array([[2.0, 1.0, 4.0, -1.0], [3.0, 6.0, 3.0, 1.5]])
    y, m = st.targets(times)
    assert np.allclose(y[0], [math.log(2.0), 0.0, math.log(4.0), 0.0])
    assert np.allclose(m, [[1, 1, 1, 0], [1, 1, 1, 1]])
    assert np.allclose(y[1], [math.log(2.0), math.log(4.0), math.log(2.0), 0.0])
    r = st.regrets(times, np.array([2, 3]))
    assert np.allclose(r, [4.0, 1.0])
    s = st.summary(r)
    assert s["mean"] == pytest.approx(2.5) and s["max"] == 4.0 and s["optimal_share"] == 0.5
    mu, sd = st.standardise(np.array([[1.0, 5.0], [3.0, 5.0]]))
    assert np.allclose(mu, [2.0, 5.0]) and np.allclose(sd, [1.001, 0.001])


def test_trainer_graph_specs_follow_the_stated_ranges():
    from paper_2501_06872_gb300 import selector_train as st
    specs = [st.graph_spec(i) for i in range(256)]
    assert all(0.25 <= s["a"] <= 0.70 for s in specs)
    assert all(abs(s["b"] - (1 - s["a"] - 0.05) / 2) < 1e-12 and s["b"] == s["c"] for s in specs)
    assert {s["scale"] for s in specs} <= set(range(18, 29)) and 28 in {s["scale"] for s in specs}
    assert all(8 <= s["edge_factor"] <= 32 and s["edge_factor"] << s["scale"] <= 1 << 32 for s in specs)
    assert {s["order"] for s in specs} == {"degree", "random"}
    assert specs[3] == st.graph_spec(3)  # seeded


def test_forward_hand_worked_2_3_2_network():
    """A 2-3-2 network with small integer weights, worked out by hand (the
    values below are not computed by any code).  The parameter vector is laid
    out in the documented order mu, sd, lo, hi, W1 (rows = hidden units), b1,
    W2, b2, W3, b3.  A transposed W2, a missing standardisation, a missing
    ReLU in either layer or a wrong bias would each change the outputs.

    sample 1: x = (3, 0) -> x' = ((3-1)/2, (0+1)/1) = (1, 1)
      a1 = (1+2+0, -3+1+1, 0-1+2) = (3, -1, 1) -> h1 = (3, 0, 1)
      a2 = (3+1-1, 0+0, -3+0-9) = (3, 0, -12) -> h2 = (3, 0, 0)
      y  = (3+0.5, 6+1) = (3.5, 7)
    sample 2: x = (-1, -1) -> x' = (-1, 0)
      a1 = (-1+0, 3+1, 0+2) = (-1, 4, 2) -> h1 = (0, 4, 2)
      a2 = (2-1, 8+0, 4-9) = (1, 8, -5) -> h2 = (1, 8, 0)
      y  = (1+8+0.5, 2+1) = (9.5, 3)
    """
    mu, sd = [1.0, -1.0], [2.0, 1.0]
    lo, hi = [0.0, 0.0], [1.0, 1.0]
    W1 = [1.0, 2.0, -3.0, 1.0, 0.0, -1.0]
    b1 = [0.0, 1.0, 2.0]
    W2 = [1.0, 0.0, 1.0, 0.0, 2.0, 0.0, -1.0, 1.0, 0.0]
    b2 = [-1.0, 0.0, -9.0]
    W3 = [1.0, 1.0, 1.0, 2.0, 0.0, -3.0]
    b3 = [0.5, 1.0]
    p = np.array(mu + sd + lo + hi + W1 + b1 + W2 + b2 + W3 + b3)
    assert so.layout(2, 3, 2)["total"] == p.size == 37
    y, _ = so.forward(p, np.array([[3.0, 0.0], [-1.0, -1.0]]), 2, 3, 2)
    assert np.array_equal(y, np.array([[3.5, 7.0], [9.5, 3.0]]))
