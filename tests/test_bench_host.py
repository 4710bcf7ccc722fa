"""Host-side logic of bench.py that needs no GPU: the traffic record taken
from an ncu CSV, the metric-formula bytes, the digit-pass byte count and the
workload table (rectangular folds, CSC direction)."""
import json
import os

import numpy as np
import pytest

import bench


def _fake_csv(path, kernel, launches):
    lines = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    for i, (rd, wr) in enumerate(launches):
        lines.append(f'"{i}","{kernel}(RadixArgs)","dram__bytes_read.sum","Gbyte","{rd}"')
        lines.append(f'"{i}","{kernel}(RadixArgs)","dram__bytes_write.sum","Mbyte","{wr}"')
        lines.append(f'"{i}","{kernel}(RadixArgs)","gpu__time_duration.sum","msecond","1.0"')
    lines.append('"9","k_other(X)","dram__bytes_read.sum","Gbyte","1000"')
    path.write_text("==PROF== noise line\n" + "\n".join(lines) + "\n")


def test_record_traffic_averages_launches_and_stamps_the_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"other@w": {"x": 1}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_2501_06872_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "include").mkdir()
    real = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    for f in bench.KERNEL_SOURCES["k_radix_down_bulk"]:
        (csrc / f).write_bytes(open(os.path.join(real, "paper_2501_06872_gb300", "csrc", f), "rb").read())
    (tmp_path / "include" / "gt.h").write_bytes(open(os.path.join(real, "include", "gt.h"), "rb").read())
    csv_path = tmp_path / "d.csv"
    _fake_csv(csv_path, "k_radix_down_bulk", [(2.0, 500.0), (4.0, 1500.0)])
    bench.record_traffic(str(csv_path), "k_radix_down_bulk", "wl", "note")
    d = json.load(open(prof / "traffic.json"))
    e = d["k_radix_down_bulk@wl"]
    assert d["other@w"] == {"x": 1}
    assert e["launches"] == 2
    assert e["dram_bytes_per_launch"] == pytest.approx((2.5e9 + 5.5e9) / 2)
    assert e["source_sha"] == bench.kernel_source_sha("k_radix_down_bulk")
    assert bench.load_traffic("k_radix_down_bulk", "wl") == pytest.approx(4.0e9)
    (csrc / "gt_radix.cu").write_text("changed")  # a changed kernel voids the record
    assert bench.load_traffic("k_radix_down_bulk", "wl") is None


def test_metric_bytes_and_pass_bytes():
    lit, withv = bench.algorithmic_bytes(4, 10, True)
    assert lit == 2 * 40 + 8 * 5 + 40 + 40 + 8 * 5 and withv == lit + 40
    lit_r, _ = bench.algorithmic_bytes(4, 10, False, n_cols=9)
    assert lit_r == 2 * 40 + 8 * 5 + 40 + 8 * 10
    assert bench.radix_passes(1 << 28) == 4 and bench.radix_passes(1 << 20) == 3 and bench.radix_passes(2) == 1
    # first pass 20 B/edge (weighted: col_idx + vals in, key + source + value out), later ones 24
    assert bench.radix_down_bytes_per_edge(True, 4) == pytest.approx((20 + 3 * 24) / 4)
    assert bench.radix_down_bytes_per_edge(False, 1) == pytest.approx(12)


def test_workload_table():
    for name, (rs, cs) in bench.FOLDS.items():
        kind, scale, ef, order, weighted = bench.WORKLOADS[name]
        assert 0 <= rs < scale and 0 <= cs < scale
    c = bench.workload_config("rmat28-tall", 1 << 28, 1 << 32, True, 1 << 20)
    assert c["n_rows"] == 1 << 28 and c["n_cols"] == 1 << 20 and "2^8" in c["fold"]
    c = bench.workload_config("rmat25-random", 1 << 25, 1 << 29, False, 1 << 25, "csc")
    assert c["direction"] == "CSC input -> CSR" and "n_cols" not in c


def test_sample_rows_keeps_whole_rows_at_spread_starts():
    import bench
    rng = np.random.default_rng(3)
    n = 1000
    deg = rng.integers(0, 20, n).astype(np.uint64)
    rp = np.zeros(n + 1, np.uint64)
    np.cumsum(deg, out=rp[1:])
    m = int(rp[-1])
    ci = rng.integers(0, n, m).astype(np.uint32)
    vv = rng.random(m).astype(np.float32)
    rp_s, ci_s, vv_s, mS, rows, desc = bench.sample_rows(rp, lambda a, b: ci[a:b], lambda a, b: vv[a:b], 400,
                                                         windows=4)
    assert rp_s.size == n + 1 and rp_s[0] == 0 and int(rp_s[-1]) == mS == ci_s.size == vv_s.size
    kept = np.nonzero(np.diff(rp_s) > 0)[0]
    # every kept row is whole and in place; the four runs start at k * n / 4
    for u in kept:
        a, b = int(rp_s[u]), int(rp_s[u + 1])
        assert np.array_equal(ci_s[a:b], ci[int(rp[u]):int(rp[u + 1])])
        assert np.array_equal(vv_s[a:b], vv[int(rp[u]):int(rp[u + 1])])
    starts = [k * n // 4 for k in range(4)]
    assert all(np.diff(rp_s)[s] == rp[s + 1] - rp[s] for s in starts)
    assert 300 <= mS <= 400 + 4 * 20


def test_roofline_uses_the_method_bytes_per_call():
    import bench
    from types import SimpleNamespace
    cfg = SimpleNamespace(method=1, radix_tile=0)
    n, m = 1 << 10, 1 << 14
    timing = {"dominant_ms": 2.0, "dominant_launches": 8, "calls": 2}
    r = bench.roofline(cfg, timing, n, n, m, True, 1000.0, "measured", "no-such-workload")
    lit, withv = bench.algorithmic_bytes(n, m, True)
    assert r["launches_per_call"] == 4
    assert r["achieved"] == pytest.approx(lit / 8e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    assert r["frac_with_vals_read"] == pytest.approx(withv / 8e-3 / 1e9 / 1000.0)
    own = bench.radix_down_bytes_per_edge(True, bench.radix_passes(n)) * m + 8 * (n + 1) / bench.radix_passes(n)
    assert r["kernel_own"]["bytes_per_launch"] == int(own)
    assert r["traffic"] is None and r["dram_over_algorithmic"] is None


def test_step3_imbalance_summary():
    import bench
    r = bench.step3_imbalance([1.0, 1.0, 2.0, 0.0])
    assert r["partitions"] == 4 and r["idle_share"] == pytest.approx(1 - 1.0 / 2.0)
    assert r["cv"] == pytest.approx(np.std([1, 1, 2, 0]) / 1.0)
    assert bench.step3_imbalance([]) is None


def test_partition_bits_keep_ranges_of_at_most_2_20_columns():
    """The two-level form's bucket width: destination ranges of 2^20 columns,
    between 1 and 8 bits (one digit pass)."""
    assert bench.partition_bits_for(1 << 28) == 8
    assert bench.partition_bits_for(1 << 24) == 4
    assert bench.partition_bits_for((1 << 24) + 1) == 5
    assert bench.partition_bits_for(1 << 20) == 1
    assert bench.partition_bits_for(1000) == 1
    assert bench.partition_bits_for(1 << 32) == 8
    for n in (1 << 21, 3 << 22, 1 << 26):
        d = bench.partition_bits_for(n)
        assert (n - 1) >> d < (1 << 20) or d == 8
