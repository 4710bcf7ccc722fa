"""Benchmark: CSR -> CSC transposition on one GB300 (or N replicas under torchrun).

One step = one gt_transpose call (sampling, count, scan, scatter, LDV sort)
over the resident workload.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "transposed edges/s & HBM GB/s vs peak; batched/learned vs plain on one GB300"
UNIT = "edges/s"

# name -> (kind, scale, edge_factor, order, weighted)
WORKLOADS = {
    "rmat28-degree": ("rmat", 28, 16, "degree", True),
    "rmat28-random": ("rmat", 28, 16, "random", True),
    "rmat24-random": ("rmat", 24, 16, "random", False),
    "rmat24-random-weighted": ("rmat", 24, 16, "random", True),
    "er24-random": ("er", 24, 16, "random", False),
    "rmat16": ("rmat", 16, 16, "natural", False),
    "rmat20-degree": ("rmat", 20, 16, "degree", True),
    "rmat22-degree": ("rmat", 22, 16, "degree", True),
    "rmat23-degree": ("rmat", 23, 16, "degree", True),
    "rmat24-degree": ("rmat", 24, 16, "degree", True),
    "rmat25-degree": ("rmat", 25, 16, "degree", True),
    "rmat26-degree": ("rmat", 26, 16, "degree", True),
    "rmat27-degree": ("rmat", 27, 16, "degree", True),
    "rmat26-random": ("rmat", 26, 16, "random", True),
    # rectangular sparse matrices from the scale-28 graph: rows merged by 2^r, columns by 2^c
    "rmat28-tall": ("rmat", 28, 16, "degree", True),   # 2^28 rows x 2^20 columns
    "rmat28-wide": ("rmat", 28, 16, "degree", True),   # 2^20 rows x 2^28 columns
    "rmat24-tall": ("rmat", 24, 16, "degree", True),   # 2^24 rows x 2^16 columns
    # the paper's representations (Sec. V-A): generated ("natural") and randomised IDs, with --direction csr|csc
    "rmat25-natural": ("rmat", 25, 16, "natural", False),
    "rmat25-random": ("rmat", 25, 16, "random", False),
}
FOLDS = {"rmat28-tall": (0, 8), "rmat28-wide": (8, 0), "rmat24-tall": (0, 8)}
SEED = 0x5EED0003


def make_workload(name, seed, direction="csr"):
    """(n_rows, n_cols, row_ptr, col_idx, vals) of a workload, on the GPU.
    direction "csc": the input is the graph's CSC (in-lists in ascending
    source order, parallel edges in CSR order, built by a stable torch sort),
    so the call transposes CSC -> CSR (the paper's CSC representations)."""
    import torch
    from paper_2501_06872_gb300.inputs import gpu as ggen
    kind, scale, ef, order, weighted = WORKLOADS[name]
    n, rp, ci, vv = ggen.graph(scale, ef, kind=kind, seed=seed, order=order, weighted=weighted)
    rs, cs = FOLDS.get(name, (0, 0))
    nr = nc = n
    if rs or cs:
        nr, nc, rp, ci = ggen.fold_rect(rp, ci, rs, cs)
    if direction == "csc":
        src = torch.repeat_interleave(torch.arange(nr, dtype=torch.int64, device=rp.device), rp.diff())
        key = (ci.to(torch.int64) << 32) | src
        del src
        key, perm = torch.sort(key, stable=True)
        cp = torch.zeros(nc + 1, dtype=torch.int64, device=rp.device)
        torch.cumsum(torch.bincount(key >> 32, minlength=nc), 0, out=cp[1:])
        ci = (key & 0xFFFFFFFF).to(torch.int32)
        del key
        vv = None if vv is None else vv[perm]
        del perm
        torch.cuda.synchronize()
        return nc, nr, cp, ci, vv
    return nr, nc, rp, ci, vv


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# sources each timed kernel is built from (a committed DRAM-byte figure is
# used only while these files are unchanged)
KERNEL_SOURCES = {
    "k_radix_down_bulk": ["gt_radix.cu", "gt_device.cuh", "gt_internal.h"],
    "k_radix_down": ["gt_radix.cu", "gt_device.cuh", "gt_internal.h"],
    "k_scatter": ["gt_steps.cu", "gt_device.cuh", "gt_internal.h"],
}


def kernel_source_sha(kernel):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2501_06872_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "gt.h"), "rb").read())
    return h.hexdigest()[:16]


def record_traffic(csv_path, kernel, workload, note, scale=1.0):
    """Writes profiles/traffic.json's entry for (kernel, workload) from an ncu
    --csv capture of dram__bytes_read.sum and dram__bytes_write.sum (one or
    more launches of the kernel): their per-launch average times `scale` (a
    smaller case's capture scaled to the workload by the edges a launch
    processes), stamped with the hash of the kernel's current sources."""
    import csv
    rows = [r for r in csv.reader(line for line in open(csv_path) if line.startswith('"'))]
    h = rows[0]
    ki, mi, ui, vi = h.index("ID"), h.index("Metric Name"), h.index("Metric Unit"), h.index("Metric Value")
    ni = h.index("Kernel Name")
    units = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    per = {}
    for r in rows[1:]:
        if kernel in r[ni] and r[mi].startswith("dram__bytes"):
            per[r[ki]] = per.get(r[ki], 0.0) + float(r[vi].replace(",", "")) * units[r[ui]]
    if not per:
        raise SystemExit(f"no dram__bytes rows for {kernel} in {csv_path}")
    vals = [v * scale for v in per.values()]
    out = os.path.join(ROOT, "profiles", "traffic.json")
    d = json.load(open(out)) if os.path.exists(out) else {}
    d[f"{kernel}@{workload}"] = {"dram_bytes_per_launch": sum(vals) / len(vals), "launches": len(vals),
                                 "per_launch": vals, "scale": scale, "source_sha": kernel_source_sha(kernel),
                                 "capture": note}
    with open(out, "w") as fh:
        json.dump(d, fh, indent=1)
    print(json.dumps(d[f"{kernel}@{workload}"]))


def load_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(f"{kernel}@{workload}")
        if e and e.get("source_sha") == kernel_source_sha(kernel):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def algorithmic_bytes(n, m, weighted, n_cols=None):
    """Bytes the transposition must move (formula of the metric): 2 x col_idx read +
    row_ptr read + row_idx (+ vals_out) write + col_ptr write; plus, separately,
    the vals read.  n: rows (row_ptr), n_cols: columns (col_ptr), default n."""
    nc = n if n_cols is None else n_cols
    literal = 2 * 4 * m + 8 * (n + 1) + 4 * m + (4 * m if weighted else 0) + 8 * (nc + 1)
    with_vals = literal + (4 * m if weighted else 0)
    return literal, with_vals


def stage_bytes(n, m, weighted):
    """Algorithmic bytes per launch of each step's kernels."""
    w = 4 * m if weighted else 0
    return {
        "count": 4 * m + 4 * n,                       # col_idx read, degrees written
        "scan": 4 * n + 8 * (n + 1),                  # degrees read, col_ptr written
        "scatter": 4 * m + w + 8 * (n + 1) + 4 * m + w,  # col_idx, vals, row_ptr read; row_idx, vals_out written
    }


def radix_passes(n):
    bits = max(1, (n - 1).bit_length())
    return (bits + 7) // 8


def radix_down_bytes_per_edge(weighted, passes):
    """Average algorithmic bytes per edge of one downsweep launch: the first
    reads col_idx (+vals) and writes key, source (+value); later passes read
    and write key, source (+value)."""
    w = 4 if weighted else 0
    first = (4 + w) + (8 + w)
    later = 2 * (8 + w)
    return (first + later * (passes - 1)) / passes


def dominant_kernel(cfg, n_cols, m, weighted):
    """(name, own algorithmic bytes per launch) of the kernel that dominates a call."""
    if cfg.method == 1:
        # the bulk-staged downsweep runs when radix_tile is 0 and every array is 16-byte aligned (torch's are)
        name = "k_radix_down_bulk" if cfg.radix_tile == 0 else "k_radix_down"
        passes = radix_passes(n_cols)
        return name, int(radix_down_bytes_per_edge(weighted, passes) * m + 8 * (n_cols + 1) / passes)
    return "k_scatter", stage_bytes(n_cols, m, weighted)["scatter"]


def roofline(cfg, timing, n, n_cols, m, weighted, peak, peak_kind, workload):
    """Roofline of the dominant kernel on the METHOD's algorithmic bytes: the
    metric formula's bytes per call (2 x col_idx read + row_ptr read + row_idx
    (+ vals_out) write + col_ptr write; a second figure adds the vals read)
    over the time the dominant kernel's launches take per call (its average
    CUDA-event launch duration x launches per call).  kernel_own: the same
    kernel on the bytes it moves itself per launch.  traffic: ncu DRAM bytes
    per launch (committed summary, only while the kernel's sources are
    unchanged)."""
    name, own_bytes = dominant_kernel(cfg, n_cols, m, weighted)
    lit, withv = algorithmic_bytes(n, m, weighted, n_cols)
    dom_ms = timing["dominant_ms"]
    per_call = timing["dominant_launches"] / max(1, timing["calls"])
    call_ms = dom_ms * per_call
    ach = lit / (call_ms * 1e-3) / 1e9
    own = own_bytes / (dom_ms * 1e-3) / 1e9
    traffic = load_traffic(name, workload)
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": traffic, "kernel": name, "launch_ms": dom_ms, "launches_per_call": per_call,
            "launches_timed": timing["dominant_launches"], "peak_kind": peak_kind,
            "algorithmic_bytes_per_call": lit, "algorithmic_bytes_per_call_with_vals_read": withv,
            "frac_with_vals_read": withv / (call_ms * 1e-3) / 1e9 / peak,
            "kernel_own": {"bytes_per_launch": own_bytes, "achieved": own, "frac": own / peak},
            "dram_over_algorithmic": (traffic * per_call / lit) if traffic else None}


def sample_rows(rp_h, ci_h_fn, vv_h_fn, target_edges, windows=16):
    """A bounded, representative sample of a workload for the host-side oracle:
    `windows` runs of consecutive rows starting at evenly spaced rows
    (k * n / windows), each holding about target_edges / windows edges; every
    other row is left empty.  ci_h_fn(a, b) / vv_h_fn(a, b) return the host
    copies of col_idx / vals over [a, b).  Returns (row_ptr, col_idx, vals,
    edges, rows, description); the sample keeps all n rows and all columns."""
    n = rp_h.size - 1
    per = max(1, target_edges // windows)
    spans, rows = [], 0
    for k in range(windows):
        r0 = (k * n) // windows
        r1 = int(np.searchsorted(rp_h, rp_h[r0] + np.uint64(per), side="left"))
        r1 = max(r0 + 1, min(r1, ((k + 1) * n) // windows, n))
        spans.append((r0, r1))
        rows += r1 - r0
    deg = np.zeros(n, dtype=np.uint64)
    cis, vvs = [], []
    for r0, r1 in spans:
        deg[r0:r1] = rp_h[r0 + 1:r1 + 1] - rp_h[r0:r1]
        a, b = int(rp_h[r0]), int(rp_h[r1])
        cis.append(ci_h_fn(a, b))
        if vv_h_fn is not None:
            vvs.append(vv_h_fn(a, b))
    rp_s = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(deg, out=rp_s[1:])
    ci_s = np.ascontiguousarray(np.concatenate(cis), dtype=np.uint32)
    vv_s = None if vv_h_fn is None else np.ascontiguousarray(np.concatenate(vvs), dtype=np.float32)
    mS = int(rp_s[-1])
    desc = (f"{windows} runs of consecutive rows at evenly spaced starts (k*n/{windows}): {rows} rows, "
            f"{mS} edges, all {n} rows and columns in the arrays")
    return rp_s, ci_s, vv_s, mS, rows, desc


def host_cores():
    return os.cpu_count() or 1


def run_reference(args, rank, world):
    """The oracle (single-threaded C, host cores) on bounded samples of the same
    workload.  Only the oracle and the input generator are built and loaded in
    this process; the CUDA library is not."""
    if rank != 0:
        return
    import torch
    import oracle
    from paper_2501_06872_gb300 import build as pkg_build
    pkg_build.build_generators()
    oracle.build()
    kind, scale, ef, order, weighted = WORKLOADS[args.workload]
    torch.cuda.set_device(0)
    n, n_cols, rp, ci, vv = make_workload(args.workload, SEED, args.direction)
    m_full = ci.numel()
    rp_h = rp.cpu().numpy().view(np.uint64)
    rp_s, ci_s, vv_s, mS, rows, desc = sample_rows(
        rp_h, lambda a, b: ci[a:b].cpu().numpy().view(np.uint32),
        None if vv is None else (lambda a, b: vv[a:b].cpu().numpy()), min(args.ref_sample_edges, m_full))
    del rp, ci, vv, rp_h
    torch.cuda.empty_cache()
    for _ in range(args.warmup):
        oracle.transpose(rp_s, ci_s, vv_s, n_cols=n_cols)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.transpose(rp_s, ci_s, vv_s, n_cols=n_cols)
        ts.append(time.perf_counter() - t0)
    total = sum(ts)
    value = mS * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": workload_config(args.workload, n, m_full, weighted, n_cols, args.direction),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": host_cores(),
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_ranks(ms_step, m, world, device=None):
    """Max over ranks of the per-step time (every rank transposes its own
    replica of m edges); the whole-job value is the edges of all ranks over
    that time.  No collective touches the data path."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms_step)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    return ms_step, m * world / (ms_step * 1e-3)


def replica_seed(rank):
    """Each replica transposes its own seeded graph of the same shape."""
    return SEED + rank


def workload_config(name, n, m, weighted, n_cols=None, direction="csr"):
    kind, scale, ef, order, _ = WORKLOADS[name]
    c = {"workload": f"{name}{'-weighted' if weighted else ''}", "graph": kind, "scale": scale,
         "edge_factor": ef, "n_vertices": n, "n_edges": m, "vertex_order": order, "weighted": weighted,
         "seed": SEED, "l2": "inputs larger than L2 (no flush needed)", "parallelism": "replicas"}
    if direction != "csr":
        c["direction"] = "CSC input -> CSR"
    if n_cols is not None and n_cols != n:
        rs, cs = FOLDS.get(name, (0, 0))
        c.update({"n_rows": n, "n_cols": n_cols, "fold": f"rows merged by 2^{rs}, columns by 2^{cs}"})
    return c


def batched_leg(n_graphs, steps, warmup, pg_reps, config_json=None):
    """Config 4: uneven matrices transposed by one batch plan (CUDA-graph
    replay) vs one plain gt_transpose_sub launch sequence per matrix (the
    library's default configuration for each size), with the outputs compared
    element by element.  Returns a dict; frees its device memory."""
    import torch
    from paper_2501_06872_gb300 import binding
    from paper_2501_06872_gb300.inputs import gpu as ggen
    b = ggen.batch(n_graphs=n_graphs, seed=0x5EED0004)
    m_tot, v_tot, ng = b["total_m"], b["total_v"], b["n_graphs"]
    cp = torch.empty(v_tot + ng, dtype=torch.int64, device="cuda")
    ri = torch.empty(m_tot, dtype=torch.int32, device="cuda")
    vo = torch.empty(m_tot, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    cfg = None
    if config_json:
        cfg = binding.default_config(1 << 20, 1 << 24)
        for k, v in json.loads(config_json).items():
            setattr(cfg, k, int(v))
    plan = binding.BatchPlan(ggen.batch_graphs(b, cp, ri, vo), True, cfg)
    for _ in range(warmup):
        plan.transpose(s)
    plan.check()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with Clocks(0) as clk:
        ev0.record(s)
        for _ in range(steps):
            plan.transpose(s)
        ev1.record(s)
        torch.cuda.synchronize()
    plan.check()
    ms = ev0.elapsed_time(ev1) / steps
    info = plan.info()
    # the same captured sequence on an empty call: its launch and layout cost
    plan.transpose_descs(0, plan.d_descs, None, s)
    torch.cuda.synchronize()
    ev0.record(s)
    for _ in range(steps):
        plan.transpose_descs(0, plan.d_descs, None, s)
    ev1.record(s)
    torch.cuda.synchronize()
    ms_empty = ev0.elapsed_time(ev1) / steps
    plan.close()
    # per-graph baseline: the library's default configuration per matrix size
    nmax, mmax = int(b["n"].max()), int(b["m"].max())
    plans = {}
    for meth in (0, 1):
        c = binding.default_config(nmax, mmax)
        c.method = meth
        plans[meth] = binding.Plan(nmax, mmax, True, c)
    rp, ci, vv = b["row_ptr"], b["col_idx"], b["vals"]
    cp2 = torch.empty_like(cp)
    ri2 = torch.empty_like(ri)
    vo2 = torch.empty_like(vo)

    def per_graph():
        for g in range(ng):
            n, m = int(b["n"][g]), int(b["m"][g])
            r0, e0 = int(b["voff"][g]) + g, int(b["eoff"][g])
            meth = binding.default_config(n, m).method
            plans[meth].transpose_sub(n, m, rp[r0:r0 + n + 1], ci[e0:e0 + m], vv[e0:e0 + m], cp2[r0:r0 + n + 1],
                                      ri2[e0:e0 + m], vo2[e0:e0 + m], s)
    per_graph()
    torch.cuda.synchronize()
    e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0_.record(s)
    for _ in range(pg_reps):
        per_graph()
    e1_.record(s)
    torch.cuda.synchronize()
    ms_pg = e0_.elapsed_time(e1_) / pg_reps
    for p_ in plans.values():
        p_.check()
        p_.close()
    same = bool(torch.equal(cp, cp2) and torch.equal(ri, ri2) and torch.equal(vo.view(torch.int32), vo2.view(torch.int32)))
    lit = sum(algorithmic_bytes(int(b["n"][g]), int(b["m"][g]), True)[0] for g in range(ng))
    del cp, ri, vo, cp2, ri2, vo2, b, rp, ci, vv
    torch.cuda.empty_cache()
    return {"value": m_tot / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "graphs": ng, "n_edges": m_tot, "n_vertices": v_tot, "algorithmic_bytes": lit,
            "per_graph_baseline": {"value": m_tot / (ms_pg * 1e-3), "unit": UNIT, "ms_per_step": ms_pg,
                                   "reps": pg_reps, "speedup_batched": ms_pg / ms, "identical_output": same},
            "batch_info": info, "clocks": clk.summary(), "gpu_launches": info["kernel_launches"] * steps,
            "empty_call_ms": ms_empty, "launch_share": ms_empty / ms}


def run_batched(args):
    """--workload batched: the batch leg as its own JSON line."""
    peak, peak_kind = load_peaks()
    r = batched_leg(args.batch_graphs, args.steps, args.warmup, max(1, min(args.steps, 2)), args.config)
    gbs = r["algorithmic_bytes"] / (r["ms_per_step"] * 1e-3) / 1e9
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "batched-4096-zipf", "graphs": r["graphs"], "n_edges": r["n_edges"],
                       "n_vertices": r["n_vertices"],
                       "sizes": "n log-uniform [1024, 262144], Zipf(2) out-degree mean U[8,32], Zipf(1.5) dst",
                       "l2": "inputs larger than L2 (no flush needed)"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "traffic": None, "kernel": "whole batch (CUDA graph replay)", "peak_kind": peak_kind},
            "per_graph_baseline": r["per_graph_baseline"], "batch_info": r["batch_info"], "clocks": r["clocks"],
            "gpu_launches": r["gpu_launches"]}
    print(json.dumps(line), flush=True)


def step3_imbalance(busy_ms):
    """Load imbalance of Step 3 over the warp partitions (Sec. V-F): the share
    of the step's time the average partition is idle, 1 - mean / max of the
    busy times, and the coefficient of variation of the busy times."""
    busy = np.asarray(busy_ms, dtype=np.float64)
    if busy.size == 0 or busy.max() <= 0:
        return None
    return {"partitions": int(busy.size), "idle_share": float(1.0 - busy.mean() / busy.max()),
            "cv": float(busy.std() / busy.mean()), "max_ms": float(busy.max()), "mean_ms": float(busy.mean())}


def partition_bits_for(n_cols):
    """Bucket width of the partitioned (two-level) form: destination ranges of
    at most 2^20 columns, whose in-degree counters, cursors and one partly
    written sector per list (about 44 MB) stay in L2."""
    kb = max(1, int(n_cols - 1).bit_length())
    return min(8, max(1, kb - 20))


def hlh_leg(n, n_cols, m, weighted, rp, ci, vv, ref_out, steps=3, warmup=1, steal=False, partition_bits=0,
            hdv_k=512, unsorted=False):
    """PoTra's own method (Algorithm 2, k = 512 HDVs, with the LDV list sort)
    on the same resident graph: per-step device time, per-step stage times,
    and whether its output equals the default method's bytes.  steal: the
    two-phase Step 3 of Sec. V-F.  partition_bits: the partitioned
    (two-level) form, bucketed by that many top destination bits first.
    hdv_k = 0: Atomic GT (Algorithm 1).  unsorted: the paper's output as
    Sec. V times it (no LDV sort); col_ptr must still equal the default
    method's."""
    import torch
    from paper_2501_06872_gb300 import binding
    cfg = binding.default_config(n_cols, m)
    cfg.method, cfg.hdv_k, cfg.table_log2 = 0, hdv_k, (10 if hdv_k else 0)
    cfg.flags |= binding.FLAG_PARTITION_TIMES  # Step 3's per-warp busy times (Sec. V-F imbalance)
    if unsorted:
        cfg.flags |= binding.FLAG_UNSORTED
    if steal:
        cfg.flags |= binding.FLAG_STEAL_TAILS
    if partition_bits:
        cfg.partition_bits = partition_bits
    plan = binding.Plan(n, m, weighted, cfg, n_cols=n_cols)
    cp = torch.empty(n_cols + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(m, dtype=torch.int32, device="cuda")
    vo = torch.empty(m, dtype=torch.float32, device="cuda") if weighted else None
    stream = torch.cuda.current_stream()
    try:
        for _ in range(warmup):
            plan.transpose(rp, ci, vv, cp, ri, vo)
        plan.check()
        plan.enable_timing(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            plan.transpose(rp, ci, vv, cp, ri, vo)
        ev1.record(stream)
        torch.cuda.synchronize()
        plan.check()
        ms = ev0.elapsed_time(ev1) / steps
        t = plan.timing()
        st = plan.stats()
        pt = np.array(plan.partition_times())
    finally:
        plan.close()
    same_cp = bool(torch.equal(cp, ref_out[0]))
    same = bool(same_cp and torch.equal(ri, ref_out[1]) and
                (vo is None or torch.equal(vo.view(torch.int32), ref_out[2].view(torch.int32))))
    del cp, ri, vo
    torch.cuda.empty_cache()
    return {"method": "hlh", "value": m / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "gt_config": cfg.as_dict(),
            "stage_ms": {k: t[k] for k in ("partition_ms", "sample_ms", "count_ms", "scan_ms", "scatter_ms",
                                           "sort_ms")},
            "scatter_launch_ms": t["dominant_ms"], "hdv_selected": st["hdv_selected"],
            "step3_imbalance": step3_imbalance(pt),
            "coverage": st["hdv_edges"] / max(1, m), "identical_output": same, "col_ptr_identical": same_cp,
            "unsorted": unsorted,
            "gpu_launches": int(st["kernel_launches"]) * steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat28-degree", choices=sorted(WORKLOADS) + ["batched"])
    ap.add_argument("--direction", default="csr", choices=["csr", "csc"],
                    help="csc: transpose the workload's CSC back to CSR")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=None, help="JSON gt_config overrides")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hlh", action="store_true", help="skip the PoTra-method leg of the default line")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched leg of the default line")
    ap.add_argument("--cpu-sample-edges", type=int, default=1 << 26)
    ap.add_argument("--ref-sample-edges", type=int, default=1 << 24)
    ap.add_argument("--record-traffic", nargs=3, metavar=("CSV", "KERNEL", "NOTE"), default=None,
                    help="write profiles/traffic.json's entry for KERNEL on --workload from an ncu CSV and exit")
    ap.add_argument("--traffic-scale", type=float, default=1.0,
                    help="with --record-traffic: scale factor from the captured case to --workload")
    args = ap.parse_args()
    if args.record_traffic:
        record_traffic(args.record_traffic[0], args.record_traffic[1], args.workload, args.record_traffic[2],
                       args.traffic_scale)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        import torch
        torch.cuda.set_device(local)
        import __graft_entry__
        __graft_entry__.build()
        if rank == 0:
            run_batched(args)
        return

    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if local == 0:  # one build per node; the other ranks wait for it
            __graft_entry__.build()
        dist.barrier()
    __graft_entry__.build()
    from paper_2501_06872_gb300 import binding

    kind, scale, ef, order, weighted = WORKLOADS[args.workload]
    n, n_cols, rp, ci, vv = make_workload(args.workload, replica_seed(rank), args.direction)
    m = ci.numel()
    cfg = binding.default_config(n_cols, m)
    if args.config:
        for k, v in json.loads(args.config).items():
            setattr(cfg, k, int(v))
    plan = binding.Plan(n, m, weighted, cfg, n_cols=n_cols)
    cp = torch.empty(n_cols + 1, dtype=torch.int64, device="cuda")
    ri = torch.empty(m, dtype=torch.int32, device="cuda")
    vo = torch.empty(m, dtype=torch.float32, device="cuda") if weighted else None
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.transpose(rp, ci, vv, cp, ri, vo)
    plan.check()

    plan.enable_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            plan.transpose(rp, ci, vv, cp, ri, vo)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    plan.check()
    ms = ev0.elapsed_time(ev1)
    timing = plan.timing()
    stats = plan.stats()
    plan.enable_timing(False)
    ms_step, value = aggregate_ranks(ms / args.steps, m, world, device="cuda")

    peak, peak_kind = load_peaks()
    method = plan.config().method
    gt_config = plan.config().as_dict()
    stage_ms = {"count": timing["count_ms"], "scan": timing["scan_ms"], "scatter": timing["scatter_ms"],
                "sort": timing["sort_ms"], "sample": timing["sample_ms"]}
    lit, withv = algorithmic_bytes(n, m, weighted, n_cols)
    roof = roofline(plan.config(), timing, n, n_cols, m, weighted, peak, peak_kind, args.workload)
    step_gbs = lit / (ms_step * 1e-3) / 1e9

    learned = None
    if rank == 0:
        learned = selector_summary(plan, rp, ci, vv, cp, ri, vo, n_cols, m)

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        import oracle
        rp_h = rp.cpu().numpy().view(np.uint64)
        rp_s, ci_s, vv_s, mS, rows, desc = sample_rows(
            rp_h, lambda a, b: ci[a:b].cpu().numpy().view(np.uint32),
            None if vv is None else (lambda a, b: vv[a:b].cpu().numpy()), min(args.cpu_sample_edges, m))
        del rp_h
        t0 = time.perf_counter()
        oracle.transpose(rp_s, ci_s, vv_s, n_cols=n_cols)
        dt = time.perf_counter() - t0
        del rp_s, ci_s, vv_s
        cpu = {"value": mS / dt, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
               "sample": f"{desc}; {dt:.1f} s"}

    hlh = None
    if not args.no_hlh and rank == 0 and world == 1 and method == 1:
        # the legs need room next to the resident graph: the main plan's
        # workspace is freed here and the end-to-end leg gets a fresh plan
        plan.close()
        plan = None
        torch.cuda.empty_cache()
        hlh = hlh_leg(n, n_cols, m, weighted, rp, ci, vv, (cp, ri, vo))
        hlh["two_phase_step3"] = hlh_leg(n, n_cols, m, weighted, rp, ci, vv, (cp, ri, vo), steal=True)
        hlh["partitioned"] = hlh_leg(n, n_cols, m, weighted, rp, ci, vv, (cp, ri, vo),
                                     partition_bits=partition_bits_for(n_cols))
        # the paper's own comparison (Sec. V-B, no LDV sort): Atomic GT against the locality-optimised form
        hlh["unsorted_atomic_gt"] = hlh_leg(n, n_cols, m, weighted, rp, ci, vv, (cp, ri, vo), hdv_k=0, unsorted=True)
        hlh["unsorted_partitioned"] = hlh_leg(n, n_cols, m, weighted, rp, ci, vv, (cp, ri, vo), unsorted=True,
                                              partition_bits=partition_bits_for(n_cols))

    e2e = None
    if not args.no_e2e and rank == 0:
        host = host_inputs(rp, ci, vv, n, m, weighted, n_cols)
        del rp, ci, vv, cp, ri, vo  # the end-to-end leg works from host memory only
        if plan is None:
            torch.cuda.empty_cache()
            plan = binding.Plan(n, m, weighted, cfg, n_cols=n_cols)
        e2e = run_e2e(plan, host, n, m, weighted, args, n_cols)
        del host
    if plan is not None:
        plan.close()
    try:
        del rp, ci, vv, cp, ri, vo
    except NameError:
        pass
    torch.cuda.empty_cache()

    batched = None
    if not args.no_batched and rank == 0 and world == 1:
        batched = batched_leg(args.batch_graphs, 2, 3, 1)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": dict(workload_config(args.workload, n, m, weighted, n_cols, args.direction),
                               gt_config=gt_config),
                "roofline": roof,
                "step_hbm": {"gbs_formula": step_gbs, "frac_of_peak": step_gbs / peak,
                             "frac_of_8tbs": step_gbs / 8000.0, "bytes_formula": lit, "bytes_with_vals_read": withv,
                             "gbs_with_vals_read": withv / (ms_step * 1e-3) / 1e9},
                "stage_ms": stage_ms, "method": "radix" if method == 1 else "hlh", "stats": stats,
                "coverage": stats["hdv_edges"] / max(1, m),
                "clocks": clk.summary(),
                "gpu_launches": int(stats["kernel_launches"]) * args.steps,
                "learned": learned, "e2e": e2e, "cpu_baseline": cpu, "hlh": hlh, "batched": batched}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def selector_summary(plan, rp, ci, vv, cp, ri, vo, n, m):
    """Grid points the learned selector, the analytic model and the default
    configuration choose for this workload (gt_plan_tune; the plan keeps its
    configuration), plus the selector's held-out evaluation (regret = time of
    the chosen grid point / the exhaustive optimum, 64 graphs)."""
    from paper_2501_06872_gb300 import binding, selector_train
    keep = plan.config()
    sel = binding.Selector.pretrained()
    li, _ = plan.tune(binding.TUNE_LEARNED, rp, ci, vv, cp, ri, vo, selector=sel)
    ai, _ = plan.tune(binding.TUNE_ANALYTIC, rp, ci, vv, cp, ri, vo)
    sel.close()
    plan.set_config(keep)
    rep = json.load(open(os.path.join(ROOT, "paper_2501_06872_gb300", "selector_report.json")))
    return {"pick_learned": li, "pick_analytic": ai, "pick_default": selector_train.default_index(n, m),
            "heldout_regret": {k: rep["test"][k]["mean"] for k in ("learned", "analytic", "default")},
            "heldout_graphs": rep["n_test"]}


def gpu_local_cpus(device):
    """CPUs of the NUMA node the GPU's PCI function reports (sysfs), or None."""
    try:
        import torch
        p = torch.cuda.get_device_properties(device)
        path = f"/sys/bus/pci/devices/{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0/numa_node"
        node = int(open(path).read().strip())
        if node < 0:
            return None
        cpus = set()
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except Exception:
        return None


def host_inputs(rp, ci, vv, n, m, weighted, n_cols=None):
    """Pinned host copies of the inputs and pinned host outputs for the
    end-to-end leg, or a note if host memory is too small."""
    import torch
    nc = n if n_cols is None else n_cols
    need = 8 * (n + 1) + 8 * (nc + 1) + (4 * m + (4 * m if weighted else 0)) * 2
    avail = 0
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except Exception:
        pass
    if avail and need > 0.7 * avail:
        return f"host memory {avail / 2**30:.0f} GiB too small for {need / 2**30:.0f} GiB pinned buffers"
    # pinned pages land on the NUMA node of the CPU that first touches them:
    # allocate and fill them from the CPUs next to the GPU
    keep = None
    cpus = gpu_local_cpus(rp.device.index if rp.device.index is not None else 0)
    if cpus:
        try:
            keep = os.sched_getaffinity(0)
            os.sched_setaffinity(0, cpus)
        except OSError:
            keep = None
    try:
        return _pinned_buffers(rp, ci, vv, n, m, weighted, nc)
    finally:
        if keep:
            try:
                os.sched_setaffinity(0, keep)
            except OSError:
                pass


def _pinned_buffers(rp, ci, vv, n, m, weighted, nc):
    import torch
    h_rp = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
    h_ci = torch.empty(m, dtype=torch.int32, pin_memory=True)
    h_vv = torch.empty(m, dtype=torch.float32, pin_memory=True) if weighted else None
    h_cp = torch.empty(nc + 1, dtype=torch.int64, pin_memory=True)
    h_ri = torch.empty(m, dtype=torch.int32, pin_memory=True)
    h_vo = torch.empty(m, dtype=torch.float32, pin_memory=True) if weighted else None
    h_rp.copy_(rp)
    h_ci.copy_(ci)
    if weighted:
        h_vv.copy_(vv)
    return h_rp, h_ci, h_vv, h_cp, h_ri, h_vo


def run_e2e(plan, host, n, m, weighted, args, n_cols=None):
    """Same metric through the host entry point (gt_transpose_host_async, then
    gt_plan_host_wait): pinned host inputs copied in and outputs copied out
    inside the timed region, every step."""
    import torch
    if isinstance(host, str):
        return {"value": None, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None, "note": host}
    nc = n if n_cols is None else n_cols
    h_rp, h_ci, h_vv, h_cp, h_ri, h_vo = host
    steps = max(2, min(args.steps, 8))
    torch.cuda.empty_cache()  # the plan's device staging comes from cudaMalloc, beside torch's pool
    plan.transpose_host_async(h_rp, h_ci, h_vv, h_cp, h_ri, h_vo)  # warm-up (allocates device staging)
    plan.host_wait()
    torch.cuda.synchronize()
    # every step copies its inputs in and its CSC out; gt_transpose_host_async
    # overlaps a step's output copies with the next step's input copies
    plan.enable_timing(True)  # events around each call's copies (and steps)
    t0 = time.perf_counter()
    for _ in range(steps):
        plan.transpose_host_async(h_rp, h_ci, h_vv, h_cp, h_ri, h_vo)
    plan.host_wait()
    dt = (time.perf_counter() - t0) / steps
    ht = plan.host_timing()
    ct = plan.timing()
    plan.enable_timing(False)
    h2d = 8 * (n + 1) + 4 * m + (4 * m if weighted else 0)
    d2h = 8 * (nc + 1) + 4 * m + (4 * m if weighted else 0)
    copies = {"h2d_gbs": h2d / (ht["h2d_ms"] * 1e-3) / 1e9 if ht["h2d_ms"] else None,
              "d2h_gbs": d2h / (ht["d2h_ms"] * 1e-3) / 1e9 if ht["d2h_ms"] else None,
              "h2d_ms": ht["h2d_ms"], "d2h_ms": ht["d2h_ms"], "overlap_ms": ht["overlap_ms"],
              "overlap_share": ht["overlap_ms"] / min(ht["h2d_ms"], ht["d2h_ms"]) if ht["calls"] else None,
              "directions_overlapped": bool(ht["calls"] and ht["overlap_ms"] > 0.25 * min(ht["h2d_ms"], ht["d2h_ms"])),
              "transpose_ms": ct["total_ms"] or None, "calls_timed": ht["calls"]}
    return {"value": m / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1e3, "steps": steps, "copies": copies}


if __name__ == "__main__":
    main()
