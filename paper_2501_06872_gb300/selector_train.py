"""Training of the learned configuration selector on the library's own timings.

    python -m paper_2501_06872_gb300.selector_train --out DIR [--graphs 256 --train 192]

1. Dataset: `graphs` seeded R-MAT graphs with a ~ U[0.25, 0.70],
   b = c = (1 - a - d) / 2, d = 0.05, scale ~ U{18..28}, edge factor ~
   U{8..32} (at most 2^(32 - scale)), vertex order degree-sorted or
   seeded-random, weighted or not.
   For each: the features (gt_graph_features) and the exhaustive autotuner's
   table (gt_plan_tune, every grid point timed with CUDA events, median of 3),
   plus the analytic model's and the default configuration's grid points.
2. Training: grid points that run the same kernel sequence on a graph (radix
   digit caps with the same pass count) share one time; targets are
   log-regrets ln(t_i / min_j t_j) per grid point; the network (gt_selector,
   GPU forward/backward/Adam with an L2 penalty) fits them with a masked MSE,
   full batch, on the first `train` graphs.
3. Evaluation on the held-out graphs: time of the selected point over the
   best point (regret), for the learned, analytic and default choices.
Writes dataset.npz, selector_params.f32 and selector_report.json into --out.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
PARAMS_FILE = os.path.join(PKG, "selector_params.f32")
DATASET_FILE = os.path.join(PKG, "selector_dataset.npz")
D_PARAM = 0.05


def graph_spec(i: int, seed: int = 0x5EED0005):
    """Scales 18-28 (the headline graph's scale included); edge factors 8-32,
    capped so that m <= 2^32 (the weighted limit): at most 32 at scale 27 and
    16 at scale 28."""
    rng = np.random.default_rng([seed, i])
    a = float(rng.uniform(0.25, 0.70))
    b = (1.0 - a - D_PARAM) / 2.0
    scale = int(rng.integers(18, 29))
    ef = int(rng.integers(8, 33))
    ef = min(ef, 1 << (32 - scale))
    return {"a": a, "b": b, "c": b, "scale": scale, "edge_factor": ef,
            "order": "degree" if rng.random() < 0.5 else "random", "weighted": bool(rng.random() < 0.5),
            "seed": int(seed + 1000 + i)}


def _norm(c: dict) -> tuple:
    if c["method"] == 1:  # the bulk-staged kernel (tile 0) runs two 256-thread CTAs per SM whatever ctas_per_sm says
        return (1, c["radix_tile"], c["ctas_per_sm"] if c["radix_tile"] else 0, c.get("radix_digit_bits", 0) or 8)
    return (0, c["hdv_k"], c["table_log2"], c["block_threads"], c["ctas_per_sm"], c["warp_edges"],
            c["stage_edges"], c["flags"])


def default_index(n: int, m: int) -> int:
    """Grid point equal to gt_default_config for this size (-1 if none)."""
    from . import binding
    d = _norm(binding.default_config(n, m).as_dict())
    for i in range(binding.TUNE_GRID):
        if _norm(binding.grid_config(i, n, m).as_dict()) == d:
            return i
    return -1


def save_dataset(path, feats, times, meta):
    tmp = path + ".tmp.npz"
    np.savez(tmp, features=np.stack(feats), times=np.stack(times), meta=json.dumps(meta))
    os.replace(tmp, path)


def build_dataset(count: int, reps: int = 3, log=print, path=None):
    """Times every grid point on `count` graphs; with `path`, saves after every
    graph and resumes from what an earlier run saved there."""
    import torch
    from . import binding
    from .inputs import gpu as ggen
    feats, times, meta = [], [], []
    if path and os.path.exists(path):
        d = np.load(path, allow_pickle=False)
        feats, times, meta = list(d["features"]), list(d["times"]), json.loads(str(d["meta"]))
        log(f"resuming after {len(meta)} graphs")
    for i in range(len(meta), count):
        sp = graph_spec(i)
        t0 = time.time()
        n, rp, ci, vv = ggen.graph(sp["scale"], sp["edge_factor"], "rmat", sp["a"], sp["b"], sp["c"], sp["seed"],
                                   sp["order"], sp["weighted"])
        m = ci.numel()
        cp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        ri = torch.empty(m, dtype=torch.int32, device="cuda")
        vo = torch.empty(m, dtype=torch.float32, device="cuda") if vv is not None else None
        f = binding.graph_features(rp, ci, sp["weighted"]).cpu().numpy()
        plan = binding.Plan(n, m, sp["weighted"])
        _, table = plan.tune(binding.TUNE_EXHAUSTIVE, rp, ci, vv, cp, ri, vo, reps=reps)
        plan.close()
        ms = np.array([t["ms"] for t in table], dtype=np.float64)
        an = binding.analytic_index(f, n, m)
        di = default_index(n, m)
        feats.append(f)
        times.append(ms)
        meta.append({**sp, "n": n, "m": m, "analytic": an, "default": di})
        log(f"[{i + 1}/{count}] scale {sp['scale']} ef {sp['edge_factor']} a {sp['a']:.2f} {sp['order']} "
            f"w{int(sp['weighted'])}: best {int(np.argmin(np.where(ms > 0, ms, np.inf)))} "
            f"{ms[ms > 0].min():.3f} ms, analytic {an}, default {di} ({time.time() - t0:.1f} s)")
        del rp, ci, vv, cp, ri, vo
        torch.cuda.empty_cache()
        if path:
            save_dataset(path, feats, times, meta)
    return np.stack(feats), np.stack(times), meta


def effective_point(i: int, n: int):
    """What grid point i runs on an n-column matrix: radix points with the same
    tile kind (and CTAs per SM for register tiles) whose digit caps give the
    same pass count are one kernel sequence (gt_plan_tune times them once)."""
    from . import binding
    c = binding.grid_config(i, n, 1 << 24).as_dict()
    if c["method"] != 1:
        return ("hlh", c["hdv_k"], c["table_log2"], c["block_threads"], c["ctas_per_sm"], c["warp_edges"],
                c["stage_edges"], c["flags"])
    bits = max(1, int(n - 1).bit_length())
    cap = c["radix_digit_bits"] or 8
    return ("radix", c["radix_tile"], c["ctas_per_sm"] if c["radix_tile"] else 0, -(-bits // cap))


def merge_equivalent(times: np.ndarray, meta) -> np.ndarray:
    """Gives grid points that run the same kernel sequence on a graph the
    time of the first of them (datasets timed before gt_plan_tune merged them
    hold separate, noisy timings of identical runs)."""
    out = np.array(times, dtype=np.float64, copy=True)
    for r, mt in enumerate(meta):
        seen = {}
        for i in range(out.shape[1]):
            e = effective_point(i, int(mt["n"]))
            if e in seen:
                out[r, i] = out[r, seen[e]]
            else:
                seen[e] = i
    return out


def targets(times: np.ndarray):
    valid = times > 0
    best = np.where(valid, times, np.inf).min(axis=1, keepdims=True)
    y = np.where(valid, np.log(np.where(valid, times, 1.0) / best), 0.0)
    return y.astype(np.float32), valid.astype(np.float32)


def standardise(x: np.ndarray):
    mu = x.mean(axis=0)
    sd = x.std(axis=0) + 1e-3
    return mu.astype(np.float32), sd.astype(np.float32)


def train(feats, times, steps=3000, lr=1e-3, weight_decay=1e-3, seed=7, val=None, every=250, log=print):
    """Full-batch Adam (with an L2 penalty on the weights) on the masked MSE
    of log-regrets.  With val = (features, times), keeps the checkpoint (every
    `every` steps) of lowest mean validation regret."""
    import torch
    from . import binding
    sel = binding.Selector(seed=seed)
    p = sel.params()
    mu, sd = standardise(feats)
    F = binding.N_FEATURES
    p[:F] = mu
    p[F:2 * F] = sd
    p[2 * F:3 * F] = feats.min(axis=0)
    p[3 * F:4 * F] = feats.max(axis=0)
    sel.set_params(p)
    y, mask = targets(times)
    X = torch.from_numpy(feats.astype(np.float32)).cuda()
    T = torch.from_numpy(y).cuda()
    M = torch.from_numpy(mask).cuda()
    Xv = None if val is None else torch.from_numpy(val[0].astype(np.float32)).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    best = (np.inf, 0, sel.params())
    for it in range(1, steps + 1):
        sel.backward(X, T, M, loss=loss)
        sel.adam_step(lr=lr, weight_decay=weight_decay)
        if it % every == 0 or it == steps:
            torch.cuda.synchronize()
            rec = {"step": it, "loss": float(loss.item())}
            if Xv is not None:
                idx = sel.forward(Xv).cpu().numpy().argmin(axis=1)
                rec["val_regret"] = float(regrets(val[1], idx).mean())
                if rec["val_regret"] < best[0]:
                    best = (rec["val_regret"], it, sel.params())
            hist.append(rec)
            log(json.dumps(rec))
    params = sel.params() if Xv is None else best[2]
    sel.close()
    return params, hist, best[1] if Xv is not None else steps


def picks(params, feats, analytic=None):
    """Grid points the learned mode picks: the smallest score, or the analytic
    choice for graphs outside the trained feature range."""
    import torch
    from . import binding
    sel = binding.Selector(params)
    s = sel.forward(torch.from_numpy(feats.astype(np.float32)).cuda()).cpu().numpy()
    idx = s.argmin(axis=1)
    if analytic is not None:
        for i in range(len(idx)):
            if not sel.in_range(feats[i]):
                idx[i] = analytic[i]
    sel.close()
    return idx, s


def _in_range(params, f):
    from . import binding
    sel = binding.Selector(params)
    ok = sel.in_range(f)
    sel.close()
    return ok


def regrets(times, idx):
    best = np.where(times > 0, times, np.inf).min(axis=1)
    chosen = times[np.arange(len(idx)), idx]
    chosen = np.where(chosen > 0, chosen, np.inf)
    return chosen / best


def summary(r):
    r = np.asarray(r, dtype=np.float64)
    return {"mean": float(r.mean()), "geomean": float(np.exp(np.log(r).mean())), "max": float(r.max()),
            "optimal_share": float((r <= 1.0 + 1e-9).mean())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--graphs", type=int, default=256)
    ap.add_argument("--train", type=int, default=192)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--weight-decay", type=float, default=1e-3)
    ap.add_argument("--val", type=int, default=32, help="training graphs held out for checkpoint choice")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--dataset", default=None, help="reuse a dataset.npz instead of timing")
    ap.add_argument("--params", default=None, help="with --dataset: evaluate these parameters, no training")
    args = ap.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    os.makedirs(args.out, exist_ok=True)
    logf = open(os.path.join(args.out, "train.log"), "a")

    def log(msg):
        print(msg, flush=True)
        logf.write(msg + "\n")
        logf.flush()
    if args.dataset:
        d = np.load(args.dataset, allow_pickle=False)
        feats, times = d["features"], d["times"]
        meta = json.loads(str(d["meta"]))
        save_dataset(os.path.join(args.out, "dataset.npz"), list(feats), list(times), meta)
    else:
        feats, times, meta = build_dataset(args.graphs, args.reps, log, os.path.join(args.out, "dataset.npz"))
    times = merge_equivalent(times, meta)
    tr = slice(0, args.train)
    te = slice(args.train, len(feats))
    fit = slice(0, args.train - args.val)
    va = slice(args.train - args.val, args.train)
    if args.params:
        params = np.fromfile(args.params, dtype="<f4")
        hist, chosen_step = [], None
        if args.dataset:
            old = os.path.join(os.path.dirname(os.path.abspath(args.dataset)), "selector_report.json")
            if os.path.exists(old):
                prev = json.load(open(old))
                hist, chosen_step = prev.get("loss", []), prev.get("chosen_step")
    else:
        params, hist, chosen_step = train(feats[fit], times[fit], steps=args.steps, lr=args.lr,
                                          weight_decay=args.weight_decay,
                                          val=(feats[va], times[va]) if args.val else None, log=log)
    params.astype("<f4").tofile(os.path.join(args.out, "selector_params.f32"))
    an = np.array([m["analytic"] for m in meta])
    de = np.array([m["default"] for m in meta])
    idx_te, _ = picks(params, feats[te], an[te])
    idx_tr, _ = picks(params, feats[tr], an[tr])
    report = {
        "graphs": len(feats), "n_train": args.train, "n_test": len(feats) - args.train, "steps": args.steps,
        "n_val": args.val, "chosen_step": chosen_step, "loss": hist, "lr": args.lr,
        "weight_decay": args.weight_decay, "equivalent_points_merged": True,
        "test": {"learned": summary(regrets(times[te], idx_te)),
                 "analytic": summary(regrets(times[te], an[te])),
                 "default": summary(regrets(times[te], de[te])),
                 "time_learned_ms": float(times[te][np.arange(len(idx_te)), idx_te].sum()),
                 "time_analytic_ms": float(times[te][np.arange(len(idx_te)), an[te]].sum()),
                 "time_default_ms": float(times[te][np.arange(len(idx_te)), de[te]].sum()),
                 "time_best_ms": float(np.where(times[te] > 0, times[te], np.inf).min(axis=1).sum())},
        "train_fit": {"learned": summary(regrets(times[tr], idx_tr))},
        "test_out_of_range": int(sum(1 for i in range(len(idx_te)) if idx_te[i] == an[te][i]
                                     and not _in_range(params, feats[te][i]))),
        "grid_best_counts": np.bincount(np.where(times > 0, times, np.inf).argmin(axis=1),
                                        minlength=times.shape[1]).tolist(),
    }
    with open(os.path.join(args.out, "selector_report.json"), "w") as fh:
        json.dump(report, fh, indent=1)
    log(json.dumps(report["test"]))


if __name__ == "__main__":
    main()
