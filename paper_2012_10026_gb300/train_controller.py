"""Trains the learned direction / binning controller on the GPU.

Data: Kronecker graphs (edgefactor 16) at the given scales and seeds are
built and RCM-relabelled by the library; for a sample of roots, g3_bfs runs in
record_both mode, which expands every level both top-down (with five candidate
bin-threshold triples) and bottom-up from the same state and times each with
CUDA events. Each level L >= 1 (level 0 is always top-down) gives one sample:

  x = the controller's 12 features of F_L (g3_mlp_features, the same device
      code the controller runs),
  y = [ln(t_BU / t_TD), log2 t1*, log2 t2*, log2 t3*]

with t_TD the fastest top-down time over the candidates and t*'s its bin
thresholds. The 12-32-4 network is trained by g3_mlp_train (full-batch Adam,
one kernel), and the parameters are written as JSON.

How the controller uses it: on a level where the alpha/beta rule's own test
is within a factor of 4 of its threshold (rule_near), the network's sign of
ln(t_BU / t_TD) decides the direction when its magnitude exceeds the margin;
everywhere else the rule decides. The margin is the widest candidate that
loses nothing on a held-out graph of the largest trained size (pick_margin);
the network's bin thresholds are used only when they time at least 1 %
faster there, and only at trained graph sizes (controller_opts).

Usage:
  python -m paper_2012_10026_gb300.train_controller --scales 20 21 22 23 24 \\
      --seeds 11 12 13 14 15 --roots 12 --out paper_2012_10026_gb300/mlp_params.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import paper_2012_10026_gb300 as g3  # noqa: E402

LOSS_WEIGHTS = [1.0, 0.05, 0.05, 0.05]


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (layout W1, b1, W2, b2)."""
    rng = np.random.default_rng(seed)
    w1 = rng.uniform(-1, 1, (32, 12)) * math.sqrt(6.0 / 12)
    w2 = rng.uniform(-1, 1, (4, 32)) * math.sqrt(6.0 / 32)
    return np.concatenate([w1.ravel(), np.zeros(32), w2.ravel(), np.zeros(4)]).astype(np.float32)


def collect(scale: int, seed: int, nroots: int, root_seed: int, device="cuda"):
    """Recorded levels of nroots searches on one graph -> (rows, (n_bfs, nnz))."""
    import torch
    import graphgen
    n = 1 << scale
    src, dst = graphgen.kronecker_edges_dev(scale, 16, seed=seed, device=device)
    flags = graphgen.nonisolated_flags_dev(src, dst, n).cpu().numpy()
    roots = graphgen.pick_roots(flags, nroots, root_seed).tolist()
    g = g3.g3_build_csr(src, dst, n)
    del src, dst
    g3.g3_rcm_relabel(g)
    nb = (g.info["n_bfs"], g.info["nnz"])
    parent = torch.empty(n, dtype=torch.int32, device=device)
    level = torch.empty(n, dtype=torch.int32, device=device)
    opts = g3.opts(record_both=1, timing=1)
    rows = []
    for r in roots:
        st = g3.g3_bfs(g, r, parent, level, opts, max_stats=256)
        rows.append(st)
    g.free()
    return rows, nb


def rule_near(prev_dir, n_f, m_f, m_u, nb, alpha=14, beta=24):
    """Whether the alpha/beta rule's own test is within a factor of 4 of its
    threshold (m_f alpha against m_u after a top-down level, n_f beta
    against n after a bottom-up one): the levels on which the controller
    consults the network; the same integer test as the device code."""
    if prev_dir == 0:
        lhs, rhs = m_f * alpha, m_u
    else:
        lhs, rhs = n_f * beta, nb
    return 4 * lhs > rhs and lhs < 4 * rhs


def dataset(runs, alpha=14, beta=24):
    """(X, Y, meta) from [(rows_of_one_search, (n_bfs, nnz))]: one sample per
    level >= 1; meta = (t_TD, t_BU, the rule's direction, rule_near) per
    sample (collect() records with the library's alpha 14, beta 24)."""
    xs, ys, meta = [], [], []
    for st, (nb, nnz) in runs:
        if not st:
            continue
        x = g3.g3_mlp_features(st, nb, nnz).cpu().numpy()
        for i, (a, row) in enumerate(zip(st, x)):
            if a["level"] == 0 or a["t_td_ms"] <= 0 or a["t_bu_ms"] <= 0:
                continue
            prev = st[i - 1]["dir"] if i > 0 else 0
            xs.append(row)
            ys.append([math.log(a["t_bu_ms"] / a["t_td_ms"]), math.log2(a["best_t1"]),
                       math.log2(a["best_t2"]), math.log2(a["best_t3"])])
            meta.append((a["t_td_ms"], a["t_bu_ms"], a["dir"],
                         rule_near(prev, a["n_f"], a["m_f"], a["m_u"], nb, alpha, beta)))
    return (np.array(xs, np.float32), np.array(ys, np.float32), meta)


def raw_rows(runs):
    """Per sample of dataset(runs), the level record itself: n_f, m_f, n_u,
    m_u, id_min, id_max, n_bfs, nnz, previous direction, level, hist[4],
    t_TD, t_BU, the rule's direction and the best bins (for offline study)."""
    out = []
    for st, (nb, nnz) in runs:
        for i, a in enumerate(st):
            if a["level"] == 0 or a["t_td_ms"] <= 0 or a["t_bu_ms"] <= 0:
                continue
            prev = st[i - 1]["dir"] if i > 0 else 0
            out.append([a["n_f"], a["m_f"], a["n_u"], a["m_u"], a["id_min"], a["id_max"], nb,
                        nnz, prev, a["level"], *a["hist"], a["t_td_ms"], a["t_bu_ms"],
                        a["dir"], a["best_t1"], a["best_t2"], a["best_t3"]])
    return np.array(out, np.float64)


def regret(meta, choice_bu):
    """sum over levels of t(chosen direction) - min(t_TD, t_BU), in ms."""
    return float(sum((m[1] if c else m[0]) - min(m[0], m[1]) for m, c in zip(meta, choice_bu)))


MARGINS = [0.0, 0.05, 0.1, 0.15, 0.2, 0.3, 0.5, 0.75, 1.0, 1e9]


def gated(o0, meta, margin):
    """Direction choices of the controller: the network decides on the levels
    where the rule is near its threshold (rule_near) and its prediction is
    outside the margin (|predicted ln(t_BU/t_TD)| > margin), the alpha/beta
    rule everywhere else."""
    return [(x < 0) if (m[3] and abs(x) > margin) else (m[2] == 1) for x, m in zip(o0, meta)]


def pick_margin(table):
    """The widest margin whose regret on a held-out graph is the smallest
    any margin reaches (table: str(margin) -> regret): the rule stands
    wherever the network is not clearly sure, which keeps its choices safe
    on graphs larger than the training ones. 1e9 (the rule everywhere) when
    no finite margin reaches that regret."""
    low = min(table.values())
    ok = [m for m in MARGINS if m < 1e9 and table[str(m)] <= low + 1e-9]
    return max(ok) if ok else 1e9


def time_controllers(scale: int, seed: int, nroots: int, root_seed: int, configs: dict,
                     reps: int = 3, device="cuda", tuned: bool = True):
    """Summed device ms of nroots searches per named option set (dicts of
    g3_bfs_opts fields, on top of the graph's autotuned options when tuned;
    the minimum over reps for each root, 256 MB written between searches)."""
    import torch
    import graphgen
    n = 1 << scale
    src, dst = graphgen.kronecker_edges_dev(scale, 16, seed=seed, device=device)
    flags = graphgen.nonisolated_flags_dev(src, dst, n).cpu().numpy()
    roots = graphgen.pick_roots(flags, nroots, root_seed).tolist()
    g = g3.g3_build_csr(src, dst, n)
    del src, dst
    g3.g3_rcm_relabel(g)
    parent = torch.empty(n, dtype=torch.int32, device=device)
    level = torch.empty(n, dtype=torch.int32, device=device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    base = {}
    if tuned:  # tuning roots drawn apart from the timed ones, no cache
        troots = graphgen.pick_roots(flags, 16, root_seed + 1000).tolist()
        t, _ = g3.autotune_bfs(g, troots, parent, level, None, g3.opts())
        base = dict(alpha=t.alpha, beta=t.beta, t1=t.t1, t2=t.t2, t3=t.t3,
                    bu_reverse=t.bu_reverse, bu_kernel=t.bu_kernel)
    out = {}
    for name, kw in configs.items():
        o = g3.opts(**dict(base, **kw))
        best = [float("inf")] * len(roots)
        for _ in range(reps + 1):  # the first round builds the level-loop graph
            for i, r in enumerate(roots):
                flush.fill_(1)
                es.record()
                g3.g3_bfs(g, r, parent, level, o)
                ee.record()
                ee.synchronize()
                best[i] = min(best[i], es.elapsed_time(ee))
        out[name] = float(sum(best))
    g.free()
    return out


FEATURES = "size-free counts"  # the feature set the controller's device code computes


def controller_opts(path: str, n_bfs: int, device="cuda", **base):
    """g3_bfs options for the trained controller in `path`, on top of the
    options in `base`: the network with its margin and bin choice, at every
    graph size. Its features come from the frontier sizes and degree sums
    alone and are all ratios of the searched graph's own counts (frontier and
    unvisited sizes over n and nnz and over each other, mean degrees, bitmap
    words per frontier edge, frontier growth), so a graph larger than the
    training ones shows the network levels it has seen. Returns (opts,
    params tensor, note); the tensor must outlive the searches. Raises when
    the file was trained on another feature set."""
    import torch
    with open(path) as f:
        mj = json.load(f)
    if mj.get("features") != FEATURES:
        raise ValueError(f"{path}: trained on feature set {mj.get('features')!r}, the "
                         f"controller computes {FEATURES!r}; retrain it")
    params = torch.tensor(mj["params"], dtype=torch.float32, device=device)
    lo, hi = mj.get("n_bfs_range", [0, 0])
    inside = lo <= n_bfs <= hi
    # the best bin thresholds follow the absolute degrees of the frontier,
    # which grow with the graph: the network's thresholds are used only at
    # the sizes it was trained on, the directions at every size
    bins = int(mj.get("mlp_bins", 1)) if inside else 0
    kw = dict(base, controller=g3.G3_CTRL_LEARNED, mlp_params=params,
              mlp_margin=int(mj.get("mlp_margin", 0)), mlp_bins=bins)
    where = "inside" if inside else "outside"
    note = (f"the network decides every level's direction (n_bfs {n_bfs}, {where} the trained "
            f"sizes {lo}..{hi}); bin thresholds "
            + ("the network's" if bins else "autotuned"))
    return g3.opts(**kw), params, note


def train(X, Y, steps=3000, lr=1e-2, seed=0, device="cuda"):
    import torch
    p = torch.from_numpy(init_params(seed)).to(device)
    w = torch.tensor(LOSS_WEIGHTS, dtype=torch.float32, device=device)
    xt = torch.from_numpy(X).to(device)
    yt = torch.from_numpy(Y).to(device)
    losses = g3.g3_mlp_train(p, xt, yt, steps=steps, lr=lr, w=w).cpu().numpy()
    return p, losses


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scales", type=int, nargs="+", default=[20, 21, 22, 23, 24])
    ap.add_argument("--seeds", type=int, nargs="+", default=[11, 12, 13, 14, 15])
    ap.add_argument("--roots", type=int, default=12)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-2)
    ap.add_argument("--out", default=os.path.join(HERE, "mlp_params.json"))
    ap.add_argument("--eval-scale", type=int, default=0,
                    help="held-out graph (seed 2) on which to compare the controllers")
    ap.add_argument("--eval-roots", type=int, default=8)
    ap.add_argument("--dump", default="",
                    help="also write the recorded samples (features, targets, per-level "
                         "times and rule directions of the training, held-out and "
                         "evaluation graphs) to this .npz file")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    t0 = time.time()
    runs = []
    for scale, seed in zip(args.scales, args.seeds):
        rows, nb = collect(scale, seed, args.roots, seed + 100)
        runs += [(st, nb) for st in rows]
    X, Y, meta = dataset(runs)
    t1 = time.time()
    p, losses = train(X, Y, args.steps, args.lr)
    out = g3.g3_mlp_forward(p, torch.from_numpy(X).cuda()).cpu().numpy()
    learned_bu = out[:, 0] < 0
    heur_bu = np.array([m[2] == 1 for m in meta])
    best_bu = np.array([m[1] < m[0] for m in meta])
    summary = {
        "params": [float(v) for v in p.cpu().numpy()],
        "features": FEATURES,
        "layout": "W1[32][12], b1[32], W2[4][32], b2[4]",
        # graph sizes seen in training (BFS vertices); see controller_opts
        "n_bfs_range": [min(nb[0] for _, nb in runs), max(nb[0] for _, nb in runs)],
        "scales": args.scales, "seeds": args.seeds, "roots_per_graph": args.roots,
        "samples": int(len(X)), "steps": args.steps, "lr": args.lr,
        "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
        "direction_accuracy_learned": float(np.mean(learned_bu == best_bu)),
        "direction_accuracy_heuristic": float(np.mean(heur_bu == best_bu)),
        "train_regret_ms_learned": regret(meta, learned_bu),
        "train_regret_ms_heuristic": regret(meta, heur_bu),
        "collect_s": t1 - t0, "train_s": time.time() - t1,
    }
    # margin chosen on a held-out graph of the largest training scale (a new
    # seed and new roots), never on the evaluation scale
    rows, nb = collect(max(args.scales), 97, args.roots, 98)
    hruns = [(st, nb) for st in rows]
    Xh, _, mh = dataset(hruns)
    oh = g3.g3_mlp_forward(p, torch.from_numpy(Xh).cuda()).cpu().numpy()[:, 0]
    table = {str(m): regret(mh, gated(oh, mh, m)) for m in MARGINS}
    best_m = pick_margin(table)
    summary["holdout"] = {"scale": max(args.scales), "levels": int(len(Xh)),
                          "regret_ms_by_margin": table}
    summary["mlp_margin"] = int(round(min(best_m, 1e6) * 1000))
    # whether the network's bin thresholds beat the fixed ones: timed on the
    # same held-out graph, with the chosen margin
    # (all three on the held-out graph's autotuned options)
    lo = dict(controller=g3.G3_CTRL_LEARNED, mlp_params=p, mlp_margin=summary["mlp_margin"])
    tt = time_controllers(max(args.scales), 97, args.roots, 98, {
        "heuristic": dict(controller=g3.G3_CTRL_HEURISTIC),
        "learned_bins": dict(mlp_bins=1, **lo),
        "learned_fixed_bins": dict(mlp_bins=0, **lo)})
    summary["holdout"]["ms"] = tt
    # the network's bins replace the tuned ones only when clearly faster
    summary["mlp_bins"] = 1 if tt["learned_bins"] < 0.99 * tt["learned_fixed_bins"] else 0
    if args.eval_scale:
        # held-out graph: per-level times of both directions under the
        # heuristic's path; regret of each controller's choices on it
        rows, nb = collect(args.eval_scale, 1, args.eval_roots, 2)
        eruns = [(st, nb) for st in rows]
        Xe, Ye, me = dataset(eruns)
        oe = g3.g3_mlp_forward(p, torch.from_numpy(Xe).cuda()).cpu().numpy()
        summary["eval"] = {
            "scale": args.eval_scale, "roots": args.eval_roots, "levels": int(len(Xe)),
            "regret_ms_learned": regret(me, oe[:, 0] < 0),
            "regret_ms_learned_gated": regret(me, gated(oe[:, 0], me, best_m)),
            "regret_ms_heuristic": regret(me, [m[2] == 1 for m in me]),
            "best_total_ms": float(sum(min(m[0], m[1]) for m in me)),
        }
    if args.dump:
        arrays = {"train": raw_rows(runs), "holdout": raw_rows(hruns)}
        if args.eval_scale:
            arrays["eval"] = raw_rows(eruns)
        np.savez(args.dump, **arrays)
    with open(args.out, "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps({k: v for k, v in summary.items() if k != "params"}))


if __name__ == "__main__":
    main()
