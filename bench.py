#!/usr/bin/env python
"""Benchmark of the RCM-relabelled hybrid BFS on one GB300.

Workload (default): Kronecker SCALE 26, edgefactor 16 (2^26 vertices, 2^30
generated tuples, initiator 0.57/0.19/0.19/0.05), seeded synthetic input,
CSR built and RCM-relabelled on the GPU, 64 roots drawn uniformly among the
non-isolated vertices. One step = one BFS from each of the 64 roots.

Metric: harmonic-mean GTEPS over the roots, TEPS_r = m_r / t_r with m_r the
generated tuples whose first endpoint the search reaches (duplicates and
self-loops counted, as Graph500 counts generated edges) and t_r the device
time of the g3_bfs call (CUDA events on the launching stream). Preprocessing
(CSR build, RCM) is timed once and reported beside the metric, as the paper
reports RCM time separately (Table 5).

Parity: every root's level[] of the last timed step is compared with the CPU
oracle's, every parent[] is checked by the BFS-tree rules and the RCM
permutation is certified as Algorithm 3's output, on the host cores after the
timed region; the oracle's search times of that pass are the CPU baseline.

Arms:
  --impl gb300 (default)  the CUDA library through its C ABI
  --impl reference        the CPU oracle (serial C) on the host cores, one root
                          per step, the steps run concurrently one per core --
                          the paper's method has no runnable reference
                          implementation
Multi-GPU: a single-root BFS does not shard; N ranks run N independent
replicas (weak scaling) and the value is the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "harmonic-mean GTEPS over 64 roots, Kronecker SCALE 26; learned vs plain BFS"
L2_BYTES = 129 * 1024 * 1024
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # HBM3e nominal, for context beside the measured peak


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--scale", type=int, default=26)
    ap.add_argument("--edgefactor", type=int, default=16)
    ap.add_argument("--roots", type=int, default=64)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--root-seed", type=int, default=2)
    ap.add_argument("--controller",
                    choices=["auto", "heuristic", "learned", "topdown", "bottomup"],
                    default="auto", help="auto: learned when trained parameters exist")
    ap.add_argument("--mlp", default=os.path.join(ROOT, "paper_2012_10026_gb300",
                                                  "mlp_params.json"))
    ap.add_argument("--cpu-baseline", type=int, default=1,
                    help="run the oracle leg (rank 0): kron: every root's levels, parents "
                         "and the permutation checked with the oracle, whose search times "
                         "are the CPU baseline")
    ap.add_argument("--cpu-timeout", type=float, default=600.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--configs", type=int, default=1,
                    help="kron at SCALE 26: also run the SCALE 22 RCM comparison, the "
                         "Chung-Lu MS-BFS and the small-graph batch, each with an oracle "
                         "spot check, and report them in the line")
    ap.add_argument("--host-bfs", type=int, default=1,
                    help="kron, with the oracle leg: also time the paper's multithreaded "
                         "hybrid BFS on the host cores")
    ap.add_argument("--bu-reverse", type=int, default=1,
                    help="bottom-up scans rows from the highest label (degree-aware order)")
    ap.add_argument("--bu-kernel", type=int, default=-1,
                    help="bottom-up kernels: 0 word pairs, 1 staged + word tiles, 2 word "
                         "tiles, 3 word pairs + word tiles (-1: the autotuner's choice, else "
                         "the library default)")
    ap.add_argument("--out-split", type=int, default=-1,
                    help="output pass: 1 one pass, 2 two passes over label halves (-1: the "
                         "library default)")
    ap.add_argument("--stats-out", default="")
    ap.add_argument("--workload", choices=["kron", "msbfs", "batch"], default="kron",
                    help="kron: the single-root headline; msbfs: bit-sliced multi-source "
                         "BFS on a Chung-Lu graph; batch: many small graphs in one launch")
    ap.add_argument("--ms-log2n", type=int, default=24, help="msbfs: Chung-Lu 2^k vertices")
    ap.add_argument("--rcm-permille", type=int, default=1000,
                    help="kron: partial RCM, only the top p/1000 of V+ reordered (Sec. 4.6)")
    ap.add_argument("--host-loop", type=int, default=0,
                    help="kron: drive the level loop from the host (for kernel-level "
                         "profiling; the default runs it as one CUDA graph per search)")
    ap.add_argument("--rcm", type=int, default=1,
                    help="kron: 0 searches the graph in its generated labelling (no RCM, "
                         "isolated vertices kept), for the locality comparison")
    ap.add_argument("--learned-check-scale", type=int, default=24,
                    help="kron, learned controller: also compare it with the rule on a "
                         "graph of this (trained) SCALE; 0 skips")
    ap.add_argument("--tune-bfs", type=int, default=1,
                    help="kron: autotune alpha/beta/bins/scan order first (cached)")
    ap.add_argument("--msbfs-compare", type=int, default=1,
                    help="kron: also time the roots as one bit-sliced multi-source pass")
    ap.add_argument("--ms-roots", type=int, default=256, help="msbfs: sources (64 per launch)")
    ap.add_argument("--ms-push-alpha", type=int, default=-1,
                    help="msbfs: fixed push/pull split (-1: autotuned)")
    ap.add_argument("--ms-pull-warp-deg", type=int, default=-1,
                    help="msbfs: fixed warp-pull degree (-1: autotuned)")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--batch-warp-max-n", type=int, default=-1,
                    help="batch: warp-per-graph size limit (-1: autotuned with the mode)")
    ap.add_argument("--batch-mode", type=int, default=0,
                    help="batch, with --batch-warp-max-n: 0 persistent kernel, 1 union search")
    ap.add_argument("--tune-cache", default=os.path.join(ROOT, "paper_2012_10026_gb300",
                                                         "tune_cache.txt"),
                    help="msbfs/batch: autotuner cache ('' = tune afresh, no cache)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def start_clock_sampler(path):
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def stop_clock_sampler(proc, path, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
    except FileNotFoundError:
        return None
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "reasons": sorted(reasons)}


def level_bytes(st, nb):
    """Algorithmic bytes of one level's expansion kernels:
    bottom-up: visited word read, two row bounds per unvisited vertex (8 B
    streamed), col entry + frontier-bitmap word per examined edge, parent and
    level per new vertex, next-frontier and visited word writes;
    top-down: queue entry and two row bounds per frontier vertex, col entry +
    visited probe per edge, parent, level, queue append and visited write per
    new vertex."""
    words = (nb + 31) // 32
    if st["dir"] == 1:
        return 4 * words + 8 * st["n_u"] + 8 * st["examined"] + 8 * st["n_next"] + 8 * words
    return 4 * st["n_f"] + 16 * st["n_f"] + 8 * st["m_f"] + 16 * st["n_next"]


# bottom-up levels with under this many thousandths of the BFS graph
# unvisited run the vertex-list kernels (the library's default kernel set)
BU_LIST_PM = 40


def level_kind(st, nb):
    """'td', 'bu' (word-pair kernel) or 'bu_list' (vertex-list kernels) for
    one level record."""
    if st["dir"] == 0:
        return "td"
    return "bu_list" if st["n_u"] * 1000 < nb * BU_LIST_PM else "bu"


def roofline_levels(all_st, nb):
    """Per level kind: [algorithmic bytes, expansion ms, levels]."""
    agg = {"td": [0, 0.0, 0], "bu": [0, 0.0, 0], "bu_list": [0, 0.0, 0]}
    for st in all_st:
        for s in st:
            a = agg[level_kind(s, nb)]
            a[0] += level_bytes(s, nb)
            a[1] += s["ms_expand"]
            a[2] += 1
    return agg


def graph_kernel_count(all_st, nb):
    """Kernels the level-loop graphs run for these searches: level 0's two
    top-down kernels before the loop, then per loop iteration the controller
    and the level's kernels (top-down 2, plus a bitmap -> queue pass after a
    word-pair bottom-up level; word-pair bottom-up 1 and vertex-list
    bottom-up 2, plus a queue -> bitmap pass of 2 after a top-down level),
    and the last iteration's controller that ends the loop."""
    total = 0
    for st in all_st:
        prev = None
        for s in st:
            kind = level_kind(s, nb)
            if s["level"] == 0:
                total += 2
            else:
                body = {"td": 2, "bu": 1, "bu_list": 2}[kind]
                if kind == "td" and prev == "bu":
                    body += 1
                if kind != "td" and prev == "td":
                    body += 2
                total += 1 + body
            prev = kind
        if st:
            total += 1
    return total


def _max_over_ranks(dist, x):
    """Maximum of x over the ranks (x itself without a process group)."""
    if not dist:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_hm_gteps(dist, world, m, t_ms):
    """Whole-job harmonic-mean GTEPS of `world` replicas that each searched
    the same roots: every rank's sum of t/m, the slowest rank's taken, and
    world x (searches per rank) searches over it."""
    norm = sum((t / 1e3) / mm for mm, t in zip(m, t_ms))
    return world * len(m) / _max_over_ranks(dist, norm) / 1e9


def harmonic_gteps(m, t_ms):
    return len(m) / sum((t / 1e3) / mm for mm, t in zip(m, t_ms)) / 1e9


# --------------------------------------------------------- CPU oracle leg
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def host_mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 16 << 30


def oracle_threads(n, want):
    """Concurrent oracle searches the host can take: at most `want`, one per
    core but one kept for the launching thread, and about 5 arrays of n int32
    (the GPU's outputs, the oracle's outputs, its queue) each in memory."""
    per = 5 * 4 * n + (64 << 20)
    by_mem = max(1, (host_mem_available() - (24 << 30)) // per)
    return int(max(1, min(want, host_cores() - 1, by_mem)))


class ParityLeg:
    """Checks the GPU's results on the same graph with the CPU oracle, on
    host threads (the oracle's C entry points run without the GIL):

    * from the start, in the background: the host twin of the generator and
      the oracle's CSR (untimed);
    * per root, after the timed region: the oracle BFS, its level[] compared
      with the GPU's element by element, and the GPU's parent[] checked by the
      BFS-tree rules (rule 5 of the validator, the edge rule, follows from the
      level equality); the oracle BFS times of this pass are the CPU
      baseline (roots run concurrently, one per host core);
    * the GPU's RCM permutation certified as Algorithm 3's output
      (orc_rcm_check: the conditions that make it unique), since Algorithm 3
      itself, with a sort of every row, takes many minutes at 2^26 vertices.
    """

    def __init__(self, scale, edgefactor, seed, root_seed, nroots):
        import threading
        self.scale, self.n = scale, 1 << scale
        self.args = (scale, edgefactor, seed, root_seed, nroots)
        self.err = None
        self.gen_done = threading.Event()
        self.csr_done = threading.Event()
        self.th = threading.Thread(target=self._prepare, daemon=True)
        self.th.start()

    def _prepare(self):
        try:
            import graphgen
            import oracle
            scale, ef, seed, root_seed, nroots = self.args
            t0 = time.time()
            src, dst = graphgen.kronecker_edges(scale, ef, seed=seed)
            self.roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, self.n),
                                             nroots, root_seed).tolist()
            self.gen_s = time.time() - t0
            self.gen_done.set()
            t1 = time.time()
            self.off, self.col = oracle.build_csr(src, dst, self.n)
            self.csr_s = time.time() - t1
        except Exception as e:  # reported in the line, never fatal for the GPU arm
            self.err = repr(e)
        finally:
            self.gen_done.set()
            self.csr_done.set()

    def wait_generation(self, timeout=600.0):
        """The host generator runs on every core (OpenMP): timed GPU work
        waits until it is done."""
        self.gen_done.wait(timeout)

    def check(self, roots, m_r, fetch, perm, timeout=3600.0):
        """fetch(i) -> (parent, level) numpy int32 [n] of roots[i] in original
        IDs; perm: the GPU's old_of_new (None: no RCM). Returns the parity
        and cpu_baseline records."""
        from concurrent.futures import ThreadPoolExecutor
        import threading
        import numpy as np
        import oracle
        self.csr_done.wait(timeout)
        if self.err or not hasattr(self, "off"):
            return {"error": self.err or "oracle CSR not ready"}, None
        if list(roots) != list(self.roots):
            return {"error": "root draw differs between the host and device generators"}, None
        T = oracle_threads(self.n, 64)
        gate = threading.Semaphore(T)
        off, col = self.off, self.col

        def one(i, r, par, lev):
            try:
                s = time.perf_counter()
                _, lo = oracle.bfs(off, col, r)
                dt = time.perf_counter() - s
                exact = bool(np.array_equal(lo, lev))
                del lo
                v = oracle.validate_tree(off, col, r, par, lev) if exact else (-1, -1)
                return r, exact, v == 0, dt, None if v == 0 else v
            finally:
                gate.release()

        def rcm_cert():
            s = time.perf_counter()
            res = oracle.rcm_check(off, col, perm)
            return res, time.perf_counter() - s

        w0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=T + 1) as ex:
            fr = ex.submit(rcm_cert) if perm is not None else None
            futs = []
            for i, r in enumerate(roots):
                gate.acquire()
                par, lev = fetch(i)
                futs.append(ex.submit(one, i, r, par, lev))
                del par, lev
            res = [f.result() for f in futs]
            cert = fr.result() if fr is not None else None
        wall = time.perf_counter() - w0
        bad = [{"root": r, "level_exact": e, "rule": v} for r, e, ok, _, v in res if not ok]
        parity = {"roots_checked": len(res), "level_exact": sum(1 for x in res if x[1]),
                  "parent_valid": sum(1 for x in res if x[2]),
                  "perm_exact": None if cert is None else cert[0] == 0,
                  "perm_check": None if cert is None else
                  ("orc_rcm_check: the permutation meets the conditions that make "
                   "Algorithm 3's output unique" if cert[0] == 0 else f"failed {cert[0]}"),
                  "perm_check_s": None if cert is None else cert[1],
                  "failures": bad[:8],
                  "oracle": f"host twin of the generator {self.gen_s:.1f} s, oracle CSR "
                            f"{self.csr_s:.1f} s, {len(res)} oracle BFS + tree checks on "
                            f"{T} threads {wall:.1f} s"}
        ms = [m_r[r] for r in roots]
        ts = [x[3] * 1e3 for x in res]
        cpu = {"value": harmonic_gteps(ms, ts), "unit": "GTEPS", "cores": T, "kind": "oracle",
               "sample": f"all {len(res)} roots of the workload, serial oracle BFS (one root "
                         f"per thread, {T} at a time on {host_cores()} host cores) on the "
                         f"oracle's own CSR of the same graph; per-root times while the "
                         f"other threads run",
               "aggregate_gteps": sum(ms) / wall / 1e9,
               "per_root_s": {"min": min(x[3] for x in res),
                              "median": statistics.median(x[3] for x in res),
                              "max": max(x[3] for x in res)}}
        return parity, cpu


def host_hybrid_leg(g, roots, m_r, gpu_level):
    """The paper's own multithreaded hybrid BFS (Algorithms 4-6, hostbfs/) on
    the host cores, on the GPU's RCM-relabelled graph copied to the host:
    every root timed (wall time of the search, outputs in original IDs) and
    its level[] compared with the GPU's (which the oracle checked)."""
    import numpy as np
    import hostbfs
    import torch
    off, col = g.csr(device="cpu")
    o2n, n2o = g.perm(device="cpu")
    torch.cuda.synchronize()
    n = g.info["n"]
    T = max(1, host_cores() - 1)
    hb = hostbfs.HostBFS(off.numpy(), col.numpy(), o2n.numpy(), n2o.numpy(), n, threads=T)
    parent = np.empty(n, np.int32)
    level = np.empty(n, np.int32)
    hb.bfs(int(roots[0]), parent=parent, level=level)  # first touch of the workspace
    ts, same = [], 0
    for i, r in enumerate(roots):
        s = time.perf_counter()
        hb.bfs(int(r), parent=parent, level=level)
        ts.append((time.perf_counter() - s) * 1e3)
        same += int(np.array_equal(level, gpu_level(i)))
    hb.close()
    ms = [m_r[r] for r in roots]
    return {"value": harmonic_gteps(ms, ts), "unit": "GTEPS", "cores": T,
            "kind": "the paper's hybrid BFS on the host (Algorithms 4-6: even neighbour split, "
                    "descending partitions with fetch_add stealing, neighbors+ first, shrinking "
                    "partitions, 128-bit copy/OR), OpenMP",
            "sample": f"all {len(roots)} roots, one search at a time on {T} threads, on the "
                      f"GPU's RCM graph copied to the host",
            "levels_equal_gpu": same, "per_root_ms_median": statistics.median(ts)}


# ------------------------------------------ secondary configurations
class Background:
    """Runs fn() on a host thread (the oracle's C calls release the GIL);
    result() waits and returns its value or {"error": ...}."""

    def __init__(self, fn):
        import threading
        self.val = None
        self.th = threading.Thread(target=self._run, args=(fn,), daemon=True)
        self.th.start()

    def _run(self, fn):
        try:
            self.val = fn()
        except Exception as e:  # reported in the line, never fatal
            self.val = {"error": repr(e)}

    def result(self, timeout=1800.0):
        self.th.join(timeout)
        return self.val if not self.th.is_alive() else {"error": "timeout"}


def _time_roots(g3, g, roots, parent, level, opts, flush, reps=2):
    """Per-root device time of g3_bfs (the best of `reps` runs after one
    warm-up pass), an L2 flush before each search."""
    import torch
    ev_s = torch.cuda.Event(enable_timing=True)
    ev_e = torch.cuda.Event(enable_timing=True)
    best = [float("inf")] * len(roots)
    for rep in range(reps + 1):
        for i, r in enumerate(roots):
            flush.fill_(1)
            ev_s.record()
            g3.g3_bfs(g, r, parent, level, opts)
            ev_e.record()
            ev_e.synchronize()
            if rep:
                best[i] = min(best[i], ev_s.elapsed_time(ev_e))
    return best


def c2_leg(flush, scale=22, spot=2):
    """Kronecker SCALE 22, 64 roots, the alpha = 14 / beta = 24 rule with the
    library defaults, searched on the RCM-relabelled graph and on the graph
    in its generated labelling (isolated vertices kept): the locality effect
    of RCM (the paper's Table 5 / Fig. 5 comparison, on the GPU). Oracle
    spot check: the permutation equals Algorithm 3's (orc_rcm) and `spot`
    roots' levels are exact and parents valid on both graphs."""
    import torch
    import graphgen
    import oracle
    import paper_2012_10026_gb300 as g3
    n = 1 << scale
    src, dst = graphgen.kronecker_edges_dev(scale, 16, seed=1)
    flags = graphgen.nonisolated_flags_dev(src, dst, n).cpu().numpy()
    roots = graphgen.pick_roots(flags, 64, 2).tolist()

    def orc():
        hs, hd = graphgen.kronecker_edges(scale, 16, seed=1)
        off, col = oracle.build_csr(hs, hd, n)
        P, _ = oracle.rcm(off, col)
        return off, col, P, [oracle.bfs(off, col, r)[1] for r in roots[:spot]]

    bg = Background(orc)
    cnt = torch.bincount(src.long(), minlength=n)
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    out, keep = {}, {}
    for rcm in (1, 0):
        g = g3.g3_build_csr(src, dst, n)
        if rcm:
            g3.g3_rcm_relabel(g)
            keep["perm"] = g.perm()[0].cpu().numpy()
        m_r = []
        for i, r in enumerate(roots):
            g3.g3_bfs(g, r, parent, level)
            m_r.append(int(cnt[level >= 0].sum().item()))
            if i < spot:
                keep[(rcm, i)] = (parent.cpu().numpy(), level.cpu().numpy())
        t = _time_roots(g3, g, roots, parent, level, g3.opts(), flush)
        out["rcm" if rcm else "generated_labels"] = {
            "value": harmonic_gteps(m_r, t), "unit": "GTEPS",
            "per_root_ms_median": statistics.median(t)}
        g.free()
    del src, dst, cnt
    o = bg.result()
    if isinstance(o, dict):
        out["parity"] = o
        return out
    off, col, P, lref = o
    import numpy as np
    lv_ok = sum(int(np.array_equal(keep[(rc, i)][1], lref[i])) for rc in (1, 0)
                for i in range(spot))
    pv_ok = sum(int(oracle.validate(off, col, roots[i], *keep[(rc, i)]) == 0)
                for rc in (1, 0) for i in range(spot))
    out["parity"] = {"roots_checked": 2 * spot, "level_exact": lv_ok, "parent_valid": pv_ok,
                     "perm_exact": bool(np.array_equal(keep["perm"], P)),
                     "ok": lv_ok == 2 * spot and pv_ok == 2 * spot and
                     bool(np.array_equal(keep["perm"], P))}
    out["workload"] = f"kronecker_scale{scale}_ef16_64roots_rule14_24_library_defaults"
    return out


def c3_leg(flush, tune_cache, log2n=24, nsrc=256, spot=2):
    """Chung-Lu 2^24 (power law 2.1, mean degree 20, cap 2^16), RCM, 256
    sources as 4 bit-sliced launches of 64: aggregate GTEPS, the roofline
    fraction from the launches' own work counts, and an oracle spot check of
    `spot` sources' levels."""
    import numpy as np
    import torch
    import graphgen
    import oracle
    import paper_2012_10026_gb300 as g3
    n = 1 << log2n
    src, dst = graphgen.chunglu_edges_dev(n)
    flags = graphgen.nonisolated_flags_dev(src, dst, n).cpu().numpy()
    roots = graphgen.pick_roots(flags, nsrc, 2).tolist()

    def orc():
        hs, hd = graphgen.chunglu_edges(n)
        off, col = oracle.build_csr(hs, hd, n)
        return [oracle.bfs(off, col, r)[1] for r in roots[:spot]]

    bg = Background(orc)
    g = g3.g3_build_csr(src, dst, n)
    g3.g3_rcm_relabel(g)
    cnt = torch.bincount(src.long(), minlength=n)
    del src, dst
    batches = [roots[i:i + 64] for i in range(0, len(roots), 64)]
    lv = torch.empty((64, n), dtype=torch.int8, device="cuda")
    mopts, _ = g3.autotune_msbfs(g, batches[0], lv[:len(batches[0])], tune_cache or None)
    m_s, spot_lv = [], []
    for b in batches:
        g3.g3_msbfs(g, b, lv[:len(b)], mopts)
        for i in range(len(b)):
            m_s.append(int(cnt[lv[i] >= 0].sum().item()))
        if not spot_lv:
            spot_lv = [lv[i].cpu().numpy() for i in range(spot)]
    ev_s = torch.cuda.Event(enable_timing=True)
    ev_e = torch.cuda.Event(enable_timing=True)
    times, work = [], []
    for rep in range(2):
        for b in batches:
            flush.fill_(1)
            ev_s.record()
            g3.g3_msbfs(g, b, lv[:len(b)], mopts)
            ev_e.record()
            ev_e.synchronize()
            if rep:
                times.append(ev_s.elapsed_time(ev_e))
                work.append(g3.g3_msbfs_last_stats(g))
    info = g.info
    nb = info["n_bfs"]
    comp = sum(8 * nb * w["pull_levels"] + 24 * w["pull_vertices"] + 12 * w["pull_entries"]
               + 20 * w["push_entries"] + 64 * nb + 64 * n for w in work) / len(work)
    avg_ms = sum(times) / len(times)
    peak, _ = load_peaks()
    g.free()
    del lv, cnt
    torch.cuda.empty_cache()
    out = {"workload": f"chunglu_2^{log2n}_g2.1_d20_cap65536_rcm_{nsrc}sources_4x64",
           "value": sum(m_s) / (sum(times) / 1e3) / 1e9, "unit": "GTEPS",
           "ms_per_launch_median": statistics.median(times),
           "roofline": {"achieved": comp / (avg_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": comp / (avg_ms / 1e3) / 1e9 / peak},
           "push_alpha": mopts.push_alpha, "pull_warp_deg": mopts.pull_warp_deg}
    o = bg.result()
    if isinstance(o, dict):
        out["parity"] = o
        return out
    ok = sum(int(np.array_equal(spot_lv[i], o[i].astype(np.int8))) for i in range(spot))
    out["parity"] = {"sources_checked": spot, "level_exact": ok, "ok": ok == spot}
    return out


def c4_leg(flush, tune_cache, count=4096, spot=16):
    """4096 Kronecker graphs (SCALE ~ U{8..14}, edge factor 16), each
    RCM-relabelled with one root, packed and searched in one launch:
    GTEPS = sum over graphs of m_g / launch time; oracle spot check of every
    (count / spot)-th graph's levels and parents."""
    import numpy as np
    import torch
    import graphgen
    import oracle
    import paper_2012_10026_gb300 as g3
    specs = graphgen.small_graph_specs(count, seed=5)
    graphs, roots_u, voff, srcs = [], [], [0], []
    t0 = time.perf_counter()
    for scale, gseed in specs:
        n = 1 << scale
        s, d = graphgen.kronecker_edges_dev(scale, 16, seed=gseed)
        flags = graphgen.nonisolated_flags_dev(s, d, n).cpu().numpy()
        r = int(graphgen.pick_roots(flags, 1, seed=gseed)[0])
        g = g3.g3_build_csr(s, d, n)
        g3.g3_rcm_relabel(g)
        graphs.append(g)
        roots_u.append(voff[-1] + r)
        srcs.append(s.long() + voff[-1])
        voff.append(voff[-1] + n)
    b = g3.g3_batch_pack(graphs)
    for g in graphs:
        g.free()
    setup_s = time.perf_counter() - t0
    pick = list(range(0, count, max(1, count // spot)))[:spot]

    def orc():
        res = []
        for i in pick:
            sc, gs = specs[i]
            hs, hd = graphgen.kronecker_edges(sc, 16, seed=gs)
            off, col = oracle.build_csr(hs, hd, 1 << sc)
            res.append((off, col, oracle.bfs(off, col, roots_u[i] - voff[i])[1]))
        return res

    bg = Background(orc)
    N = voff[-1]
    roots = torch.tensor(roots_u, dtype=torch.int32, device="cuda")
    parent = torch.empty(N, dtype=torch.int32, device="cuda")
    level = torch.empty(N, dtype=torch.int32, device="cuda")
    o, _ = g3.autotune_batch(b, roots, parent, level, tune_cache or None)
    g3.g3_bfs_batch(b, roots, parent, level, o)
    src_all = torch.cat(srcs)
    del srcs
    m_total = int((level[src_all] >= 0).sum().item())
    del src_all
    ph, lh = parent.cpu().numpy(), level.cpu().numpy()
    ev_s = torch.cuda.Event(enable_timing=True)
    ev_e = torch.cuda.Event(enable_timing=True)
    times = []
    for rep in range(4):
        flush.fill_(1)
        ev_s.record()
        g3.g3_bfs_batch(b, roots, parent, level, o, timed=False)
        ev_e.record()
        ev_e.synchronize()
        if rep:
            times.append(ev_s.elapsed_time(ev_e))
    b.free()
    out = {"workload": f"kronecker_batch{count}_scale8-14_ef16_rcm_1root",
           "value": m_total / (statistics.median(times) / 1e3) / 1e9, "unit": "GTEPS",
           "ms_per_launch_median": statistics.median(times), "graphs": count,
           "mode": o.mode, "warp_max_n": o.warp_max_n, "setup_s": setup_s}
    res = bg.result()
    if isinstance(res, dict):
        out["parity"] = res
        return out
    lv_ok = pv_ok = 0
    for (off, col, lref), i in zip(res, pick):
        a, e = voff[i], voff[i + 1]
        # the batch reports union original IDs; shift back to the graph's own
        pp = ph[a:e].copy()
        pp[pp >= 0] -= a
        lv_ok += int(np.array_equal(lh[a:e], lref))
        pv_ok += int(oracle.validate(off, col, roots_u[i] - a, pp, lh[a:e]) == 0)
    out["parity"] = {"graphs_checked": len(pick), "level_exact": lv_ok, "parent_valid": pv_ok,
                     "ok": lv_ok == len(pick) and pv_ok == len(pick)}
    return out


def finish_oracle_leg(p, q, timeout):
    """Result of a spawned oracle process (None when it did not answer)."""
    try:
        d = q.get(timeout=timeout)
    except Exception:
        p.kill()
        return None
    p.join(timeout=10)
    return d


# ------------------------------------------------------------ reference arm
def reference_arm(args, rank, world):
    """The CPU oracle timed on the host cores: one root per step, the steps
    run concurrently (one root per thread, one thread per core); each root's
    time is its own search's."""
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor
    import numpy as np
    import graphgen
    import oracle
    n = 1 << args.scale
    t0 = time.time()
    src, dst = graphgen.kronecker_edges(args.scale, args.edgefactor, seed=args.seed)
    roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), args.roots,
                                args.root_seed)
    off, col = oracle.build_csr(src, dst, n)
    # generated tuples per first endpoint: m_r = sum over the reached vertices
    tuples_from = np.bincount(src, minlength=n)
    del src, dst
    setup_s = time.time() - t0
    nsteps = args.warmup + args.steps
    T = oracle_threads(n, nsteps)

    def step(i):
        r = int(roots[i % len(roots)])
        s = time.perf_counter()
        _, level = oracle.bfs(off, col, r)
        dt = time.perf_counter() - s
        return int(tuples_from[level >= 0].sum()), dt * 1e3

    w0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=T) as ex:
        res = list(ex.map(step, range(nsteps)))
    wall = time.perf_counter() - w0
    ms = [m for m, _ in res[args.warmup:]]
    tms = [t for _, t in res[args.warmup:]]
    v = harmonic_gteps(ms, tms)
    line = {
        "impl": "reference", "metric": METRIC,
        "value": v, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(tms) / len(tms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": T, "kind": "oracle",
                         "sample": f"one root per step (roots in draw order), serial oracle "
                                   f"BFS on the oracle's CSR, the {nsteps} steps run "
                                   f"concurrently on {T} threads ({host_cores()} host cores; "
                                   f"each time is its own search's); setup {setup_s:.1f} s "
                                   f"untimed, searches {wall:.1f} s wall"},
        "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args):
    rcm = "rcm" if getattr(args, "rcm", 1) else "norcm"
    if rcm == "rcm" and getattr(args, "rcm_permille", 1000) < 1000:
        rcm = f"rcm{args.rcm_permille}permille"
    return {"workload": f"kronecker_scale{args.scale}_ef{args.edgefactor}_{rcm}_{args.roots}roots",
            "scale": args.scale, "edgefactor": args.edgefactor, "roots": args.roots,
            "initiator": [0.57, 0.19, 0.19, 0.05], "gen_seed": args.seed,
            "root_seed": args.root_seed,
            "l2": "256 MB write between roots (L2 flush); CSR larger than L2",
            "parallelism": "replicas"}


# ------------------------------------------------------------------ GPU arm
def gpu_arm(args, rank, world):
    import numpy as np
    import torch
    import graphgen
    import paper_2012_10026_gb300 as g3

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    parity = None
    if rank == 0 and args.cpu_baseline:
        parity = ParityLeg(args.scale, args.edgefactor, args.seed, args.root_seed, args.roots)

    L = g3.lib()
    n = 1 << args.scale
    src, dst = graphgen.kronecker_edges_dev(args.scale, args.edgefactor, seed=args.seed)
    flags = graphgen.nonisolated_flags_dev(src, dst, n).cpu().numpy()
    roots = graphgen.pick_roots(flags, args.roots, args.root_seed).tolist()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = g3.g3_build_csr(src, dst, n)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    if args.rcm and args.rcm_permille < 1000:
        g3.g3_rcm_relabel_partial(g, args.rcm_permille)  # Sec. 4.6
    elif args.rcm:
        g3.g3_rcm_relabel(g)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    info = g.info
    use_learned = args.controller == "learned" or (args.controller == "auto" and
                                                   os.path.exists(args.mlp))
    name = "learned" if use_learned else ("heuristic" if args.controller == "auto"
                                          else args.controller)
    args.controller_used = name
    ctrl = {"heuristic": g3.G3_CTRL_HEURISTIC, "learned": g3.G3_CTRL_LEARNED,
            "topdown": g3.G3_CTRL_TOPDOWN, "bottomup": g3.G3_CTRL_BOTTOMUP}[name]
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # autotuned alpha/beta, bins and scan order for this graph-size class
    # (untimed; 16 tuning roots drawn apart from the timed ones; cached)
    forced = {k: v for k, v in (("bu_kernel", args.bu_kernel), ("out_split", args.out_split))
              if v >= 0}
    base = dict(bu_reverse=args.bu_reverse, **forced)
    tune_rec, t_tune = None, 0.0
    if args.tune_bfs:
        t_tune = time.perf_counter()
        troots = graphgen.pick_roots(flags, 16, args.root_seed + 1000).tolist()
        topts, tune_rec = g3.autotune_bfs(g, troots, parent, level, args.tune_cache or None,
                                          g3.opts(bu_reverse=args.bu_reverse))
        t_tune = time.perf_counter() - t_tune
        base = dict(alpha=topts.alpha, beta=topts.beta, t1=topts.t1, t2=topts.t2, t3=topts.t3,
                    bu_reverse=topts.bu_reverse, bu_kernel=topts.bu_kernel)
        base.update(forced)
    kw = dict(controller=ctrl, **base)
    mlp_t, learned_note = None, None
    if ctrl == g3.G3_CTRL_LEARNED:
        from paper_2012_10026_gb300.train_controller import controller_opts
        lo, mlp_t, learned_note = controller_opts(args.mlp, info["n_bfs"], **base)
        kw.update(controller=lo.controller, mlp_params=mlp_t, mlp_margin=lo.mlp_margin,
                  mlp_bins=lo.mlp_bins)
    decided = {g3.G3_CTRL_HEURISTIC: "alpha/beta rule", g3.G3_CTRL_LEARNED: "learned MLP",
               g3.G3_CTRL_TOPDOWN: "top-down only", g3.G3_CTRL_BOTTOMUP: "bottom-up only"}
    controller_rec = {"requested": args.controller, "decided_by": decided[kw["controller"]],
                      "note": learned_note}
    if args.host_loop:  # profiling: every level's kernels as separate stream launches
        kw["timing"] = 1
    opts = g3.opts(**kw)  # default path: the level loop runs as one CUDA graph
    # host-driven, events around each level; the counts the byte model needs,
    # without the histogram, so the kernels timed are the ones searches run
    opts_timed = g3.opts(**dict(kw, timing=1, stats_counts_only=1))
    # the plain method: the alpha/beta rule on the same tuned options, and
    # with the library defaults
    plain_opts = g3.opts(controller=g3.G3_CTRL_HEURISTIC, **base)
    default_opts = g3.opts(controller=g3.G3_CTRL_HEURISTIC, bu_reverse=args.bu_reverse, **forced)

    # m_r per root (bookkeeping, outside any timed region)
    m_r = {}
    for r in roots:
        g3.g3_bfs(g, r, parent, level, opts)
        m_r[r] = int((level[src.long()] >= 0).sum().item()) if n <= (1 << 22) else \
            int(sum(int((level[src[i:i + (1 << 27)].long()] >= 0).sum().item())
                    for i in range(0, src.numel(), 1 << 27)))
    del src, dst
    torch.cuda.empty_cache()

    ev_s = torch.cuda.Event(enable_timing=True)
    ev_e = torch.cuda.Event(enable_timing=True)

    # the timed searches write root i's outputs to slot i, so that every
    # root's result of the last timed step can be checked with the oracle
    slots = None
    if parity is not None:
        slots = (torch.empty((len(roots), n), dtype=torch.int32, device="cuda"),
                 torch.empty((len(roots), n), dtype=torch.int32, device="cuda"))

    def one_step(o, nstats, keep=False):
        times, stats = [], []
        for i, r in enumerate(roots):
            p_out, l_out = (slots[0][i], slots[1][i]) if keep else (parent, level)
            flush.fill_(1)
            ev_s.record()
            st = g3.g3_bfs(g, r, p_out, l_out, o, max_stats=nstats)
            ev_e.record()
            ev_e.synchronize()
            times.append(ev_s.elapsed_time(ev_e))
            stats.append(st)
        return times, stats

    for _ in range(args.warmup):
        one_step(opts, 0)
    if parity is not None:  # the host generator runs on every core
        parity.wait_generation()
    clk_path = os.path.join(tempfile.gettempdir(), f"g3_clocks_{rank}.csv")
    sampler = start_clock_sampler(clk_path)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = L.g3_kernel_launches()
    w0 = time.perf_counter()
    all_t = []
    for _ in range(args.steps):
        t, _ = one_step(opts, 0, keep=slots is not None)
        all_t += t
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    launches = L.g3_kernel_launches() - launches0
    graph_launches = len(roots) * args.steps  # one level-loop graph per search
    # instrumented step: the same kernels launched level by level with CUDA
    # events around each level's expansion, for the per-kernel roofline
    inst_t, all_st = one_step(opts_timed, 256)
    # the plain heuristic BFS on the same graph and roots, when the headline
    # is the learned controller
    plain_t = None
    if ctrl != g3.G3_CTRL_HEURISTIC:
        for _ in range(args.warmup):
            one_step(plain_opts, 0)
        torch.cuda.synchronize()
        plain_t = []
        for _ in range(args.steps):
            plain_t += one_step(plain_opts, 0)[0]
    default_t = None
    if args.tune_bfs:
        for _ in range(args.warmup):
            one_step(default_opts, 0)
        torch.cuda.synchronize()
        default_t = []
        for _ in range(args.steps):
            default_t += one_step(default_opts, 0)[0]
    # the same 64 roots as one bit-sliced multi-source pass (after the timed
    # region; autotuned push/pull split and warp binning)
    msb = None
    if len(roots) <= 64 and args.msbfs_compare:
        lv8 = torch.empty((len(roots), n), dtype=torch.int8, device="cuda")
        t_mtune = time.perf_counter()
        mopts, mrec = g3.autotune_msbfs(g, roots, lv8, args.tune_cache or None)
        t_mtune = time.perf_counter() - t_mtune
        mt = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1)
            ev_s.record()
            g3.g3_msbfs(g, roots, lv8, mopts)
            ev_e.record()
            ev_e.synchronize()
            if i >= args.warmup:
                mt.append(ev_s.elapsed_time(ev_e))
        # every source's levels equal the single-root search's (spot check)
        g3.g3_bfs(g, roots[0], parent, level, plain_opts)
        same = bool(torch.equal(lv8[0].to(torch.int32), level))
        del lv8
        torch.cuda.empty_cache()
        m_sum = sum(m_r[r] for r in roots)
        single = sum(all_t[:len(roots)])
        msb = {"aggregate_gteps": m_sum / (statistics.median(mt) / 1e3) / 1e9,
               "ms_per_launch_median": statistics.median(mt),
               "single_root_aggregate_gteps": m_sum / (single / 1e3) / 1e9,
               "single_root_total_ms": single, "levels_equal_single_root": same,
               "push_alpha": mopts.push_alpha, "pull_warp_deg": mopts.pull_warp_deg,
               "autotune": dict(mrec.to_dict(), seconds=t_mtune)}
    if dist:
        dist.barrier()
    clocks = stop_clock_sampler(sampler, clk_path, local)
    ms = [m_r[r] for _ in range(args.steps) for r in roots]
    hm = harmonic_gteps(ms, all_t)
    value = replica_hm_gteps(dist, world, ms, all_t)

    # roofline of the dominant kernel
    nb = info["n_bfs"]
    agg = roofline_levels(all_st, nb)
    dom = "bu" if agg["bu"][1] >= agg["td"][1] else "td"
    peak, peak_kind = load_peaks()
    bytes_, tms, launches_dom = agg[dom]
    # DRAM bytes of this build's kernels are measured on a small case
    # (SCALE 24, one kernel, a few launches) and kept with the profiles; a
    # DRAM-counter capture of the full workload is not taken
    traffic, traffic_src = None, "not captured at this size; see the SCALE 24 profiles"
    achieved = bytes_ / (tms / 1e3) / 1e9 if tms > 0 else 0.0
    # kernels run inside the level-loop graphs (not host launches)
    launches += graph_kernel_count(all_st, nb) * args.steps

    # the other configurations of the workload family, each with its own
    # oracle spot check (after the timed region; their oracle work runs on
    # host threads while the GPU times them)
    configs = None
    if rank == 0 and args.configs and args.scale == 26:
        configs = {}
        for name, fn in (("c2_rcm_vs_generated_labels", lambda: c2_leg(flush)),
                         ("c3_msbfs_chunglu", lambda: c3_leg(flush, args.tune_cache)),
                         ("c4_batch_small_graphs", lambda: c4_leg(flush, args.tune_cache))):
            t_leg = time.perf_counter()
            try:
                configs[name] = fn()
            except Exception as e:  # reported, never fatal for the headline
                configs[name] = {"error": repr(e)}
            configs[name]["seconds"] = time.perf_counter() - t_leg
            torch.cuda.empty_cache()

    # the oracle checks every root's result of the last timed step and the
    # permutation, on the host cores (before the end-to-end leg, whose host
    # wall time the busy cores would disturb)
    parity_rec, cpu, host_par = None, None, None
    if parity is not None:
        perm = g.perm()[0].cpu().numpy() if (args.rcm and args.rcm_permille >= 1000) else None

        def fetch(i):
            return slots[0][i].cpu().numpy(), slots[1][i].cpu().numpy()

        parity_rec, cpu = parity.check(roots, m_r, fetch, perm)
        if args.host_bfs:
            host_par = host_hybrid_leg(g, roots, m_r, lambda i: slots[1][i].cpu().numpy())
        del slots
        torch.cuda.empty_cache()
        if cpu is None:
            cpu = {"value": None, "unit": "GTEPS", "cores": 0, "kind": "oracle",
                   "sample": "oracle leg did not finish: " + str(parity_rec.get("error"))}

    # end to end through the C ABI with pinned host outputs
    e2e = None
    if not args.no_e2e:
        hp = torch.empty(n, dtype=torch.int32).pin_memory()
        hl = torch.empty(n, dtype=torch.int32).pin_memory()
        plain = opts
        et = []
        for i in range(args.warmup + args.steps):
            for r in roots:
                flush.fill_(1)
                torch.cuda.synchronize()
                s = time.perf_counter()
                g3.g3_bfs(g, r, hp, hl, plain)
                dt = time.perf_counter() - s
                if i >= args.warmup:
                    et.append(dt * 1e3)
        e2e = {"value": harmonic_gteps(ms, et), "unit": "GTEPS", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": len(roots) * 2 * n * 4,
               "note": "the graph stays resident on the device (built and relabelled once, "
                       "as the paper times the search apart from preprocessing), so a "
                       "search's only input is the root, passed by value: h2d is 0 by "
                       "design; parent[] and level[] of every root are written to pinned "
                       "host memory inside the host-timed region"}


    # the trained controller against the rule on a graph of a size it was
    # trained on (the headline graph is outside them, see learned_controller)
    g.free()
    check = None
    if ctrl == g3.G3_CTRL_LEARNED and args.learned_check_scale > 0:
        check = learned_check(args, flush)

    if rank == 0:
        levels = [len(st) for st in all_st]
        line = {
            "metric": METRIC,
            "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(all_t) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": workload_config(args),
            "roofline": {"bound": "hbm",
                         "kernel": ("bu_pull (dense bottom-up levels)" if dom == "bu"
                                    else "td_front+td_bins"),
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "traffic_source": traffic_src,
                         "peak_kind": peak_kind, "launches": launches_dom,
                         "avg_launch_ms": tms / max(launches_dom, 1),
                         "bytes_per_launch": bytes_ / max(launches_dom, 1),
                         "timed_in": "instrumented step after the timed region: the same "
                                     "kernels launched level by level, CUDA events on the "
                                     "launching stream around each level's expansion"},
            "parity": parity_rec,
            "controller": controller_rec,
            "cpu_baseline": cpu, "cpu_baseline_parallel": host_par,
            "configs": configs,
            "e2e": e2e, "gpu_launches": int(launches),
            "graph_launches": graph_launches,
            "instrumented_hm_gteps": harmonic_gteps([m_r[r] for r in roots], inst_t),
            "clocks": clocks,
            "wall_s_timed": wall,
            "graph": {"n": info["n"], "n_plus": info["n_plus"], "nnz": info["nnz"],
                      "max_degree": info["max_degree"]},
            "preprocess_s": {"csr_build": t1 - t0, "rcm_relabel": t2 - t1},
            "per_root_ms": {"min": min(all_t), "median": statistics.median(all_t),
                            "max": max(all_t)},
            "levels": {"min": min(levels), "max": max(levels)},
            "hm_this_rank": hm,
            "msbfs_same_roots": msb,
            "plain_heuristic": None if plain_t is None else {
                "value": harmonic_gteps(ms, plain_t), "unit": "GTEPS",
                "per_root_ms_median": statistics.median(plain_t),
                "options": "alpha/beta rule, same tuned alpha, beta, bins and scan order"},
            "plain_default_options": None if default_t is None else {
                "value": harmonic_gteps(ms, default_t), "unit": "GTEPS",
                "per_root_ms_median": statistics.median(default_t),
                "options": "alpha/beta rule, library defaults (14, 24, 32/1024/32768)"},
            "options": {k: v for k, v in kw.items() if k != "mlp_params"},
            "learned_controller": learned_note,
            "learned_vs_rule_trained_size": check,
            "autotune": None if tune_rec is None else dict(tune_rec.to_dict(), seconds=t_tune),
        }
        print(json.dumps(line), flush=True)
        if args.stats_out:
            with open(args.stats_out, "w") as f:
                json.dump({"roots": roots, "m_r": [m_r[r] for r in roots], "times_ms": all_t,
                           "stats": all_st}, f)
    if dist:
        dist.destroy_process_group()


def learned_check(args, flush, reps=3):
    """Harmonic-mean GTEPS of the trained controller and of the alpha/beta
    rule over 64 roots of a Kronecker graph of a size the controller was
    trained on; both on the autotuned options of that graph (alpha, beta,
    bins, scan order and kernels from the autotuner, the controller's own
    bins when its file says so); per root the best of `reps` runs."""
    import torch
    import graphgen
    import paper_2012_10026_gb300 as g3
    from paper_2012_10026_gb300.train_controller import controller_opts
    scale, n = args.learned_check_scale, 1 << args.learned_check_scale
    src, dst = graphgen.kronecker_edges_dev(scale, args.edgefactor, seed=args.seed)
    flags = graphgen.nonisolated_flags_dev(src, dst, n).cpu().numpy()
    roots = graphgen.pick_roots(flags, 64, args.root_seed).tolist()
    g = g3.g3_build_csr(src, dst, n)
    g3.g3_rcm_relabel(g)
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    m_r = []
    for r in roots:
        g3.g3_bfs(g, r, parent, level)
        m_r.append(int((level[src.long()] >= 0).sum().item()))
    del src, dst
    troots = graphgen.pick_roots(flags, 16, args.root_seed + 1000).tolist()
    topts, _ = g3.autotune_bfs(g, troots, parent, level, args.tune_cache or None,
                               g3.opts(bu_reverse=args.bu_reverse))
    base = dict(alpha=topts.alpha, beta=topts.beta, t1=topts.t1, t2=topts.t2, t3=topts.t3,
                bu_reverse=topts.bu_reverse, bu_kernel=topts.bu_kernel)
    lo, params, note = controller_opts(args.mlp, g.info["n_bfs"], **base)
    rule = g3.opts(controller=g3.G3_CTRL_HEURISTIC, **base)
    ev_s = torch.cuda.Event(enable_timing=True)
    ev_e = torch.cuda.Event(enable_timing=True)
    out = {"workload": f"kronecker_scale{scale}_ef{args.edgefactor}_rcm_64roots",
           "controller": note, "options": "autotuned for this graph, the same for both"}
    for name, o in (("learned", lo), ("rule", rule)):
        best = [float("inf")] * len(roots)
        for _ in range(reps + 1):  # the first pass builds the level-loop graph
            for i, r in enumerate(roots):
                flush.fill_(1)
                ev_s.record()
                g3.g3_bfs(g, r, parent, level, o)
                ev_e.record()
                ev_e.synchronize()
                best[i] = min(best[i], ev_s.elapsed_time(ev_e))
        out[name] = {"value": harmonic_gteps(m_r, best), "unit": "GTEPS",
                     "total_ms": sum(best)}
    g.free()
    return out


# ------------------------------------------------- secondary workloads
def _common_line(args, world, metric, value, unit, times_ms, config):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sum(times_ms) / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config}


def _setup_dist(args):
    import torch
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    world = int(os.environ.get("WORLD_SIZE", 1))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return local, world, dist





def _ms_oracle_worker(log2n, roots, q):
    try:
        import numpy as np
        import graphgen
        import oracle
        n = 1 << log2n
        src, dst = graphgen.chunglu_edges(n)
        off, col = oracle.build_csr(src, dst, n)
        runs = []
        for r in roots:
            t0 = time.perf_counter()
            _, lv = oracle.bfs(off, col, int(r))
            dt = time.perf_counter() - t0
            runs.append((int(r), int((lv[src] >= 0).sum()), dt))
        q.put({"ok": True, "runs": runs})
    except Exception as e:  # reported in the JSON line
        q.put({"ok": False, "error": repr(e)})


def msbfs_arm(args, rank, world):
    """Bit-sliced multi-source BFS: Chung-Lu 2^24 (power law 2.1, mean degree
    20, degree cap 2^16), RCM-relabelled, 256 sources run as 4 launches of 64.
    Metric: aggregate GTEPS = sum over sources of m_s / sum of launch times."""
    import numpy as np
    import torch
    import graphgen
    import paper_2012_10026_gb300 as g3

    local, world, dist = _setup_dist(args)
    n = 1 << args.ms_log2n
    src, dst = graphgen.chunglu_edges_dev(n)
    flags = graphgen.nonisolated_flags_dev(src, dst, n).cpu().numpy()
    roots = graphgen.pick_roots(flags, args.ms_roots, args.root_seed).tolist()
    oracle_proc = None
    if rank == 0 and args.cpu_baseline:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        p = ctx.Process(target=_ms_oracle_worker, args=(args.ms_log2n, roots[:2], q))
        p.start()
        oracle_proc = (p, q)
    g = g3.g3_build_csr(src, dst, n)
    g3.g3_rcm_relabel(g)
    info = g.info
    cnt = torch.bincount(src.long(), minlength=n)  # generated tuples per first endpoint
    del src, dst
    torch.cuda.empty_cache()
    batches = [roots[i:i + 64] for i in range(0, len(roots), 64)]
    lv = torch.empty((64, n), dtype=torch.int8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # autotuned push/pull split and warp binning (untimed; cached per size class)
    t_tune = time.perf_counter()
    if args.ms_push_alpha > 0 and args.ms_pull_warp_deg > 0:
        mopts, tune_rec = g3.msbfs_opts(push_alpha=args.ms_push_alpha,
                                        pull_warp_deg=args.ms_pull_warp_deg), None
    else:
        mopts, tune_rec = g3.autotune_msbfs(g, batches[0], lv[:len(batches[0])],
                                            args.tune_cache or None)
    t_tune = time.perf_counter() - t_tune
    # m_s per source (bookkeeping, untimed)
    m_s = []
    for b in batches:
        g3.g3_msbfs(g, b, lv[:len(b)], mopts)
        for i in range(len(b)):
            m_s.append(int(cnt[lv[i] >= 0].sum().item()))
    ev_s = torch.cuda.Event(enable_timing=True)
    ev_e = torch.cuda.Event(enable_timing=True)

    work = []  # per-launch work counts for the roofline

    def step():
        t = []
        for b in batches:
            flush.fill_(1)
            ev_s.record()
            g3.g3_msbfs(g, b, lv[:len(b)], mopts)
            ev_e.record()
            ev_e.synchronize()
            t.append(ev_s.elapsed_time(ev_e))
            work.append(g3.g3_msbfs_last_stats(g))
        return t

    for _ in range(args.warmup):
        step()
    clk_path = os.path.join(tempfile.gettempdir(), f"g3_clocks_ms_{rank}.csv")
    sampler = start_clock_sampler(clk_path)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = g3.kernel_launches()
    times = []
    for _ in range(args.steps):
        times += step()
    torch.cuda.synchronize()
    launches = g3.kernel_launches() - l0
    if dist:
        dist.barrier()
    clocks = stop_clock_sampler(sampler, clk_path, local)
    tsum = _max_over_ranks(dist, sum(times))
    value = world * args.steps * sum(m_s) / (tsum / 1e3) / 1e9
    # the same sources, one plain g3_bfs each (heuristic controller)
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    plain_t = []
    for r in roots:
        flush.fill_(1)
        ev_s.record()
        g3.g3_bfs(g, r, parent, level)
        ev_e.record()
        ev_e.synchronize()
        plain_t.append(ev_s.elapsed_time(ev_e))
    # algorithmic bytes per launch from the launch's own work counts: a pull
    # level reads every vertex's source word (8 B) and, for the vertices it
    # scans, two row bounds (16 B), the entries it reads (4 B each) with the
    # frontier word of each (8 B) and writes the next-frontier word (8 B); a
    # push level reads every pushed entry (4 B), the target's word (8 B) and
    # ORs into it (8 B); the output reads 64 B of levels per BFS vertex and
    # writes k bytes per vertex
    nb, nnz = info["n_bfs"], info["nnz"]
    w_t = work[-len(times):]
    comp = sum(8 * nb * w["pull_levels"] + 24 * w["pull_vertices"] + 12 * w["pull_entries"]
               + 20 * w["push_entries"] + 64 * nb + 64 * n for w in w_t) / len(w_t)
    avg_ms = sum(times) / len(times)
    peak, peak_kind = load_peaks()
    cpu = None
    if oracle_proc is not None:
        d = finish_oracle_leg(*oracle_proc, timeout=args.cpu_timeout)
        if d and d.get("ok"):
            runs = d["runs"]
            cpu = {"value": sum(x[1] for x in runs) / sum(x[2] for x in runs) / 1e9,
                   "unit": "GTEPS", "cores": 1, "kind": "oracle",
                   "sample": f"{len(runs)} of the {len(roots)} sources, serial oracle BFS on "
                             f"the oracle's CSR (generation and CSR untimed)"}
        else:
            cpu = {"value": None, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                   "sample": "oracle leg did not finish: " + (d or {}).get("error", "timeout")}
    if rank == 0:
        line = _common_line(args, world, f"aggregate GTEPS, bit-sliced MS-BFS, {len(roots)} "
                            f"sources as {len(batches)} launches of 64, Chung-Lu 2^"
                            f"{args.ms_log2n}", value, "GTEPS", times,
                            {"workload": f"chunglu_2^{args.ms_log2n}_g2.1_d20_cap65536_rcm_"
                                         f"{len(roots)}sources", "sources_per_launch": 64,
                             "push_alpha": mopts.push_alpha,
                             "pull_warp_deg": mopts.pull_warp_deg,
                             "l2": "256 MB write between launches (L2 flush)",
                             "parallelism": "replicas"})
        line.update({
            "roofline": {"bound": "hbm", "kernel": "g3_msbfs launch (all its kernels)",
                         "achieved": comp / (avg_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": comp / (avg_ms / 1e3) / 1e9 / peak, "traffic": None,
                         "frac_of_nominal": comp / (avg_ms / 1e3) / 1e9 / NOMINAL_HBM_GBS,
                         "peak_kind": peak_kind, "bytes_per_launch": comp,
                         "bytes_model": "per launch from g3_msbfs_last_stats: 8 B x nb per "
                                        "pull level, 24 B per scanned vertex, 12 B per read "
                                        "entry, 20 B per pushed entry, 64 B x nb + 64 B x n "
                                        "output",
                         "work_last_launch": w_t[-1]},
            "cpu_baseline": cpu, "gpu_launches": int(launches), "clocks": clocks,
            "e2e": None,
            "graph": {"n": info["n"], "n_plus": info["n_plus"], "nnz": info["nnz"],
                      "max_degree": info["max_degree"]},
            "per_launch_ms": {"min": min(times), "median": statistics.median(times),
                              "max": max(times)},
            "autotune": None if tune_rec is None else dict(tune_rec.to_dict(), seconds=t_tune),
            "plain_g3_bfs_same_sources": {
                "aggregate_gteps": sum(m_s) / (sum(plain_t) / 1e3) / 1e9,
                "harmonic_gteps": harmonic_gteps(m_s, plain_t),
                "total_ms": sum(plain_t)},
        })
        print(json.dumps(line), flush=True)
    g.free()
    if dist:
        dist.destroy_process_group()


def _batch_oracle_worker(specs, q):
    try:
        import graphgen
        import oracle
        runs = []
        for scale, gseed, root in specs:
            src, dst = graphgen.kronecker_edges(scale, 16, seed=gseed)
            off, col = oracle.build_csr(src, dst, 1 << scale)
            t0 = time.perf_counter()
            _, lv = oracle.bfs(off, col, int(root))
            dt = time.perf_counter() - t0
            runs.append((int((lv[src] >= 0).sum()), dt))
        q.put({"ok": True, "runs": runs})
    except Exception as e:
        q.put({"ok": False, "error": repr(e)})


def batch_arm(args, rank, world):
    """Many small Kronecker graphs (SCALE ~ U{8..14}, edge factor 16, graph g
    seeded 5*2^20+g), each RCM-relabelled with one random non-isolated root,
    packed and searched in one captured persistent launch.
    Metric: GTEPS = sum over graphs of m_g / launch time."""
    import numpy as np
    import torch
    import graphgen
    import paper_2012_10026_gb300 as g3

    local, world, dist = _setup_dist(args)
    specs = graphgen.small_graph_specs(args.batch_graphs, seed=5)
    graphs, roots_u, m_g, voff, srcs = [], [], [], [0], []
    t0 = time.perf_counter()
    for i, (scale, gseed) in enumerate(specs):
        n = 1 << scale
        s, d = graphgen.kronecker_edges_dev(scale, 16, seed=gseed)
        flags = graphgen.nonisolated_flags_dev(s, d, n).cpu().numpy()
        r = int(graphgen.pick_roots(flags, 1, seed=gseed)[0])
        g = g3.g3_build_csr(s, d, n)
        g3.g3_rcm_relabel(g)
        graphs.append(g)
        roots_u.append(voff[-1] + r)
        srcs.append(s.long() + voff[-1])
        voff.append(voff[-1] + n)
    b = g3.g3_batch_pack(graphs)
    for g in graphs:
        g.free()
    setup_s = time.perf_counter() - t0
    N = voff[-1]
    oracle_proc = None
    if rank == 0 and args.cpu_baseline:
        sample = [(specs[i][0], specs[i][1], roots_u[i] - voff[i]) for i in range(0, len(specs), 16)]
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        p = ctx.Process(target=_batch_oracle_worker, args=(sample, q))
        p.start()
        oracle_proc = (p, q, len(sample))
    roots = torch.tensor(roots_u, dtype=torch.int32, device="cuda")
    parent = torch.empty(N, dtype=torch.int32, device="cuda")
    level = torch.empty(N, dtype=torch.int32, device="cuda")
    tune_rec, t_tune = None, 0.0
    if args.batch_warp_max_n < 0:
        t_tune = time.perf_counter()
        o, tune_rec = g3.autotune_batch(b, roots, parent, level, args.tune_cache or None)
        t_tune = time.perf_counter() - t_tune
    else:
        o = g3.batch_opts(warp_max_n=args.batch_warp_max_n, mode=args.batch_mode)
    g3.g3_bfs_batch(b, roots, parent, level, o)
    src_all = torch.cat(srcs)
    del srcs
    m_total = int((level[src_all] >= 0).sum().item())
    del src_all
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev_s = torch.cuda.Event(enable_timing=True)
    ev_e = torch.cuda.Event(enable_timing=True)

    def step():
        flush.fill_(1)
        ev_s.record()
        g3.g3_bfs_batch(b, roots, parent, level, o, timed=False)
        ev_e.record()
        ev_e.synchronize()
        return ev_s.elapsed_time(ev_e)

    for _ in range(args.warmup):
        step()
    clk_path = os.path.join(tempfile.gettempdir(), f"g3_clocks_b_{rank}.csv")
    sampler = start_clock_sampler(clk_path)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = g3.kernel_launches()
    times = [step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    launches = g3.kernel_launches() - l0
    if dist:
        dist.barrier()
    clocks = stop_clock_sampler(sampler, clk_path, local)
    tsum = _max_over_ranks(dist, sum(times))
    value = world * args.steps * m_total / (tsum / 1e3) / 1e9
    # end to end: roots from pinned host memory in, parent/level to pinned host out
    e2e = None
    if not args.no_e2e:
        h_roots = roots.cpu().pin_memory()
        hp = torch.empty(N, dtype=torch.int32).pin_memory()
        hl = torch.empty(N, dtype=torch.int32).pin_memory()
        et = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            roots.copy_(h_roots, non_blocking=True)
            g3.g3_bfs_batch(b, roots, parent, level, o, timed=False)
            hp.copy_(parent, non_blocking=True)
            hl.copy_(level, non_blocking=True)
            torch.cuda.synchronize()
            if i >= args.warmup:
                et.append((time.perf_counter() - s0) * 1e3)
        e2e = {"value": m_total / (sum(et) / len(et) / 1e3) / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": len(roots_u) * 4, "d2h_bytes_per_step": 2 * N * 4}
    info = b.info
    comp = 8 * (N + 1) + 4 * info["nnz"] + 8 * N + 4 * N
    avg_ms = sum(times) / len(times)
    peak, peak_kind = load_peaks()
    cpu = None
    if oracle_proc is not None:
        p, q, ns = oracle_proc
        d = finish_oracle_leg(p, q, timeout=args.cpu_timeout)
        if d and d.get("ok"):
            runs = d["runs"]
            cpu = {"value": sum(x[0] for x in runs) / sum(x[1] for x in runs) / 1e9,
                   "unit": "GTEPS", "cores": 1, "kind": "oracle",
                   "sample": f"{ns} of the {len(specs)} graphs (every 16th), serial oracle "
                             f"BFS from the same root (generation and CSR untimed)"}
        else:
            cpu = {"value": None, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                   "sample": "oracle leg did not finish: " + (d or {}).get("error", "timeout")}
    if rank == 0:
        line = _common_line(args, world, f"GTEPS, {len(specs)} small Kronecker graphs "
                            "(SCALE 8-14) in one captured launch", value, "GTEPS", times,
                            {"workload": f"kronecker_batch{len(specs)}_scale8-14_ef16_rcm_1root",
                             "warp_max_n": o.warp_max_n, "mode": o.mode,
                             "l2": "256 MB write between launches (L2 flush)",
                             "parallelism": "replicas"})
        line.update({
            "roofline": {"bound": "hbm", "kernel": "batch_bfs (warp- and CTA-group launches)",
                         "achieved": comp / (avg_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": comp / (avg_ms / 1e3) / 1e9 / peak, "traffic": None,
                         "frac_of_nominal": comp / (avg_ms / 1e3) / 1e9 / NOMINAL_HBM_GBS,
                         "peak_kind": peak_kind, "bytes_per_launch": comp,
                         "bytes_model": "compulsory: union CSR once + parent/level written + "
                                        "label map read once"},
            "cpu_baseline": cpu, "gpu_launches": int(launches), "clocks": clocks, "e2e": e2e,
            "batch": {"graphs": len(specs), "N": N, "nnz": info["nnz"], "m_total": m_total,
                      "setup_s": setup_s},
            "autotune": None if tune_rec is None else dict(tune_rec.to_dict(), seconds=t_tune),
            "per_launch_ms": {"min": min(times), "median": statistics.median(times),
                              "max": max(times)},
        })
        print(json.dumps(line), flush=True)
    b.free()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.workload == "msbfs" and args.impl != "reference":
        return msbfs_arm(args, rank, world)
    if args.workload == "batch" and args.impl != "reference":
        return batch_arm(args, rank, world)
    if args.impl == "reference":
        reference_arm(args, rank, world)
    else:
        gpu_arm(args, rank, world)


if __name__ == "__main__":
    main()
