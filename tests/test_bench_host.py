"""bench.py's host-side logic (no GPU): the TEPS mean, the per-level
algorithmic-bytes model and the oracle parity pass (with the oracle's own
results in the GPU's place, and planted errors)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_harmonic_gteps_hand_values():
    # two searches of 1e9 edges in 1 s and 0.5 s: rates 1 and 2 GTEPS, harmonic
    # mean 2 / (1 + 0.5) = 4/3
    assert bench.harmonic_gteps([10 ** 9, 10 ** 9], [1000.0, 500.0]) == pytest.approx(4 / 3)
    assert bench.harmonic_gteps([5 * 10 ** 8], [250.0]) == pytest.approx(2.0)


def test_level_bytes_model_hand_values():
    nb = 64  # two bitmap words
    bu = {"dir": 1, "n_u": 10, "examined": 7, "n_next": 3, "n_f": 0, "m_f": 0}
    # 4*2 visited words + 8*10 row bounds + 8*7 probes + 8*3 outputs + 8*2 writes
    assert bench.level_bytes(bu, nb) == 8 + 80 + 56 + 24 + 16
    td = {"dir": 0, "n_f": 5, "m_f": 40, "n_next": 6, "n_u": 0, "examined": 0}
    # 20 per frontier vertex + 8 per edge + 16 per new vertex
    assert bench.level_bytes(td, nb) == 100 + 320 + 96


def _parity_case(scale, nroots):
    import graphgen
    import oracle
    n = 1 << scale
    src, dst = graphgen.kronecker_edges(scale, 16, seed=1)
    roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), nroots, 2).tolist()
    off, col = oracle.build_csr(src, dst, n)
    P, _ = oracle.rcm(off, col)
    outs = [oracle.bfs(off, col, r) for r in roots]
    m_r = {r: int((lv[src] >= 0).sum()) for r, (_, lv) in zip(roots, outs)}
    return roots, outs, P, m_r


def test_parity_leg_accepts_oracle_results_and_flags_planted_errors():
    """The bench's oracle pass on the CPU, with the oracle's own results in
    the GPU's place: all roots pass; a planted level error, a planted parent
    error and a swapped permutation entry are each reported."""
    roots, outs, P, m_r = _parity_case(12, 6)
    leg = bench.ParityLeg(12, 16, 1, 2, 6)
    rec, cpu = leg.check(roots, m_r, lambda i: outs[i], P)
    assert rec["roots_checked"] == 6 and rec["level_exact"] == 6
    assert rec["parent_valid"] == 6 and rec["perm_exact"] is True
    assert cpu["value"] > 0 and cpu["cores"] >= 1 and cpu["kind"] == "oracle"

    bad = [(p.copy(), lv.copy()) for p, lv in outs]
    v = int(np.flatnonzero(bad[1][1] > 1)[0])
    bad[1][1][v] += 1                      # a wrong level
    w = int(np.flatnonzero(bad[3][1] > 1)[0])
    bad[3][0][w] = roots[3]                # a parent that is not a neighbour one level up
    Q = P.copy()
    Q[[0, 1]] = Q[[1, 0]]
    rec, _ = leg.check(roots, m_r, lambda i: bad[i], Q)
    assert rec["level_exact"] == 5 and rec["parent_valid"] == 4
    assert rec["perm_exact"] is False
    assert {f["root"] for f in rec["failures"]} == {roots[1], roots[3]}


def test_parity_leg_rejects_other_roots():
    roots, outs, P, m_r = _parity_case(10, 3)
    leg = bench.ParityLeg(10, 16, 1, 2, 3)
    other = list(reversed(roots))
    rec, cpu = leg.check(other, m_r, lambda i: outs[i], P)
    assert "error" in rec and cpu is None


def test_oracle_threads_bounds():
    assert 1 <= bench.oracle_threads(1 << 26, 64) <= max(1, bench.host_cores() - 1)
    assert bench.oracle_threads(1 << 10, 1) == 1


def test_level_kinds_and_graph_kernel_count():
    """Roofline split and the level-loop kernel count: dense bottom-up levels
    (at least 4 % of the graph unvisited) are the word-pair kernel's, sparse
    ones the vertex-list kernels'; the count follows the loop's structure."""
    nb = 100000

    def lv(level, d, n_u, ms=0.1):
        return {"level": level, "dir": d, "n_u": n_u, "n_f": 10, "m_f": 100,
                "examined": 50, "n_next": 5, "ms_expand": ms}
    # TD (level 0), TD, BU dense, BU dense, BU sparse, TD, TD
    st = [lv(0, 0, nb - 1), lv(1, 0, nb - 50), lv(2, 1, 90000), lv(3, 1, 5000),
          lv(4, 1, 3999), lv(5, 0, 100), lv(6, 0, 90)]
    kinds = [bench.level_kind(s, nb) for s in st]
    assert kinds == ["td", "td", "bu", "bu", "bu_list", "td", "td"]
    agg = bench.roofline_levels([st], nb)
    assert agg["bu"][2] == 2 and agg["bu_list"][2] == 1 and agg["td"][2] == 4
    assert agg["bu"][0] == bench.level_bytes(st[2], nb) + bench.level_bytes(st[3], nb)
    # level 0: 2; level 1: 1 + 2; level 2: 1 + 1 + 2 (queue -> bitmap);
    # level 3: 1 + 1; level 4: 1 + 2; level 5 after the list level: 1 + 2;
    # level 6: 1 + 2; the final controller: 1
    assert bench.graph_kernel_count([st], nb) == 2 + 3 + 4 + 2 + 3 + 3 + 3 + 1
    # a top-down level after a word-pair bottom-up level converts the bitmap
    st2 = [lv(0, 0, nb - 1), lv(1, 1, 90000), lv(2, 0, 100)]
    assert bench.graph_kernel_count([st2], nb) == 2 + (1 + 1 + 2) + (1 + 2 + 1) + 1
