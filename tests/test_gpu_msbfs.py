"""Bit-sliced multi-source BFS against one oracle BFS per source."""
import numpy as np
import pytest

import graphgen
import oracle
from _graphs import path_graph, random_graph, star_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_10026_gb300 as g3  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _run(g, n, roots, **kw):
    lv = torch.full((len(roots), n), 99, dtype=torch.int8, device="cuda")
    nl, ms = g3.g3_msbfs(g, roots, lv, g3.msbfs_opts(**kw) if kw else None)
    return lv.cpu().numpy(), nl, ms


def _expect(off, col, roots):
    return np.stack([oracle.bfs(off, col, r)[1] for r in roots]).astype(np.int8)


def _cases():
    out = []
    rng = np.random.default_rng(5)
    for i in range(6):
        n = int(rng.integers(2, 400))
        s, d = random_graph(rng, n, int(rng.integers(n // 2, 3 * n)))
        out.append((f"random{i}", s, d, n))
    s, d = graphgen.kronecker_edges(12, 16, seed=4)
    out.append(("kron12", s, d, 1 << 12))
    s, d = graphgen.chunglu_edges(5000, seed=3)
    out.append(("chunglu5000", s, d, 5000))
    out.append(("star", *star_graph(100, 3), 100))
    # rows longer than one 2048-entry work chunk: split hubs in push and pull
    out.append(("star20k", *star_graph(20000, 5), 20000))
    s, d = graphgen.kronecker_edges(16, 16, seed=8)
    out.append(("kron16", s, d, 1 << 16))
    out.append(("path100", *path_graph(100), 100))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("relabel", [True, False])
@pytest.mark.parametrize("kw", [dict(), dict(push_alpha=1 << 30), dict(push_alpha=1),
                                dict(pull_warp_deg=1), dict(pull_warp_deg=1 << 30)],
                         ids=["default", "always_pull", "mostly_push", "all_warp", "no_warp"])
def test_msbfs_levels_equal_oracle(case, relabel, kw):
    name, src, dst, n = case
    off, col = oracle.build_csr(src, dst, n)
    g = g3.g3_build_csr(_dev(src), _dev(dst), n)
    if relabel:
        g3.g3_rcm_relabel(g)
    rng = np.random.default_rng(n)
    for k in (1, 7, 64):
        roots = rng.integers(0, n, k).tolist()
        lv, nl, ms = _run(g, n, roots, **kw)
        assert np.array_equal(lv, _expect(off, col, roots)), (name, k)
        # a non-isolated root gives at least one level to expand
        assert ms > 0 and (nl >= 1 or not (np.diff(off)[roots] > 0).any())
    g.free()


def test_msbfs_duplicate_and_isolated_roots():
    src, dst = graphgen.kronecker_edges(11, 8, seed=6)
    n = 1 << 11
    off, col = oracle.build_csr(src, dst, n)
    deg = np.diff(off)
    iso = np.nonzero(deg == 0)[0][:3].tolist()
    hub = int(np.argmax(deg))
    roots = [hub, hub, iso[0], 5, iso[1], hub, 5] + list(range(20, 77))
    roots = roots[:64]
    g = g3.g3_build_csr(_dev(src), _dev(dst), n)
    g3.g3_rcm_relabel(g)
    lv, _, _ = _run(g, n, roots)
    assert np.array_equal(lv, _expect(off, col, roots))
    assert (lv[2] >= 0).sum() == 1 and lv[2][iso[0]] == 0
    g.free()


def test_msbfs_level_range_and_bad_args():
    n = 200
    src, dst = path_graph(n)
    g = g3.g3_build_csr(_dev(src), _dev(dst), n)
    lv = torch.empty((1, n), dtype=torch.int8, device="cuda")
    with pytest.raises(g3.G3Error) as e:
        g3.g3_msbfs(g, [0], lv)  # levels up to 199 do not fit int8
    assert e.value.status == g3.G3_ERANGE
    # 126 levels still fit: root in the middle of a 253-vertex path
    n2 = 253
    s2, d2 = path_graph(n2)
    g2 = g3.g3_build_csr(_dev(s2), _dev(d2), n2)
    lv2 = torch.empty((1, n2), dtype=torch.int8, device="cuda")
    g3.g3_msbfs(g2, [126], lv2)
    assert lv2.cpu().numpy()[0].max() == 126
    with pytest.raises(g3.G3Error):
        g3.g3_msbfs(g, list(range(65)), torch.empty((65, n), dtype=torch.int8, device="cuda"))
    with pytest.raises(g3.G3Error):
        g3.g3_msbfs(g, [n], lv)
    g.free()
    g2.free()


def test_msbfs_work_counts():
    src, dst = graphgen.kronecker_edges(12, 16, seed=4)
    n = 1 << 12
    off, col = oracle.build_csr(src, dst, n)
    deg = np.diff(off)
    g = g3.g3_build_csr(_dev(src), _dev(dst), n)
    g3.g3_rcm_relabel(g)
    root = int(np.argmax(deg))
    _, lref = oracle.bfs(off, col, root)
    # push only, one source: every reached vertex is pushed once
    lv, nl, _ = _run(g, n, [root], push_alpha=1)
    st = g3.g3_msbfs_last_stats(g)
    assert st["levels"] == nl == st["push_levels"] and st["pull_levels"] == 0
    assert st["push_entries"] == int(deg[lref >= 0].sum())
    assert st["pull_entries"] == 0 and st["pull_vertices"] == 0
    # pull only: each pull level scans the vertices not yet reached by every
    # source; one source -> the unreached vertices of the level, early exits
    lv, nl, _ = _run(g, n, [root], push_alpha=1 << 30)
    st = g3.g3_msbfs_last_stats(g)
    assert st["pull_levels"] == nl and st["push_levels"] == 0
    nb = g.info["n_bfs"]
    reached_by = [int(((lref >= 0) & (lref <= L) & (deg > 0)).sum()) for L in range(nl)]
    assert st["pull_vertices"] == sum(nb - r for r in reached_by)
    assert 0 < st["pull_entries"] <= int(deg.sum()) * nl
    g.free()
