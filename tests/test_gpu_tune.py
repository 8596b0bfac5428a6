"""Autotuner on the device: picks a candidate no slower than its start,
caches it, reuses the cache without launching anything, and the tuned
options still give the oracle's levels."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_10026_gb300 as g3  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


@pytest.fixture(scope="module")
def kron14():
    src, dst = graphgen.kronecker_edges(14, 16, seed=11)
    n = 1 << 14
    off, col = oracle.build_csr(src, dst, n)
    g = g3.g3_build_csr(_dev(src), _dev(dst), n)
    g3.g3_rcm_relabel(g)
    roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 3, 4).tolist()
    yield g, off, col, n, roots
    g.free()


def test_autotune_bfs_cache_and_parity(kron14, tmp_path):
    g, off, col, n, roots = kron14
    cache = str(tmp_path / "tune.txt")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    o, rec = g3.autotune_bfs(g, roots, parent, level, cache)
    assert rec.points > 10 and rec.ms <= rec.ms_default
    assert rec.kind == g3.G3_TUNE_BFS
    assert (rec.size_class, rec.deg_class) == g3.tune_key(g3.G3_TUNE_BFS, g.info["n_bfs"],
                                                          g.info["nnz"])
    assert list(rec.p) == [o.alpha, o.beta, o.t1, o.t2, o.t3, o.bu_reverse | (o.bu_kernel << 1)]
    assert o.t1 < o.t2 < o.t3 and o.bu_reverse in (0, 1) and o.bu_kernel in (0, 1, 3)
    # second call: a cache hit, nothing launched
    l0 = g3.kernel_launches()
    o2, rec2 = g3.autotune_bfs(g, roots, parent, level, cache)
    assert g3.kernel_launches() == l0 and rec2.points == 0
    assert list(rec2.p) == list(rec.p)
    for r in roots:
        g3.g3_bfs(g, r, parent, level, o2)
        _, want = oracle.bfs(off, col, r)
        assert np.array_equal(level.cpu().numpy(), want)
        assert oracle.validate(off, col, r, parent.cpu().numpy(), want) == 0


def test_autotune_msbfs(kron14, tmp_path):
    g, off, col, n, roots = kron14
    cache = str(tmp_path / "tune.txt")
    srcs = list(range(0, n, n // 40))[:40] + roots
    lv = torch.empty((len(srcs), n), dtype=torch.int8, device="cuda")
    o, rec = g3.autotune_msbfs(g, srcs, lv, cache)
    assert rec.points == 7 * 8 and rec.ms <= rec.ms_default
    assert (rec.p[0], rec.p[1]) == (o.push_alpha, o.pull_warp_deg)
    _, rec2 = g3.autotune_msbfs(g, srcs, lv, cache)
    assert rec2.points == 0
    g3.g3_msbfs(g, srcs, lv, o)
    want = np.stack([oracle.bfs(off, col, s)[1] for s in srcs]).astype(np.int8)
    assert np.array_equal(lv.cpu().numpy(), want)


def test_autotune_batch(tmp_path):
    graphs, voff, roots = [], [0], []
    specs = graphgen.small_graph_specs(24, seed=7)
    host = []
    for scale, gseed in specs:
        s, d = graphgen.kronecker_edges(scale, 16, seed=gseed)
        n = 1 << scale
        g = g3.g3_build_csr(_dev(s), _dev(d), n)
        g3.g3_rcm_relabel(g)
        graphs.append(g)
        r = int(graphgen.pick_roots(graphgen.nonisolated_flags(s, d, n), 1, gseed)[0])
        roots.append(voff[-1] + r)
        host.append((s, d, n, r))
        voff.append(voff[-1] + n)
    b = g3.g3_batch_pack(graphs)
    for g in graphs:
        g.free()
    N = voff[-1]
    d_roots = _dev(roots)
    parent = torch.empty(N, dtype=torch.int32, device="cuda")
    level = torch.empty(N, dtype=torch.int32, device="cuda")
    cache = str(tmp_path / "tune.txt")
    o, rec = g3.autotune_batch(b, d_roots, parent, level, cache)
    assert rec.points == 8 and rec.ms <= rec.ms_default
    assert (rec.p[0], rec.p[1]) == (o.warp_max_n, o.mode)
    _, rec2 = g3.autotune_batch(b, d_roots, parent, level, cache)
    assert rec2.points == 0 and (rec2.p[0], rec2.p[1]) == (o.warp_max_n, o.mode)
    g3.g3_bfs_batch(b, d_roots, parent, level, o)
    p, lv = parent.cpu().numpy(), level.cpu().numpy()
    for (s, d, n, r), vb in zip(host, voff):
        off, col = oracle.build_csr(s, d, n)
        _, want = oracle.bfs(off, col, r)
        assert np.array_equal(lv[vb:vb + n], want)
        local = np.where(p[vb:vb + n] >= 0, p[vb:vb + n] - vb, -1).astype(np.int32)
        assert oracle.validate(off, col, r, local, want) == 0
    b.free()
