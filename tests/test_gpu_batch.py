"""Batched BFS over many small relabelled graphs against one oracle BFS per graph."""
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


def _graph_set(count, seed):
    """Small Kronecker graphs (SCALE 8..14, edge factor 16) plus a few shapes
    that stress the level loop: a long path (many levels), a star (one huge
    level), a sparse random graph with many isolated vertices."""
    out = []
    for scale, gseed in graphgen.small_graph_specs(count, seed=seed):
        s, d = graphgen.kronecker_edges(scale, 16, seed=gseed)
        out.append((s, d, 1 << scale))
    out.append((*path_graph(3000), 3000))
    out.append((*star_graph(500, 7), 500))
    rng = np.random.default_rng(seed)
    out.append((*random_graph(rng, 900, 300), 900))
    return out


def _pack(graphs):
    built = []
    for s, d, n in graphs:
        g = g3.g3_build_csr(_dev(s), _dev(d), n)
        g3.g3_rcm_relabel(g)
        built.append(g)
    b = g3.g3_batch_pack(built)
    for g in built:  # the batch holds its own copy
        g.free()
    return b


def _check(graphs, roots_local, parent, level):
    vb = 0
    for (s, d, n), r in zip(graphs, roots_local):
        off, col = oracle.build_csr(s, d, n)
        p = parent[vb:vb + n]
        lv = level[vb:vb + n]
        if r < 0:
            assert (p == -1).all() and (lv == -1).all()
        else:
            _, want = oracle.bfs(off, col, r)
            assert np.array_equal(lv, want), (n, r)
            local = np.where(p >= 0, p - vb, -1).astype(np.int32)
            assert oracle.validate(off, col, r, local, lv) == 0, (n, r)
        vb += n


GRAPHS = _graph_set(40, seed=5)


@pytest.fixture(scope="module")
def batch():
    b = _pack(GRAPHS)
    yield b
    b.free()


def _roots(graphs, seed):
    rng = np.random.default_rng(seed)
    roots = []
    for s, d, n in graphs:
        deg = np.bincount(np.concatenate([s, d]), minlength=n)
        nz = np.nonzero(deg)[0]
        roots.append(int(rng.choice(nz)) if len(nz) else 0)
    return roots


@pytest.mark.parametrize("warp_max_n,mode", [(0, 0), (256, 0), (1024, 0), (1 << 30, 0),
                                             (1024, 1)])
def test_batch_levels_equal_oracle(batch, warp_max_n, mode):
    info = batch.info
    assert info["G"] == len(GRAPHS)
    assert info["N"] == sum(n for _, _, n in GRAPHS)
    voff = np.cumsum([0] + [n for _, _, n in GRAPHS])
    for seed in (1, 2):
        roots = _roots(GRAPHS, seed)
        d_roots = _dev(np.asarray(roots) + voff[:-1])
        parent = torch.full((info["N"],), 7, dtype=torch.int32, device="cuda")
        level = torch.full((info["N"],), 7, dtype=torch.int32, device="cuda")
        ms = g3.g3_bfs_batch(batch, d_roots, parent, level,
                             g3.batch_opts(warp_max_n=warp_max_n, mode=mode))
        assert ms > 0
        _check(GRAPHS, roots, parent.cpu().numpy(), level.cpu().numpy())


def test_batch_relaunch_reuses_capture(batch):
    """Same buffers twice (the second call only launches the captured graph),
    then new roots written into the same root buffer."""
    info = batch.info
    voff = np.cumsum([0] + [n for _, _, n in GRAPHS])
    roots = _roots(GRAPHS, 3)
    d_roots = _dev(np.asarray(roots) + voff[:-1])
    parent = torch.empty((info["N"],), dtype=torch.int32, device="cuda")
    level = torch.empty((info["N"],), dtype=torch.int32, device="cuda")
    launches0 = g3.kernel_launches()
    g3.g3_bfs_batch(batch, d_roots, parent, level)
    g3.g3_bfs_batch(batch, d_roots, parent, level)
    assert g3.kernel_launches() - launches0 == 2  # one persistent kernel per launch
    _check(GRAPHS, roots, parent.cpu().numpy(), level.cpu().numpy())
    roots = _roots(GRAPHS, 4)
    d_roots.copy_(_dev(np.asarray(roots) + voff[:-1]))
    g3.g3_bfs_batch(batch, d_roots, parent, level)
    _check(GRAPHS, roots, parent.cpu().numpy(), level.cpu().numpy())


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_isolated_and_foreign_roots(mode):
    graphs = GRAPHS[:1] + GRAPHS[-1:] + GRAPHS[1:6]  # graph 1: the sparse random one
    b = _pack(graphs)
    N = b.info["N"]
    voff = np.cumsum([0] + [n for _, _, n in graphs])
    roots = _roots(graphs, 9)
    # graph 1: an isolated root; graph 2: a root inside graph 3's range
    s1, d1, n1 = graphs[1]
    deg1 = np.bincount(np.concatenate([s1, d1]), minlength=n1)
    iso = np.nonzero(deg1 == 0)[0]
    assert len(iso)
    roots[1] = int(iso[0])
    glob = (np.asarray(roots) + voff[:-1]).astype(np.int64)
    glob[2] = voff[3]
    parent = torch.empty((N,), dtype=torch.int32, device="cuda")
    level = torch.empty((N,), dtype=torch.int32, device="cuda")
    g3.g3_bfs_batch(b, _dev(glob), parent, level, g3.batch_opts(mode=mode))
    roots[2] = -1
    p, lv = parent.cpu().numpy(), level.cpu().numpy()
    _check(graphs, roots, p, lv)
    one = slice(voff[1], voff[2])
    assert (lv[one] >= 0).sum() == 1 and p[voff[1] + iso[0]] == voff[1] + iso[0]
    b.free()


def test_batch_pack_rejects_bad_graphs():
    s, d = graphgen.kronecker_edges(9, 16, seed=1)
    g = g3.g3_build_csr(_dev(s), _dev(d), 1 << 9)
    with pytest.raises(g3.G3Error):
        g3.g3_batch_pack([g])  # not relabelled
    s2, d2 = path_graph(20000)
    big = g3.g3_build_csr(_dev(s2), _dev(d2), 20000)
    g3.g3_rcm_relabel(big)
    with pytest.raises(g3.G3Error):
        g3.g3_batch_pack([big])  # more than 16384 BFS vertices
    g.free()
    big.free()
