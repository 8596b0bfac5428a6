"""The host hybrid BFS (the paper's CPU design, Algorithms 4-6) against the
oracle: level[] bit-exact and parent[] valid on random graphs, star/path
closed forms and Kronecker graphs, for several thread counts and both
top-down forms; its bottom-up edge count equals the oracle's count for the
levels the direction rule sends bottom-up; its partitions are a descending
sequence that covers the bitmap. No GPU."""
import numpy as np
import pytest

import graphgen
import hostbfs
import oracle
from oracle import direction
from _graphs import path_graph, random_graph, star_graph


def _check(ref, n, hb, roots, **kw):
    for r in roots:
        p, l, st = hb.bfs(int(r), **kw)
        _, lo = oracle.bfs(ref["off"], ref["col"], int(r))
        assert np.array_equal(l, lo), r
        assert oracle.validate(ref["off"], ref["col"], int(r), p, l) == 0, r
    return st


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_random_graphs(threads):
    rng = np.random.default_rng(threads)
    for _ in range(30):
        n = int(rng.integers(1, 400))
        src, dst = random_graph(rng, n, int(rng.integers(0, 3 * n)))
        ref = oracle.pipeline(src, dst, n)
        hb = hostbfs.HostBFS(ref["off_r"], ref["col_r"], ref["old_of_new"], ref["new_of_old"],
                             n, threads=threads, lam=int(rng.integers(1, 30)))
        roots = rng.integers(0, n, 4)
        for kw in (dict(), dict(td_kind=1), dict(td_kind=2), dict(alpha=1 << 20, beta=1)):
            _check(ref, n, hb, roots, **kw)
        hb.close()


def test_closed_forms():
    n = 300
    ref = oracle.pipeline(*path_graph(n), n)
    hb = hostbfs.HostBFS(ref["off_r"], ref["col_r"], ref["old_of_new"], ref["new_of_old"], n,
                         threads=4)
    _, l, _ = hb.bfs(0)
    assert l.tolist() == list(range(n))
    ref = oracle.pipeline(*star_graph(50, 9), 50)
    hb = hostbfs.HostBFS(ref["off_r"], ref["col_r"], ref["old_of_new"], ref["new_of_old"], 50,
                         threads=4)
    _, l, _ = hb.bfs(9)
    assert l[9] == 0 and (l[np.arange(50) != 9] == 1).all()


@pytest.mark.parametrize("scale,threads", [(12, 2), (14, 8), (16, 5)])
def test_kronecker_and_bottom_up_edge_count(scale, threads):
    n = 1 << scale
    src, dst = graphgen.kronecker_edges(scale, 16, seed=scale)
    ref = oracle.pipeline(src, dst, n)
    hb = hostbfs.HostBFS(ref["off_r"], ref["col_r"], ref["old_of_new"], ref["new_of_old"], n,
                         threads=threads)
    roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 6, seed=3)
    for r in roots.tolist():
        p, l, st = hb.bfs(r)
        _, lo = oracle.bfs(ref["off"], ref["col"], r)
        assert np.array_equal(l, lo)
        assert oracle.validate(ref["off"], ref["col"], r, p, l) == 0
        lnew = lo[ref["old_of_new"][:ref["n_plus"]]]
        dirs = direction.heuristic_directions(ref["off_r"], lnew)
        want = sum(oracle.bu_examined(ref["off_r"], ref["col_r"], lnew, L, reverse=True)
                   for L, d in enumerate(dirs) if d == direction.BU)
        assert st["bu_examined"] == want
        assert st["levels"] == len(dirs) and st["bu_levels"] == dirs.count(direction.BU)


def test_isolated_root_and_unrelabelled_graph():
    n = 1 << 11
    src, dst = graphgen.kronecker_edges(11, 16, seed=4)
    off, col = oracle.build_csr(src, dst, n)
    iso = int(np.nonzero(np.diff(off) == 0)[0][0])
    hb = hostbfs.HostBFS(off, col, None, None, n, threads=4)
    p, l, _ = hb.bfs(iso)
    assert l[iso] == 0 and p[iso] == iso and (l >= 0).sum() == 1
    for r in graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 4, 5).tolist():
        p, l, _ = hb.bfs(r)
        _, lo = oracle.bfs(off, col, r)
        assert np.array_equal(l, lo) and oracle.validate(off, col, r, p, l) == 0
    with pytest.raises(ValueError):
        hb.bfs(n)


@pytest.mark.parametrize("blocks,nparts", [(1, 1), (10, 3), (1000, 40), (65536, 300)])
def test_partitions_descending_and_covering(blocks, nparts):
    b = hostbfs.partitions(blocks, nparts)
    assert b[0] == 0 and b[-1] == blocks and len(b) == nparts + 1
    sizes = np.diff(b)
    assert (sizes >= 0).all()
    # a descending arithmetic sequence up to rounding: consecutive sizes never
    # grow by more than one block, and the sequence falls from the first to
    # the last partition
    assert (np.diff(sizes) <= 1).all()
    if blocks >= 4 * nparts and nparts > 1:
        assert sizes[0] > sizes[-1]
