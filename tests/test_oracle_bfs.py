"""Pins the oracle BFS (Algorithm 1, serial) and validator (Sec. 2.1 rules)
to brute-force all-pairs distances, a library shortest-path routine, closed
forms and hand-worked fixtures; mutation tests check the validator."""
import numpy as np
import pytest
from conftest import read_golden_cases

import oracle
from _graphs import (adjacency_sets, complete_graph, cycle_graph, path_graph,
                     random_graph, star_graph)


def floyd_warshall_hops(src, dst, n):
    INF = 10 ** 9
    D = np.full((n, n), INF, np.int64)
    np.fill_diagonal(D, 0)
    for u, v in zip(src.tolist(), dst.tolist()):
        if u != v:
            D[u, v] = D[v, u] = 1
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return np.where(D >= INF, -1, D)


@pytest.mark.parametrize("seed", range(30))
def test_bfs_level_equals_floyd_warshall(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 48))
    m = int(rng.integers(0, 3 * n))
    src, dst = random_graph(rng, n, m)
    off, col = oracle.build_csr(src, dst, n)
    D = floyd_warshall_hops(src, dst, n)
    for root in range(n):
        parent, level = oracle.bfs(off, col, root)
        assert np.array_equal(level, D[root]), (root, level, D[root])
        assert oracle.validate(off, col, root, parent, level) == 0


def test_bfs_level_equals_scipy_shortest_path():
    scipy_sp = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp
    import graphgen
    src, dst = graphgen.kronecker_edges(11, 16, seed=3)
    n = 1 << 11
    off, col = oracle.build_csr(src, dst, n)
    A = sp.csr_matrix((np.ones(len(col)), col, off), shape=(n, n))
    for root in [0, 5, 77, 1024, 2047]:
        d = scipy_sp.shortest_path(A, unweighted=True, indices=root, directed=False)
        expect = np.where(np.isinf(d), -1, d).astype(np.int64)
        parent, level = oracle.bfs(off, col, root)
        assert np.array_equal(level, expect)
        assert oracle.validate(off, col, root, parent, level) == 0


@pytest.mark.parametrize("n", [1, 2, 3, 10, 33])
def test_bfs_closed_forms(n):
    # path from an endpoint: level i
    if n >= 2:
        off, col = oracle.build_csr(*path_graph(n), n)
        _, level = oracle.bfs(off, col, 0)
        assert level.tolist() == list(range(n))
    # cycle C_n from 0: min(i, n-i)
    if n >= 3:
        off, col = oracle.build_csr(*cycle_graph(n), n)
        _, level = oracle.bfs(off, col, 0)
        assert level.tolist() == [min(i, n - i) for i in range(n)]
    # star from the centre: every leaf at 1; from a leaf: centre 1, others 2
    if n >= 2:
        off, col = oracle.build_csr(*star_graph(n, 0), n)
        _, level = oracle.bfs(off, col, 0)
        assert level.tolist() == [0] + [1] * (n - 1)
        _, level = oracle.bfs(off, col, n - 1)
        assert level[0] == 1 and level[n - 1] == 0
        assert all(level[i] == 2 for i in range(1, n - 1))
    # complete graph: every other vertex at 1
    if n >= 2:
        off, col = oracle.build_csr(*complete_graph(n), n)
        p, level = oracle.bfs(off, col, 1)
        assert level.tolist() == [1 if i != 1 else 0 for i in range(n)]
        assert all(p[i] == 1 for i in range(n))


def test_bfs_golden_cases():
    for case in read_golden_cases("rcm_bfs_cases.txt"):
        off, col = oracle.build_csr(np.array(case["src"], np.int32),
                                    np.array(case["dst"], np.int32), case["n"])
        for root, expect in case["bfs"]:
            parent, level = oracle.bfs(off, col, root)
            assert level.tolist() == expect, (case["name"], root)
            assert oracle.validate(off, col, root, parent, level) == 0


def test_bfs_parent_is_first_discoverer():
    # star with centre 2 plus edge 0-1: from root 0 the BFS tree is 0-1 and
    # 0-2; vertex 3 and 4 hang off 2; serial order makes parent[3] == 2
    src = np.array([0, 0, 2, 2], np.int32)
    dst = np.array([1, 2, 3, 4], np.int32)
    off, col = oracle.build_csr(src, dst, 5)
    parent, level = oracle.bfs(off, col, 0)
    assert parent.tolist() == [0, 0, 0, 2, 2]
    assert level.tolist() == [0, 1, 1, 2, 2]


def _valid_instance(seed=5, n=40):
    rng = np.random.default_rng(seed)
    src, dst = random_graph(rng, n, 3 * n)
    off, col = oracle.build_csr(src, dst, n)
    root = int(np.argmax(np.diff(off)))
    parent, level = oracle.bfs(off, col, root)
    return off, col, root, parent, level


def test_validator_mutations_fail():
    off, col, root, parent, level = _valid_instance()
    assert oracle.validate(off, col, root, parent, level) == 0
    reached = [v for v in range(len(level)) if level[v] > 0]
    # 1: root's own parent wrong
    p = parent.copy(); p[root] = reached[0]
    assert oracle.validate(off, col, root, p, level)[0] == 1
    # 2: parent that is not a neighbour / wrong level
    v = reached[-1]
    non_nb = [u for u in range(len(level))
              if u != v and u not in col[off[v]:off[v + 1]] and level[u] == level[v] - 1]
    if non_nb:
        p = parent.copy(); p[v] = non_nb[0]
        assert oracle.validate(off, col, root, p, level)[0] == 2
    lv = level.copy(); lv[v] += 1
    assert oracle.validate(off, col, root, parent, lv)[0] in (2, 5)
    # 4: parent set on an unreached vertex
    unreached = [u for u in range(len(level)) if level[u] < 0]
    if unreached:
        p = parent.copy(); p[unreached[0]] = root
        assert oracle.validate(off, col, root, p, level)[0] == 4
    # 4: a reached vertex marked unreached in both arrays breaks rule 5
    p = parent.copy(); lv = level.copy()
    leaf = max(reached, key=lambda u: level[u])
    p[leaf] = -1; lv[leaf] = -1
    assert oracle.validate(off, col, root, p, lv)[0] == 5
    # 3: a second level-0 vertex
    lv = level.copy(); p = parent.copy(); u = reached[0]
    lv[u] = 0; p[u] = u
    assert oracle.validate(off, col, root, p, lv)[0] == 3


def test_validator_rejects_shortcut_levels():
    # path 0-1-2-3 with a consistent-looking but too deep labelling
    off, col = oracle.build_csr(*path_graph(4), 4)
    parent = np.array([0, 0, 1, 2], np.int32)
    level = np.array([0, 1, 2, 3], np.int32)
    assert oracle.validate(off, col, 0, parent, level) == 0
    # a triangle 0-1-2 plus 2-3: claiming level 2 for vertex 2 breaks rule 5
    src = np.array([0, 1, 0, 2], np.int32); dst = np.array([1, 2, 2, 3], np.int32)
    off, col = oracle.build_csr(src, dst, 4)
    parent = np.array([0, 0, 1, 2], np.int32)
    level = np.array([0, 1, 2, 3], np.int32)
    assert oracle.validate(off, col, 0, parent, level)[0] == 5


def test_bu_examined_brute_force():
    rng = np.random.default_rng(9)
    for _ in range(20):
        n = int(rng.integers(2, 40))
        src, dst = random_graph(rng, n, 3 * n)
        off, col = oracle.build_csr(src, dst, n)
        _, level = oracle.bfs(off, col, 0)
        for L in range(int(level.max()) + 1):
            for rev in (False, True):
                expect = 0
                for v in range(n):
                    if 0 <= level[v] <= L:
                        continue
                    row = col[off[v]:off[v + 1]].tolist()
                    if rev:
                        row = row[::-1]
                    k = 0
                    for w in row:
                        k += 1
                        if level[w] == L:
                            break
                    expect += k
                assert oracle.bu_examined(off, col, level, L, rev) == expect


@pytest.mark.parametrize("n", [3, 4, 9, 20])
def test_bu_examined_closed_forms(n):
    # path 0-1-...-(n-1) from root 0, levels equal IDs. At step L the unvisited
    # vertices are L+1..n-1: vertex L+1 hits on its first neighbour (L), the
    # interior ones scan both neighbours, the end one its single neighbour.
    off, col = oracle.build_csr(*path_graph(n), n)
    _, level = oracle.bfs(off, col, 0)
    for L in range(n - 2):
        assert oracle.bu_examined(off, col, level, L) == 2 * (n - L - 2)
        assert oracle.bu_examined(off, col, level, L, reverse=True) == 2 * (n - L - 2) + 1
    # star from the centre: each leaf examines exactly its one neighbour
    off, col = oracle.build_csr(*star_graph(n, 0), n)
    _, level = oracle.bfs(off, col, 0)
    assert oracle.bu_examined(off, col, level, 0) == n - 1
    # after the last level nothing is found: every unvisited row is scanned
    assert oracle.bu_examined(off, col, level, 1) == 0


def test_validate_tree_equals_validate_when_levels_exact():
    """validate_tree (rules 1-4) decides like validate whenever level[] is
    the oracle's: on random valid BFS trees (any neighbour one level up as
    parent) and on parent mutations of each kind."""
    rng = np.random.default_rng(21)
    for _ in range(40):
        n = int(rng.integers(5, 60))
        src, dst = random_graph(rng, n, int(rng.integers(n, 3 * n)))
        off, col = oracle.build_csr(src, dst, n)
        root = int(rng.integers(0, n))
        _, level = oracle.bfs(off, col, root)
        parent = np.full(n, -1, np.int32)
        parent[root] = root
        for v in range(n):
            if level[v] > 0:
                up = [u for u in col[off[v]:off[v + 1]] if level[u] == level[v] - 1]
                parent[v] = up[int(rng.integers(0, len(up)))]
        assert oracle.validate(off, col, root, parent, level) == 0
        assert oracle.validate_tree(off, col, root, parent, level) == 0
        reached = [v for v in range(n) if level[v] > 0]
        for v in reached[:5]:
            for u in range(n):
                if u == parent[v]:
                    continue
                p = parent.copy()
                p[v] = u
                a = oracle.validate(off, col, root, p, level)
                b = oracle.validate_tree(off, col, root, p, level)
                assert (a == 0) == (b == 0)
                if a:
                    assert a == b
    off, col, root, parent, level = _valid_instance()
    p = parent.copy(); p[root] = int(np.flatnonzero(level > 0)[0])
    assert oracle.validate_tree(off, col, root, p, level)[0] == 1
