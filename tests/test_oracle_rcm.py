"""Pins the oracle RCM (Algorithm 3) to an independent level-sort
restatement, hand-worked fixtures, closed forms on path/band/star graphs and
invariants stated in Sec. 3.2."""
import numpy as np
import pytest
from conftest import read_golden_cases

import oracle
from _graphs import adjacency_sets, band_graph, path_graph, random_graph, star_graph


def rcm_by_level_sort(src, dst, n):
    """Independent restatement (not Algorithm 3's queue): components are
    taken in order of their minimal (degree, id) vertex, which starts them;
    inside a component, BFS level k+1 is ordered by (position of the
    earliest-placed neighbour in level k, degree, id). Reversed, then the
    isolated vertices in ascending order."""
    adj = adjacency_sets(src, dst, n)
    deg = [len(a) for a in adj]
    # components by union-find
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for u in range(n):
        for w in adj[u]:
            ru, rw = find(u), find(w)
            if ru != rw:
                parent[ru] = rw
    comps = {}
    for v in range(n):
        if deg[v] > 0:
            comps.setdefault(find(v), []).append(v)
    starts = sorted(min(c, key=lambda v: (deg[v], v)) for c in comps.values())
    starts.sort(key=lambda v: (deg[v], v))
    order, pos = [], {}
    for s in starts:
        pos[s] = len(order)
        order.append(s)
        level = [s]
        while level:
            cand = {}
            for v in level:
                for w in adj[v]:
                    if w not in pos:
                        cand[w] = min(cand.get(w, 1 << 60), pos[v])
            nxt = sorted(cand, key=lambda w: (cand[w], deg[w], w))
            for w in nxt:
                pos[w] = len(order)
                order.append(w)
            level = nxt
    n_plus = len(order)
    return order[::-1] + [v for v in range(n) if deg[v] == 0], n_plus


@pytest.mark.parametrize("block", range(10))
def test_rcm_equals_level_sort_restatement(block):
    rng = np.random.default_rng(1000 + block)
    for _ in range(300):
        n = int(rng.integers(1, 15))
        m = int(rng.integers(0, 2 * n + 1))
        src, dst = random_graph(rng, n, m)
        off, col = oracle.build_csr(src, dst, n)
        P, n_plus = oracle.rcm(off, col)
        P2, n_plus2 = rcm_by_level_sort(src, dst, n)
        assert n_plus == n_plus2
        assert P.tolist() == P2, (src.tolist(), dst.tolist())


def test_rcm_equals_level_sort_on_kronecker():
    import graphgen
    src, dst = graphgen.kronecker_edges(9, 8, seed=4)
    n = 1 << 9
    off, col = oracle.build_csr(src, dst, n)
    P, n_plus = oracle.rcm(off, col)
    P2, n_plus2 = rcm_by_level_sort(src, dst, n)
    assert n_plus == n_plus2 and P.tolist() == P2


def test_rcm_golden_cases():
    for case in read_golden_cases("rcm_bfs_cases.txt"):
        off, col = oracle.build_csr(np.array(case["src"], np.int32),
                                    np.array(case["dst"], np.int32), case["n"])
        P, n_plus = oracle.rcm(off, col)
        assert P.tolist() == case["P"], case["name"]
        assert n_plus == case["n_plus"], case["name"]


@pytest.mark.parametrize("n", [2, 3, 10, 57])
def test_rcm_path_is_reversal(n):
    # Cuthill-McKee from the minimal-degree endpoint 0 visits 0,1,..,n-1, so
    # the reverse permutation maps vertex i to label n-1-i: bandwidth 1.
    off, col = oracle.build_csr(*path_graph(n), n)
    P, n_plus = oracle.rcm(off, col)
    assert n_plus == n
    assert P.tolist() == list(range(n - 1, -1, -1))
    _, new_of_old = oracle.permutation_arrays(P)
    assert oracle.bandwidth(off, col, new_of_old) == 1


@pytest.mark.parametrize("n,b", [(12, 2), (30, 3), (40, 5), (25, 1)])
def test_rcm_band_graph(n, b):
    # identity-labelled band: CM from vertex 0 is the identity -> bandwidth b.
    off, col = oracle.build_csr(*band_graph(n, b), n)
    P, _ = oracle.rcm(off, col)
    assert P.tolist() == list(range(n - 1, -1, -1))
    _, lab = oracle.permutation_arrays(P)
    assert oracle.bandwidth(off, col, lab) == b
    # randomly relabelled band: BFS levels from an end of the band are blocks
    # of b consecutive band positions, so RCM bandwidth <= 2b-1, whereas the
    # random labelling is far wider.
    rng = np.random.default_rng(n * 7 + b)
    for _ in range(5):
        sigma = rng.permutation(n).astype(np.int32)
        off, col = oracle.build_csr(*band_graph(n, b, sigma), n)
        P, _ = oracle.rcm(off, col)
        _, lab = oracle.permutation_arrays(P)
        assert oracle.bandwidth(off, col, lab) <= 2 * b - 1
        assert oracle.bandwidth(off, col, lab) <= oracle.bandwidth(off, col)


def test_rcm_star():
    # start at the smallest leaf, then the centre, then the other leaves.
    n = 9
    off, col = oracle.build_csr(*star_graph(n, 4), n)
    P, n_plus = oracle.rcm(off, col)
    cm = [0, 4, 1, 2, 3, 5, 6, 7, 8]
    assert P.tolist() == cm[::-1] and n_plus == n


@pytest.mark.parametrize("seed", range(8))
def test_rcm_invariants(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 300))
    src, dst = random_graph(rng, n, int(rng.integers(n // 2, 2 * n)))
    off, col = oracle.build_csr(src, dst, n)
    deg = np.diff(off)
    P, n_plus = oracle.rcm(off, col)
    # a permutation of 0..n-1
    assert sorted(P.tolist()) == list(range(n))
    # isolated vertices take labels >= n_plus in ascending ID order
    assert n_plus == int((deg > 0).sum())
    assert P[n_plus:].tolist() == [v for v in range(n) if deg[v] == 0]
    # every component occupies one contiguous label range; the component of
    # the first start (minimal (degree, id) over V+) occupies the top range
    _, lab = oracle.permutation_arrays(P)
    adj = adjacency_sets(src, dst, n)
    seen = np.zeros(n, bool)
    first = min((v for v in range(n) if deg[v] > 0), key=lambda v: (deg[v], v), default=None)
    for s in range(n):
        if seen[s] or deg[s] == 0:
            continue
        stack, comp = [s], []
        seen[s] = True
        while stack:
            v = stack.pop()
            comp.append(v)
            for w in adj[v]:
                if not seen[w]:
                    seen[w] = True
                    stack.append(w)
        labels = sorted(lab[comp].tolist())
        assert labels == list(range(labels[0], labels[0] + len(labels)))
        if first in comp:
            assert labels[-1] == n_plus - 1
    # the relabelled CSR is the same graph under the labelling
    off_r, col_r = oracle.permute_csr(off, col, P, n_plus)
    for i in range(n_plus):
        v = P[i]
        assert sorted(lab[col[off[v]:off[v + 1]]].tolist()) == col_r[off_r[i]:off_r[i + 1]].tolist()


def test_rcm_bandwidth_vs_scipy_sanity():
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp
    rng = np.random.default_rng(3)
    n, b = 200, 4
    sigma = rng.permutation(n).astype(np.int32)
    off, col = oracle.build_csr(*band_graph(n, b, sigma), n)
    P, _ = oracle.rcm(off, col)
    _, lab = oracle.permutation_arrays(P)
    A = sp.csr_matrix((np.ones(len(col)), col, off), shape=(n, n))
    perm = csgraph.reverse_cuthill_mckee(A, symmetric_mode=True)
    lab2 = np.empty(n, np.int32)
    lab2[perm] = np.arange(n, dtype=np.int32)
    # both orderings recover a narrow band from the scrambled labelling
    assert oracle.bandwidth(off, col, lab) <= 2 * b - 1
    assert oracle.bandwidth(off, col, lab2) <= 2 * b - 1
    assert oracle.bandwidth(off, col) > 10 * b


# ------------------------------------------------------------- partial RCM
def partial_rcm_by_level_sort(src, dst, n, p_permille):
    """The level-sort restatement above restricted to S, the last k vertices
    of V+ in (degree, id) order, k = ceil(p * |V+|): components and levels
    use only edges inside S (degrees stay the graph's). S's reversed order
    comes first, then the rest of V+ by id, then the isolated vertices."""
    adj = adjacency_sets(src, dst, n)
    deg = [len(a) for a in adj]
    vplus = sorted((v for v in range(n) if deg[v] > 0), key=lambda v: (deg[v], v))
    k = (len(vplus) * p_permille + 999) // 1000
    S = set(vplus[len(vplus) - k:])
    sadj = [set(w for w in adj[v] if w in S) if v in S else set() for v in range(n)]
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for u in S:
        for w in sadj[u]:
            ru, rw = find(u), find(w)
            if ru != rw:
                parent[ru] = rw
    comps = {}
    for v in S:
        comps.setdefault(find(v), []).append(v)
    starts = sorted((min(c, key=lambda v: (deg[v], v)) for c in comps.values()),
                    key=lambda v: (deg[v], v))
    order, pos = [], {}
    for s in starts:
        pos[s] = len(order)
        order.append(s)
        level = [s]
        while level:
            cand = {}
            for v in level:
                for w in sadj[v]:
                    if w not in pos:
                        cand[w] = min(cand.get(w, 1 << 60), pos[v])
            nxt = sorted(cand, key=lambda w: (cand[w], deg[w], w))
            for w in nxt:
                pos[w] = len(order)
                order.append(w)
            level = nxt
    rest = sorted(v for v in vplus if v not in S)
    return order[::-1] + rest + [v for v in range(n) if deg[v] == 0], len(vplus)


@pytest.mark.parametrize("block", range(5))
def test_partial_rcm_equals_level_sort_restatement(block):
    rng = np.random.default_rng(2000 + block)
    for _ in range(300):
        n = int(rng.integers(1, 15))
        m = int(rng.integers(0, 2 * n + 1))
        src, dst = random_graph(rng, n, m)
        pm = int(rng.choice([0, 1, 250, 333, 500, 750, 999, 1000]))
        off, col = oracle.build_csr(src, dst, n)
        P, n_plus = oracle.rcm_partial(off, col, pm)
        P2, n_plus2 = partial_rcm_by_level_sort(src, dst, n, pm)
        assert n_plus == n_plus2
        assert P.tolist() == P2, (src.tolist(), dst.tolist(), pm)


def test_partial_rcm_end_points_and_invariants():
    import graphgen
    src, dst = graphgen.kronecker_edges(10, 16, seed=3)
    n = 1 << 10
    off, col = oracle.build_csr(src, dst, n)
    deg = np.diff(off)
    P_full, n_plus = oracle.rcm(off, col)
    P, np2 = oracle.rcm_partial(off, col, 1000)  # p = 1: Algorithm 3 itself
    assert np2 == n_plus and np.array_equal(P, P_full)
    P0, _ = oracle.rcm_partial(off, col, 0)  # p = 0: nothing reordered
    assert np.array_equal(P0, np.concatenate([np.nonzero(deg > 0)[0], np.nonzero(deg == 0)[0]]))
    for pm in (100, 500):
        P, _ = oracle.rcm_partial(off, col, pm)
        k = (n_plus * pm + 999) // 1000
        assert sorted(P.tolist()) == list(range(n))
        vplus = sorted(np.nonzero(deg > 0)[0].tolist(), key=lambda v: (deg[v], v))
        assert set(P[:k].tolist()) == set(vplus[n_plus - k:])  # the top k come first
        assert P[k:n_plus].tolist() == sorted(vplus[:n_plus - k])
        assert P[n_plus:].tolist() == np.nonzero(deg == 0)[0].tolist()
