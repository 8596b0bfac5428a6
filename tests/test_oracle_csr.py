"""Pins the oracle CSR (Sec. 3.1, Eq. 2) to a set-of-pairs construction."""
import numpy as np
import pytest

import oracle
from _graphs import adjacency_sets, random_graph


@pytest.mark.parametrize("seed", range(20))
def test_csr_matches_set_of_pairs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    m = int(rng.integers(0, 4 * n))
    src, dst = random_graph(rng, n, m)
    off, col = oracle.build_csr(src, dst, n)
    adj = adjacency_sets(src, dst, n)
    assert off[0] == 0 and len(off) == n + 1
    for v in range(n):
        row = col[off[v]:off[v + 1]].tolist()
        assert row == sorted(adj[v]), v
    assert off[-1] == sum(len(a) for a in adj)


def test_csr_empty_and_loops_only():
    off, col = oracle.build_csr(np.zeros(0, np.int32), np.zeros(0, np.int32), 5)
    assert off.tolist() == [0] * 6 and len(col) == 0
    s = np.array([1, 2, 2], np.int32)
    off, col = oracle.build_csr(s, s, 4)
    assert off.tolist() == [0] * 5 and len(col) == 0


def test_csr_kronecker_scale10_against_numpy_unique():
    import graphgen
    src, dst = graphgen.kronecker_edges(10, 16, seed=7)
    n = 1 << 10
    off, col = oracle.build_csr(src, dst, n)
    s = np.concatenate([src, dst]).astype(np.int64)
    d = np.concatenate([dst, src]).astype(np.int64)
    keep = s != d
    keys = np.unique(s[keep] * n + d[keep])
    assert np.array_equal(col, (keys % n).astype(np.int32))
    assert np.array_equal(np.diff(off), np.bincount(keys // n, minlength=n))
