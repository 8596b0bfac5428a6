"""Small test graphs built in plain Python (edge tuples), shared by tests."""
import numpy as np


def random_graph(rng, n, m, allow_loops=True):
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if not allow_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    return src, dst


def path_graph(n):
    s = np.arange(n - 1, dtype=np.int32)
    return s, s + 1


def cycle_graph(n):
    s = np.arange(n, dtype=np.int32)
    return s, (s + 1) % n


def star_graph(n, centre=0):
    leaves = np.array([v for v in range(n) if v != centre], np.int32)
    return np.full(len(leaves), centre, np.int32), leaves


def complete_graph(n):
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    a = np.array(pairs, np.int32).reshape(-1, 2)
    return a[:, 0].copy(), a[:, 1].copy()


def band_graph(n, b, relabel=None):
    pairs = [(i, j) for i in range(n) for j in range(i + 1, min(n, i + b + 1))]
    a = np.array(pairs, np.int32).reshape(-1, 2)
    s, d = a[:, 0].copy(), a[:, 1].copy()
    if relabel is not None:
        s, d = relabel[s], relabel[d]
    return s.astype(np.int32), d.astype(np.int32)


def adjacency_sets(src, dst, n):
    adj = [set() for _ in range(n)]
    for u, v in zip(src.tolist(), dst.tolist()):
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    return adj
