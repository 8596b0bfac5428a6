"""Pins the oracle's RCM certificate check (orc_rcm_check), which certifies
Algorithm 3's permutation at sizes where running Algorithm 3 takes too long:

* brute force: on tiny random graphs, of all n! permutations exactly one
  passes, and it is the permutation of the independent level-sort
  restatement of Algorithm 3 (the check is a characterisation, not a
  restatement of orc_rcm);
* the permutations of Algorithm 3 pass on random multi-component graphs;
* every transposition of Algorithm 3's permutation fails, and each failure
  names the rule that a swapped pair breaks."""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from _graphs import random_graph
from test_oracle_rcm import rcm_by_level_sort


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_exactly_one_permutation_passes(n):
    rng = np.random.default_rng(40 + n)
    reps = {3: 40, 4: 40, 5: 25, 6: 8}[n]
    for _ in range(reps):
        m = int(rng.integers(0, 2 * n + 1))
        src, dst = random_graph(rng, n, m)
        off, col = oracle.build_csr(src, dst, n)
        passing = [p for p in itertools.permutations(range(n))
                   if oracle.rcm_check(off, col, np.array(p, np.int32)) == 0]
        want, _ = rcm_by_level_sort(src, dst, n)
        assert passing == [tuple(want)]


def test_seven_vertex_graphs_brute_force():
    rng = np.random.default_rng(77)
    for _ in range(2):
        src, dst = random_graph(rng, 7, 9)
        off, col = oracle.build_csr(src, dst, 7)
        passing = [p for p in itertools.permutations(range(7))
                   if oracle.rcm_check(off, col, np.array(p, np.int32)) == 0]
        want, _ = rcm_by_level_sort(src, dst, 7)
        assert passing == [tuple(want)]


@pytest.mark.parametrize("seed", range(6))
def test_algorithm3_passes(seed):
    rng = np.random.default_rng(500 + seed)
    for _ in range(60):
        n = int(rng.integers(1, 120))
        src, dst = random_graph(rng, n, int(rng.integers(0, 2 * n + 1)))
        off, col = oracle.build_csr(src, dst, n)
        P, _ = oracle.rcm(off, col)
        assert oracle.rcm_check(off, col, P) == 0


def test_kronecker_passes_and_transpositions_fail():
    n = 1 << 8
    src, dst = graphgen.kronecker_edges(8, 16, seed=9)
    off, col = oracle.build_csr(src, dst, n)
    P, n_plus = oracle.rcm(off, col)
    assert oracle.rcm_check(off, col, P) == 0
    rng = np.random.default_rng(1)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, n, (3000, 2)) if a != b]
    for a, b in pairs:
        Q = P.copy()
        Q[[a, b]] = Q[[b, a]]
        r = oracle.rcm_check(off, col, Q)
        assert r != 0, (a, b)
        # isolated and non-isolated swapped, or two isolated out of order:
        # rule 1; two vertices of V+ swapped: the ordering rules 2/3
        if (a >= n_plus) or (b >= n_plus):
            assert r[0] == 1
        else:
            assert r[0] in (2, 3)


def test_wrong_length_and_repeats_fail():
    src, dst = graphgen.kronecker_edges(6, 16, seed=2)
    off, col = oracle.build_csr(src, dst, 64)
    P, _ = oracle.rcm(off, col)
    assert oracle.rcm_check(off, col, P[:-1]) != 0
    Q = P.copy()
    Q[5] = Q[6]
    assert oracle.rcm_check(off, col, Q)[0] == 1
