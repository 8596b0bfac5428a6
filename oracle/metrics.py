"""TEPS arithmetic -- TEST INFRASTRUCTURE ONLY.

The paper reports Graph500 TEPS (Sec. 2.1) without defining the edge count;
its remark on superlinear scaling (Sec. 4.5) implies generated edges are
counted, duplicates included. Reading used: for root r, m_r is the number of
generated edge tuples (u, v) whose endpoint u is reached (level[u] >= 0), and
TEPS_r = m_r / t_r. Over k roots the harmonic mean is k / sum_r (t_r / m_r).
"""
from __future__ import annotations

import numpy as np


def edges_traversed(src, level_orig) -> int:
    """Generated tuples with a reached first endpoint (level in original IDs)."""
    level_orig = np.asarray(level_orig)
    return int(np.count_nonzero(level_orig[np.asarray(src)] >= 0))


def unique_edges_traversed(off, level) -> int:
    """Secondary count: undirected cleaned edges inside the reached set."""
    deg = np.diff(np.asarray(off, np.int64))
    return int(deg[np.asarray(level) >= 0].sum() // 2)


def harmonic_mean_teps(m, t) -> float:
    m = np.asarray(m, np.float64)
    t = np.asarray(t, np.float64)
    return float(len(m) / np.sum(t / m))
