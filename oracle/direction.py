"""Per-level top-down / bottom-up switching rule -- TEST INFRASTRUCTURE ONLY.

Algorithm 2 starts top-down and, after every level, calls
update_traversal_policy(), which the paper does not spell out (Sec. 2.1 and
Sec. 3.6 point to Beamer et al. and to alpha/beta tuning). Reading used here
(Beamer's direction-optimizing rule), in exact integer arithmetic:

  * the expansion of level 0 (the root) is top-down;
  * after a top-down level, expand the next frontier bottom-up when
        m_f * alpha > m_u
    (m_f: sum of degrees of the frontier, m_u: sum of degrees of the vertices
    not yet visited);
  * after a bottom-up level, go back to top-down when the frontier shrank
    and n_f * beta < n (n_f: frontier size, n: vertices of the searched graph);
    otherwise stay bottom-up.

The direction changes time and the predecessor choice only, never level[].
"""
from __future__ import annotations

import numpy as np

TD, BU = 0, 1


def level_stats(off, level):
    """Per level L (frontier F_L = {v : level[v] == L}, L = 0 .. max):
    n_f, m_f, n_u, m_u where "unvisited" means level > L or -1."""
    off = np.asarray(off, np.int64)
    level = np.asarray(level, np.int64)
    deg = np.diff(off)
    lmax = int(level.max()) if len(level) else -1
    out = []
    for L in range(lmax + 1):
        f = level == L
        u = (level > L) | (level < 0)
        out.append(dict(n_f=int(f.sum()), m_f=int(deg[f].sum()), n_u=int(u.sum()),
                        m_u=int(deg[u].sum())))
    return out


def heuristic_directions(off, level, alpha: int = 14, beta: int = 24):
    """Direction used to expand each non-empty frontier F_0 .. F_max."""
    n = len(off) - 1
    st = level_stats(off, level)
    dirs = []
    prev_nf = 0
    for L, s in enumerate(st):
        if L == 0:
            d = TD
        elif dirs[-1] == TD:
            d = BU if s["m_f"] * alpha > s["m_u"] else TD
        else:
            d = TD if (s["n_f"] < prev_nf and s["n_f"] * beta < n) else BU
        dirs.append(d)
        prev_nf = s["n_f"]
    return dirs
