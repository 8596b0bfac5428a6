"""CPU oracle for the RCM-relabelled hybrid BFS -- TEST INFRASTRUCTURE ONLY.

Plain, slow, serial restatements of what the GPU path computes, used by the
tests, by ``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline leg
only. The product library never imports this package, and this package never
imports the product library: the two share nothing but the seeded input
generators (``graphgen``).

The arithmetic lives in ``oracle.c`` (serial C, compiled with plain gcc) and in
the pure-Python/numpy modules next to it:

* ``oracle.c``       CSR (Sec. 3.1, Eq. 2), RCM (Algorithm 3) and a
                     certificate check of it, partial RCM (Sec. 4.6),
                     relabelled CSR,
                     serial BFS (Algorithm 1), validator, bandwidth (Eq. 1),
                     bottom-up edges examined (Algorithm 2).
* ``direction.py``   the per-level top-down / bottom-up switching rule.
* ``mlp.py``         float64 forward/backward/training of the 12-32-4 MLP.
* ``metrics.py``     TEPS and its harmonic mean (Sec. 2.1, Graph500 TEPS).

Parity: every function here is pinned by ``tests/test_oracle_*.py`` against
brute force, closed forms, library routines or invariants (see the tests).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")

_lib = None
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def _p32(a):
    return a.ctypes.data_as(_i32p)


def _p64(a):
    return a.ctypes.data_as(_i64p)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _b
            _b.build()
        L = ctypes.CDLL(LIB_PATH)
        L.orc_build_csr.argtypes = [_i32p, _i32p, ctypes.c_int64, ctypes.c_int32, _i64p, _i32p]
        L.orc_build_csr.restype = ctypes.c_int64
        L.orc_rcm.argtypes = [_i64p, _i32p, ctypes.c_int32, _i32p]
        L.orc_rcm.restype = ctypes.c_int32
        L.orc_rcm_partial.argtypes = [_i64p, _i32p, ctypes.c_int32, ctypes.c_int32, _i32p]
        L.orc_rcm_partial.restype = ctypes.c_int32
        L.orc_rcm_check.argtypes = [_i64p, _i32p, ctypes.c_int32, _i32p, _i64p]
        L.orc_rcm_check.restype = ctypes.c_int32
        L.orc_permute_csr.argtypes = [_i64p, _i32p, ctypes.c_int32, _i32p, ctypes.c_int32,
                                      _i64p, _i32p]
        L.orc_permute_csr.restype = None
        L.orc_bfs.argtypes = [_i64p, _i32p, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p]
        L.orc_bfs.restype = None
        L.orc_validate.argtypes = [_i64p, _i32p, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                   _i64p]
        L.orc_validate.restype = ctypes.c_int32
        L.orc_validate_tree.argtypes = L.orc_validate.argtypes
        L.orc_validate_tree.restype = ctypes.c_int32
        L.orc_bandwidth.argtypes = [_i64p, _i32p, ctypes.c_int32, _i32p]
        L.orc_bandwidth.restype = ctypes.c_int64
        L.orc_bu_examined.argtypes = [_i64p, _i32p, ctypes.c_int32, _i32p, ctypes.c_int32,
                                      ctypes.c_int32]
        L.orc_bu_examined.restype = ctypes.c_int64
        _lib = L
    return _lib


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def build_csr(src, dst, n: int):
    """Cleaned undirected CSR (both directions, no self-loops, no duplicates,
    rows ascending) -> (off int64[n+1], col int32[nnz])."""
    src, dst = _c32(src), _c32(dst)
    m = len(src)
    off = np.empty(n + 1, np.int64)
    col = np.empty(max(2 * m, 1), np.int32)
    nnz = lib().orc_build_csr(_p32(src), _p32(dst), m, n, _p64(off), _p32(col))
    return off, col[:nnz].copy()


def rcm(off, col):
    """Algorithm 3 -> (P int32[n] position -> original ID, n_plus)."""
    off, col = _c64(off), _c32(col)
    n = len(off) - 1
    P = np.empty(max(n, 1), np.int32)
    n_plus = lib().orc_rcm(_p64(off), _p32(col), n, _p32(P))
    return P[:n].copy(), int(n_plus)


def rcm_partial(off, col, p_permille: int):
    """Partial RCM (Sec. 4.6, reading in oracle.c) -> (P, n_plus)."""
    off, col = _c64(off), _c32(col)
    n = len(off) - 1
    P = np.empty(max(n, 1), np.int32)
    n_plus = lib().orc_rcm_partial(_p64(off), _p32(col), n, int(p_permille), _p32(P))
    return P[:n].copy(), int(n_plus)


def rcm_check(off, col, P):
    """0 when P is Algorithm 3's permutation of the graph, checked through
    the conditions that make it unique (no re-run of Algorithm 3), else
    (rule number, offending Cuthill-McKee position); see oracle.c."""
    off, col, P = _c64(off), _c32(col), _c32(P)
    n = len(off) - 1
    if len(P) != n:
        return (1, -1)
    bad = np.zeros(1, np.int64)
    r = lib().orc_rcm_check(_p64(off), _p32(col), n, _p32(P), _p64(bad))
    return 0 if r == 0 else (int(r), int(bad[0]))


def permutation_arrays(P):
    """(old_of_new, new_of_old) from the RCM permutation P."""
    P = _c32(P)
    new_of_old = np.empty_like(P)
    new_of_old[P] = np.arange(len(P), dtype=np.int32)
    return P.copy(), new_of_old


def permute_csr(off, col, P, n_plus: int):
    """Relabelled CSR over the n_plus non-isolated vertices, rows ascending."""
    off, col, P = _c64(off), _c32(col), _c32(P)
    n = len(off) - 1
    nnz = int(off[-1])
    off_new = np.empty(n_plus + 1, np.int64)
    col_new = np.empty(max(nnz, 1), np.int32)
    lib().orc_permute_csr(_p64(off), _p32(col), n, _p32(P), n_plus, _p64(off_new), _p32(col_new))
    return off_new, col_new[:nnz].copy()


def bfs(off, col, root: int):
    """Serial BFS -> (parent int32[n], level int32[n]); -1 when unreachable."""
    off, col = _c64(off), _c32(col)
    n = len(off) - 1
    parent = np.empty(max(n, 1), np.int32)
    level = np.empty(max(n, 1), np.int32)
    lib().orc_bfs(_p64(off), _p32(col), n, int(root), _p32(parent), _p32(level))
    return parent[:n].copy(), level[:n].copy()


def validate(off, col, root: int, parent, level):
    """0 when (parent, level) is a valid BFS result for root, else
    (rule number, offending vertex); see oracle.c for the rules."""
    off, col, parent, level = _c64(off), _c32(col), _c32(parent), _c32(level)
    n = len(off) - 1
    bad = np.zeros(1, np.int64)
    r = lib().orc_validate(_p64(off), _p32(col), n, int(root), _p32(parent), _p32(level),
                           _p64(bad))
    return 0 if r == 0 else (int(r), int(bad[0]))


def validate_tree(off, col, root: int, parent, level):
    """Rules 1-4 of validate() (no pass over every edge): for a level[]
    already found equal to bfs()'s, where rule 5 holds by itself."""
    off, col, parent, level = _c64(off), _c32(col), _c32(parent), _c32(level)
    n = len(off) - 1
    bad = np.zeros(1, np.int64)
    r = lib().orc_validate_tree(_p64(off), _p32(col), n, int(root), _p32(parent),
                                _p32(level), _p64(bad))
    return 0 if r == 0 else (int(r), int(bad[0]))


def bandwidth(off, col, label=None) -> int:
    """Eq. 1 under label[v] (identity when None)."""
    off, col = _c64(off), _c32(col)
    n = len(off) - 1
    lp = None
    if label is not None:
        label = _c32(label)
        lp = _p32(label)
    return int(lib().orc_bandwidth(_p64(off), _p32(col), n, lp))


def bu_examined(off, col, level, L: int, reverse: bool = False) -> int:
    """Edges the bottom-up step from level L examines (CSR order, early break)."""
    off, col, level = _c64(off), _c32(col), _c32(level)
    n = len(off) - 1
    return int(lib().orc_bu_examined(_p64(off), _p32(col), n, _p32(level), int(L),
                                      1 if reverse else 0))


def pipeline(src, dst, n: int):
    """CSR -> RCM -> relabelled CSR, as the library's preprocessing does it.
    Returns dict(off, col, P, n_plus, new_of_old, off_r, col_r)."""
    off, col = build_csr(src, dst, n)
    P, n_plus = rcm(off, col)
    old_of_new, new_of_old = permutation_arrays(P)
    off_r, col_r = permute_csr(off, col, P, n_plus)
    return dict(off=off, col=col, P=P, n_plus=n_plus, old_of_new=old_of_new,
                new_of_old=new_of_old, off_r=off_r, col_r=col_r)
