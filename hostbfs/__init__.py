"""Multithreaded hybrid BFS on the host cores -- the paper's own CPU design
(Algorithms 4-6, Sec. 3.3-3.5), kept as a CPU baseline beside the serial
oracle. Separate from the GPU library, which never calls it; see hostbfs.c
for what each step follows.

    ws = HostBFS(off_r, col_r, old_of_new, new_of_old, n, threads=15)
    parent, level, stats = ws.bfs(root)      # original IDs, -1 unreached
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhostbfs.so")
_lib = None
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


class hb_opts(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("lambda_", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("td_kind", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class hb_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("bu_levels", ctypes.c_int32),
                ("td_levels", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("bu_examined", ctypes.c_int64)]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _b
            _b.build()
        L = ctypes.CDLL(LIB_PATH)
        L.hb_ws_create.argtypes = [_i64p, _i32p, ctypes.c_int32, _i32p, _i32p, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32]
        L.hb_ws_create.restype = ctypes.c_void_p
        L.hb_ws_free.argtypes = [ctypes.c_void_p]
        L.hb_ws_free.restype = None
        L.hb_bfs.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(hb_opts), _i32p,
                             _i32p, ctypes.POINTER(hb_stats)]
        L.hb_bfs.restype = ctypes.c_int32
        L.hb_partitions.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p]
        L.hb_partitions.restype = None
        _lib = L
    return _lib


def partitions(blocks: int, nparts: int) -> np.ndarray:
    """Partition boundaries (in 64-byte blocks) of the bottom-up step."""
    b = np.zeros(nparts + 1, np.int64)
    lib().hb_partitions(int(blocks), int(nparts), b.ctypes.data_as(_i64p))
    return b


class HostBFS:
    """Workspace over an RCM-relabelled CSR (off int64[nb+1], col int32) with
    its permutation (old_of_new, new_of_old int32[n]; None for a graph in its
    own labelling). Keeps references to the arrays it borrows."""

    def __init__(self, off, col, old_of_new, new_of_old, n, threads=0, lam=20):
        self.off = np.ascontiguousarray(off, np.int64)
        self.col = np.ascontiguousarray(col, np.int32)
        self.o2n = None if old_of_new is None else np.ascontiguousarray(old_of_new, np.int32)
        self.n2o = None if new_of_old is None else np.ascontiguousarray(new_of_old, np.int32)
        self.n = int(n)
        nb = len(self.off) - 1
        p = lambda a: None if a is None else a.ctypes.data_as(_i32p)
        self.ws = lib().hb_ws_create(self.off.ctypes.data_as(_i64p), p(self.col), nb,
                                     p(self.o2n), p(self.n2o), self.n, int(lam), int(threads))
        if not self.ws:
            raise MemoryError("hb_ws_create")

    def bfs(self, root, alpha=14, beta=24, td_kind=0, parent=None, level=None):
        o = hb_opts(alpha=alpha, beta=beta, td_kind=td_kind)
        parent = np.empty(self.n, np.int32) if parent is None else parent
        level = np.empty(self.n, np.int32) if level is None else level
        st = hb_stats()
        r = lib().hb_bfs(self.ws, int(root), ctypes.byref(o), parent.ctypes.data_as(_i32p),
                         level.ctypes.data_as(_i32p), ctypes.byref(st))
        if r != 0:
            raise ValueError(f"hb_bfs: bad root {root}")
        return parent, level, {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if self.ws:
            lib().hb_ws_free(self.ws)
            self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
