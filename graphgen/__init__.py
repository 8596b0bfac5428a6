"""Seeded synthetic inputs for the BFS/RCM library and its oracle.

A module of its own: it holds generators only, none of the method's
arithmetic, and is the one piece of code both sides use. The host generator
(C + OpenMP, ``gg_host.c``) and its CUDA twin (``gg_dev.cu``) compile the same
integer definitions from ``gg_common.h`` and produce identical bytes.

Workloads (stand-ins for the paper's Graph500 inputs, Sec. 4.2):

* Kronecker / R-MAT: ``2^scale`` vertices, ``edgefactor * 2^scale`` edge
  tuples, initiator (A, B, C, D) = (0.57, 0.19, 0.19, 0.05), one 32-bit draw per
  bit level, no per-level noise, then a seeded bijective relabelling of the
  vertex IDs. Self-loops and duplicate tuples are kept (the CSR builder drops
  them), as in the paper's description of its inputs.
* Chung-Lu power law: weights ``w_i = c (i+1)^(-1/(gamma-1))`` capped at
  ``cap``, ``c`` fixed by bisection so the mean weight is ``mean_degree``;
  ``n * mean_degree / 2`` tuples with both endpoints drawn proportional to
  ``w`` through an integer cumulative table; then relabelled.
"""
from __future__ import annotations

import ctypes
import os
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
HOST_LIB = os.path.join(_BUILD, "libgg_host.so")
DEV_LIB = os.path.join(_BUILD, "libgg_dev.so")

KRON_INITIATOR = ("0.57", "0.19", "0.19", "0.05")

_host = None
_dev = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def _ptr(a, t):
    return a.ctypes.data_as(t)


def host_lib():
    global _host
    if _host is None:
        if not os.path.exists(HOST_LIB):
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(HOST_LIB)
        lib.gg_kron.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _i32p, _i32p]
        lib.gg_kron.restype = None
        lib.gg_chunglu.argtypes = [ctypes.c_uint64, ctypes.c_int64, _u64p, ctypes.c_int64,
                                   ctypes.c_int64, _i32p, _i32p]
        lib.gg_chunglu.restype = None
        lib.gg_mark_nonisolated.argtypes = [_i32p, _i32p, ctypes.c_int64, ctypes.c_int32, _u8p]
        lib.gg_mark_nonisolated.restype = None
        lib.gg_pick_roots.argtypes = [_u8p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _i32p]
        lib.gg_pick_roots.restype = ctypes.c_int32
        lib.gg_perm_value.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
        lib.gg_perm_value.restype = ctypes.c_int64
        lib.gg_draw_value.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_draw_value.restype = ctypes.c_uint64
        _host = lib
    return _host


def dev_lib():
    global _dev
    if _dev is None:
        if not os.path.exists(DEV_LIB):
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(DEV_LIB)
        vp = ctypes.c_void_p
        lib.gg_kron_dev.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, vp, vp, vp]
        lib.gg_chunglu_dev.argtypes = [ctypes.c_uint64, ctypes.c_int64, vp, ctypes.c_int64,
                                       ctypes.c_int64, vp, vp, vp]
        lib.gg_mark_nonisolated_dev.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
        for f in (lib.gg_kron_dev, lib.gg_chunglu_dev, lib.gg_mark_nonisolated_dev):
            f.restype = ctypes.c_int
        _dev = lib
    return _dev


def kron_thresholds(initiator=KRON_INITIATOR):
    """Cumulative initiator probabilities as 32-bit integer thresholds."""
    a, b, c, _ = (Fraction(x) for x in initiator)
    scale = 1 << 32
    return (int(a * scale), int((a + b) * scale), int((a + b + c) * scale))


def kronecker_edges(scale: int, edgefactor: int = 16, seed: int = 1, e0: int = 0,
                    count: int | None = None):
    """Host generation of Kronecker edge tuples [e0, e0+count) -> (src, dst) int32."""
    m = edgefactor << scale
    if count is None:
        count = m - e0
    src = np.empty(count, np.int32)
    dst = np.empty(count, np.int32)
    tA, tAB, tABC = kron_thresholds()
    host_lib().gg_kron(seed, scale, e0, count, tA, tAB, tABC, _ptr(src, _i32p), _ptr(dst, _i32p))
    return src, dst


def kronecker_edges_dev(scale: int, edgefactor: int = 16, seed: int = 1, device="cuda"):
    """CUDA-twin generation of all Kronecker tuples -> (src, dst) int32 device tensors."""
    import torch
    m = edgefactor << scale
    src = torch.empty(m, dtype=torch.int32, device=device)
    dst = torch.empty(m, dtype=torch.int32, device=device)
    tA, tAB, tABC = kron_thresholds()
    st = torch.cuda.current_stream(src.device).cuda_stream
    rc = dev_lib().gg_kron_dev(seed, scale, 0, m, tA, tAB, tABC, src.data_ptr(), dst.data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"gg_kron_dev failed: cuda error {rc}")
    return src, dst


def chunglu_weights(n: int, gamma: float = 2.1, mean_degree: float = 20.0,
                    cap: float = 2.0 ** 16):
    """Expected degrees w_i = c (i+1)^(-1/(gamma-1)), capped; c set by bisection."""
    base = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (gamma - 1.0))
    lo, hi = 0.0, float(cap) * 4.0
    for _ in range(200):
        c = 0.5 * (lo + hi)
        if np.minimum(c * base, cap).mean() < mean_degree:
            lo = c
        else:
            hi = c
    return np.minimum(0.5 * (lo + hi) * base, cap)


def chunglu_table(n: int, gamma: float = 2.1, mean_degree: float = 20.0,
                  cap: float = 2.0 ** 16):
    """Integer cumulative table: cum[i] ~ 2^64 * sum_{j<=i} w_j / sum w."""
    w = chunglu_weights(n, gamma, mean_degree, cap)
    frac = np.cumsum(w) / w.sum()
    cum = np.floor(np.minimum(frac, 1.0) * 2.0 ** 63).astype(np.uint64) * np.uint64(2)
    cum[-1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    return cum


def chunglu_num_edges(n: int, mean_degree: float = 20.0) -> int:
    return int(n * mean_degree) // 2


def chunglu_edges(n: int, seed: int = 3, mean_degree: float = 20.0, gamma: float = 2.1,
                  cap: float = 2.0 ** 16, e0: int = 0, count: int | None = None):
    cum = chunglu_table(n, gamma, mean_degree, cap)
    m = chunglu_num_edges(n, mean_degree)
    if count is None:
        count = m - e0
    src = np.empty(count, np.int32)
    dst = np.empty(count, np.int32)
    host_lib().gg_chunglu(seed, n, _ptr(cum, _u64p), e0, count, _ptr(src, _i32p), _ptr(dst, _i32p))
    return src, dst


def chunglu_edges_dev(n: int, seed: int = 3, mean_degree: float = 20.0, gamma: float = 2.1,
                      cap: float = 2.0 ** 16, device="cuda"):
    import torch
    cum = torch.from_numpy(chunglu_table(n, gamma, mean_degree, cap).view(np.int64)).to(device)
    m = chunglu_num_edges(n, mean_degree)
    src = torch.empty(m, dtype=torch.int32, device=device)
    dst = torch.empty(m, dtype=torch.int32, device=device)
    st = torch.cuda.current_stream(src.device).cuda_stream
    rc = dev_lib().gg_chunglu_dev(seed, n, cum.data_ptr(), 0, m, src.data_ptr(), dst.data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"gg_chunglu_dev failed: cuda error {rc}")
    return src, dst


def nonisolated_flags(src: np.ndarray, dst: np.ndarray, n: int) -> np.ndarray:
    flags = np.empty(n, np.uint8)
    host_lib().gg_mark_nonisolated(_ptr(src, _i32p), _ptr(dst, _i32p), len(src), n,
                                   _ptr(flags, _u8p))
    return flags


def nonisolated_flags_dev(src, dst, n: int):
    import torch
    flags = torch.zeros(n, dtype=torch.uint8, device=src.device)
    st = torch.cuda.current_stream(src.device).cuda_stream
    rc = dev_lib().gg_mark_nonisolated_dev(src.data_ptr(), dst.data_ptr(), src.numel(),
                                           flags.data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"gg_mark_nonisolated_dev failed: cuda error {rc}")
    return flags


def pick_roots(flags: np.ndarray, k: int = 64, seed: int = 2) -> np.ndarray:
    """Up to k distinct roots drawn uniformly among non-isolated vertices."""
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    out = np.empty(k, np.int32)
    got = host_lib().gg_pick_roots(_ptr(flags, _u8p), len(flags), k, seed, _ptr(out, _i32p))
    return out[:got].copy()


def perm_value(seed: int, n: int, x: int) -> int:
    return int(host_lib().gg_perm_value(seed, n, x))


def draw_value(seed: int, purpose: int, ctr: int) -> int:
    return int(host_lib().gg_draw_value(seed, purpose, ctr))


def small_graph_specs(count: int = 4096, seed: int = 5, smin: int = 8, smax: int = 14):
    """Per-graph (scale, seed) of a batch of small Kronecker graphs: scale drawn
    uniformly from [smin, smax]; graph g uses seed * 2^20 + g."""
    span = smax - smin + 1
    specs = []
    for g in range(count):
        s = smin + draw_value(seed, 4, g) % span
        specs.append((s, seed * (1 << 20) + g))
    return specs
