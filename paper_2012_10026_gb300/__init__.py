"""Python binding of libg3bfs (the C ABI declared in include/g3bfs.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. Tensors are passed as raw pointers (``tensor.data_ptr()``) together
with the current CUDA stream; PyTorch only provides device memory and
streams. There is no CPU fallback: if the shared library cannot be loaded the
import of ``lib()`` raises.

The module-level functions carry the C names (``g3_build_csr``,
``g3_rcm_relabel``, ``g3_bfs`` ...). ``Graph`` is a small owner object around
a ``g3_graph*``.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libg3bfs.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "g3bfs.h")

G3_OK, G3_EINVAL, G3_ENOMEM, G3_ECUDA, G3_ETIMEOUT, G3_ERANGE, G3_ESTATE = range(7)
G3_CTRL_HEURISTIC, G3_CTRL_LEARNED, G3_CTRL_TOPDOWN, G3_CTRL_BOTTOMUP = range(4)
G3_DIR_TD, G3_DIR_BU = 0, 1
MLP_NPARAMS = 32 * 12 + 32 + 4 * 32 + 4


class G3Error(RuntimeError):
    def __init__(self, status, where, detail):
        super().__init__(f"{where}: {detail} (status {status})")
        self.status = status


class g3_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_bfs", ctypes.c_int32), ("n_plus", ctypes.c_int32),
                ("relabelled", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("max_degree", ctypes.c_int64)]


class g3_bfs_opts(ctypes.Structure):
    _fields_ = [("controller", ctypes.c_int32), ("alpha", ctypes.c_int32),
                ("beta", ctypes.c_int32), ("t1", ctypes.c_int32), ("t2", ctypes.c_int32),
                ("t3", ctypes.c_int32), ("bu_reverse", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("mlp_params", ctypes.c_void_p),
                ("record_both", ctypes.c_int32), ("mlp_margin", ctypes.c_int32),
                ("mlp_bins", ctypes.c_int32), ("out_split", ctypes.c_int32),
                ("bu_kernel", ctypes.c_int32), ("stats_counts_only", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class g3_level_stats(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("dir", ctypes.c_int32), ("n_f", ctypes.c_int64),
                ("m_f", ctypes.c_int64), ("n_u", ctypes.c_int64), ("m_u", ctypes.c_int64),
                ("examined", ctypes.c_int64), ("n_next", ctypes.c_int64),
                ("id_min", ctypes.c_int32), ("id_max", ctypes.c_int32),
                ("hist", ctypes.c_int64 * 4), ("t1", ctypes.c_int32), ("t2", ctypes.c_int32),
                ("t3", ctypes.c_int32), ("ms", ctypes.c_float), ("ms_expand", ctypes.c_float),
                ("t_td_ms", ctypes.c_float), ("t_bu_ms", ctypes.c_float),
                ("best_t1", ctypes.c_int32), ("best_t2", ctypes.c_int32),
                ("best_t3", ctypes.c_int32), ("mlp_out", ctypes.c_float * 4)]

    def to_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["hist"] = list(self.hist)
        d["mlp_out"] = list(self.mlp_out)
        return d


class g3_msbfs_opts(ctypes.Structure):
    _fields_ = [("push_alpha", ctypes.c_int32), ("pull_warp_deg", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


class g3_msbfs_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("pull_levels", ctypes.c_int32),
                ("push_levels", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("pull_entries", ctypes.c_int64), ("pull_vertices", ctypes.c_int64),
                ("push_entries", ctypes.c_int64)]


class g3_batch_opts(ctypes.Structure):
    _fields_ = [("warp_max_n", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


class g3_tune_entry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("size_class", ctypes.c_int32),
                ("deg_class", ctypes.c_int32), ("p", ctypes.c_int32 * 6),
                ("points", ctypes.c_int32), ("ms", ctypes.c_float),
                ("ms_default", ctypes.c_float)]

    def to_dict(self):
        return {"kind": self.kind, "size_class": self.size_class, "deg_class": self.deg_class,
                "p": list(self.p), "points": self.points, "ms": self.ms,
                "ms_default": self.ms_default}


G3_TUNE_BFS, G3_TUNE_MSBFS, G3_TUNE_BATCH = 1, 2, 3

_lib = None
_vp = ctypes.c_void_p

# name -> (restype, argtypes)
_SIGS = {
    "g3_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "g3_last_error_detail": (ctypes.c_char_p, []),
    "g3_version": (ctypes.c_char_p, []),
    "g3_kernel_launches": (ctypes.c_uint64, []),
    "g3_build_csr": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32, _vp,
                                    ctypes.POINTER(_vp)]),
    "g3_rcm_relabel": (ctypes.c_int, [_vp, _vp]),
    "g3_rcm_relabel_partial": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "g3_graph_info_get": (ctypes.c_int, [_vp, ctypes.POINTER(g3_graph_info)]),
    "g3_get_perm": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "g3_get_csr": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "g3_graph_free": (None, [_vp]),
    "g3_bfs_opts_default": (None, [ctypes.POINTER(g3_bfs_opts)]),
    "g3_bfs": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(g3_bfs_opts), _vp, _vp,
                              ctypes.POINTER(g3_level_stats), ctypes.c_int32,
                              ctypes.POINTER(ctypes.c_int32), _vp]),
    "g3_bfs_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                      _vp]),
    "g3_msbfs_opts_default": (None, [ctypes.POINTER(g3_msbfs_opts)]),
    "g3_msbfs": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                ctypes.POINTER(g3_msbfs_opts), _vp,
                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
                                _vp]),
    "g3_msbfs_last_stats": (ctypes.c_int, [_vp, ctypes.POINTER(g3_msbfs_stats)]),
    "g3_batch_opts_default": (None, [ctypes.POINTER(g3_batch_opts)]),
    "g3_batch_pack": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, _vp,
                                     ctypes.POINTER(_vp)]),
    "g3_batch_info_get": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int64)]),
    "g3_bfs_batch": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(g3_batch_opts), _vp, _vp,
                                    ctypes.POINTER(ctypes.c_float), _vp]),
    "g3_batch_free": (None, [_vp]),
    "g3_tune_key": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32)]),
    "g3_tune_cache_lookup": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.POINTER(g3_tune_entry),
                                            ctypes.POINTER(ctypes.c_int32)]),
    "g3_tune_cache_store": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(g3_tune_entry)]),
    "g3_autotune_bfs": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp, ctypes.c_char_p,
                                       ctypes.POINTER(g3_bfs_opts),
                                       ctypes.POINTER(g3_tune_entry), _vp]),
    "g3_autotune_msbfs": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, ctypes.c_char_p,
                                         ctypes.POINTER(g3_msbfs_opts),
                                         ctypes.POINTER(g3_tune_entry), _vp]),
    "g3_autotune_batch": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_char_p,
                                         ctypes.POINTER(g3_batch_opts),
                                         ctypes.POINTER(g3_tune_entry), _vp]),
    "g3_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp]),
    "g3_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp]),
    "g3_mlp_train": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_float, _vp, _vp]),
    "g3_mlp_features": (ctypes.c_int, [ctypes.POINTER(g3_level_stats), ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int64, _vp, _vp]),
    "g3_debug_inject": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64]),
    "g3_debug_pool_used": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
}
NOALLOC_MAX_N = 1 << 20
G3_INJECT_ALLOC, G3_INJECT_RCM_ROUNDS, G3_INJECT_STAGED_STALL = 1, 2, 3


def lib():
    """Loads the in-tree libg3bfs.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libg3bfs.so not built ({LIB_PATH}); run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    """Function names declared in include/g3bfs.h."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(g3_[a-z0-9_]+)\s*\(", txt)) - {"g3_graph"})


def kernel_launches() -> int:
    """Kernels this library has launched so far (graph nodes included)."""
    return int(lib().g3_kernel_launches())


def _check(st, where):
    if st != G3_OK:
        L = lib()
        raise G3Error(st, where, L.g3_last_error_detail().decode() or
                      L.g3_status_str(st).decode())


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def opts(**kw) -> g3_bfs_opts:
    o = g3_bfs_opts()
    lib().g3_bfs_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "mlp_params":
            v = ctypes.c_void_p(v.data_ptr() if hasattr(v, "data_ptr") else v)
        setattr(o, k, v)
    return o


# ------------------------------------------------------------- C-named calls
def g3_build_csr(src, dst, n: int, stream=None) -> "Graph":
    """Cleaned CSR of the undirected graph of int32 device tuples (src, dst)."""
    assert src.is_cuda and dst.is_cuda and src.numel() == dst.numel()
    g = ctypes.c_void_p()
    _check(lib().g3_build_csr(_ptr(src), _ptr(dst), src.numel(), int(n), _stream(stream),
                              ctypes.byref(g)), "g3_build_csr")
    return Graph(g)


def g3_rcm_relabel(graph: "Graph", stream=None):
    _check(lib().g3_rcm_relabel(graph.handle, _stream(stream)), "g3_rcm_relabel")


def g3_rcm_relabel_partial(graph: "Graph", p_permille: int, stream=None):
    """Partial RCM: only the top p_permille / 1000 of V+ reordered (Sec. 4.6)."""
    _check(lib().g3_rcm_relabel_partial(graph.handle, int(p_permille), _stream(stream)),
           "g3_rcm_relabel_partial")


def g3_graph_info_get(graph: "Graph") -> dict:
    info = g3_graph_info()
    _check(lib().g3_graph_info_get(graph.handle, ctypes.byref(info)), "g3_graph_info_get")
    return {k: getattr(info, k) for k, _ in info._fields_}


def g3_get_perm(graph: "Graph", old_of_new=None, new_of_old=None, stream=None):
    _check(lib().g3_get_perm(graph.handle, _ptr(old_of_new) if old_of_new is not None else None,
                             _ptr(new_of_old) if new_of_old is not None else None,
                             _stream(stream)), "g3_get_perm")


def g3_get_csr(graph: "Graph", off=None, col=None, stream=None):
    _check(lib().g3_get_csr(graph.handle, _ptr(off) if off is not None else None,
                            _ptr(col) if col is not None else None, _stream(stream)),
           "g3_get_csr")


def g3_bfs(graph: "Graph", root: int, parent, level, options: g3_bfs_opts | None = None,
           max_stats: int = 0, stream=None):
    """BFS from root (original ID) into parent/level (int32, n entries, device
    tensors or host tensors/arrays). Returns the list of per-level stats."""
    stats = (g3_level_stats * max_stats)() if max_stats > 0 else None
    nlev = ctypes.c_int32(0)

    def addr(x):
        if hasattr(x, "data_ptr"):
            return ctypes.c_void_p(x.data_ptr())
        return ctypes.c_void_p(x.ctypes.data)

    _check(lib().g3_bfs(graph.handle, int(root),
                        ctypes.byref(options) if options is not None else None,
                        addr(parent), addr(level), stats, max_stats, ctypes.byref(nlev),
                        _stream(stream)), "g3_bfs")
    if stats is None:
        return []
    return [stats[i].to_dict() for i in range(min(nlev.value, max_stats))]


def g3_debug_inject(kind: int, value: int):
    """Test hook: fail the value-th device allocation from now (G3_INJECT_ALLOC)
    or cap the RCM hooking rounds (G3_INJECT_RCM_ROUNDS); value <= 0 resets."""
    _check(lib().g3_debug_inject(int(kind), int(value)), "g3_debug_inject")


def g3_debug_pool_used() -> int:
    """Bytes in use from the current device's default memory pool."""
    v = ctypes.c_int64()
    _check(lib().g3_debug_pool_used(ctypes.byref(v)), "g3_debug_pool_used")
    return int(v.value)


def g3_bfs_noalloc(off, col, n: int, root: int, parent, level, stream=None):
    """Top-down BFS over a caller-provided device CSR that allocates nothing
    (scratch in a fixed static device array; n <= NOALLOC_MAX_N). For callers
    that cannot allocate device memory while they search. Calls sharing a
    device must not overlap on the GPU."""
    _check(lib().g3_bfs_noalloc(_ptr(off), _ptr(col), int(n), int(root), _ptr(parent),
                                _ptr(level), _stream(stream)), "g3_bfs_noalloc")


def msbfs_opts(**kw) -> g3_msbfs_opts:
    o = g3_msbfs_opts()
    lib().g3_msbfs_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def g3_msbfs(graph: "Graph", roots, level, options: g3_msbfs_opts | None = None, stream=None):
    """Bit-sliced BFS from up to 64 roots (original IDs) into level, a k x n
    int8 device tensor. Returns (levels run, device ms)."""
    roots = [int(r) for r in roots]
    arr = (ctypes.c_int32 * len(roots))(*roots)
    nl = ctypes.c_int32(0)
    ms = ctypes.c_float(0.0)
    _check(lib().g3_msbfs(graph.handle, arr, len(roots),
                          ctypes.byref(options) if options is not None else None,
                          _ptr(level), ctypes.byref(nl), ctypes.byref(ms), _stream(stream)),
           "g3_msbfs")
    return nl.value, ms.value


def g3_msbfs_last_stats(graph: "Graph") -> dict:
    """Work counts of the last g3_msbfs call on the graph."""
    st = g3_msbfs_stats()
    _check(lib().g3_msbfs_last_stats(graph.handle, ctypes.byref(st)), "g3_msbfs_last_stats")
    return {k: getattr(st, k) for k, _ in st._fields_ if k != "reserved"}


class Batch:
    """Owner of a g3_batch* (many small relabelled graphs packed together)."""

    def __init__(self, handle):
        self.handle = handle

    def free(self):
        if self.handle and self.handle.value:
            import torch
            torch.cuda.synchronize()
            lib().g3_batch_free(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            if self.handle and self.handle.value:
                lib().g3_batch_free(self.handle)
        except Exception:
            pass

    @property
    def info(self):
        G = ctypes.c_int32()
        N = ctypes.c_int64()
        E = ctypes.c_int64()
        _check(lib().g3_batch_info_get(self.handle, ctypes.byref(G), ctypes.byref(N),
                                       ctypes.byref(E)), "g3_batch_info_get")
        return {"G": G.value, "N": N.value, "nnz": E.value}


def batch_opts(**kw) -> g3_batch_opts:
    o = g3_batch_opts()
    lib().g3_batch_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def g3_batch_pack(graphs, stream=None) -> Batch:
    arr = (_vp * len(graphs))(*[g.handle.value for g in graphs])
    b = ctypes.c_void_p()
    _check(lib().g3_batch_pack(arr, len(graphs), _stream(stream), ctypes.byref(b)),
           "g3_batch_pack")
    return Batch(b)


def g3_bfs_batch(batch: Batch, roots, parent, level, options: g3_batch_opts | None = None,
                 timed: bool = True, stream=None):
    """One BFS per packed graph; returns the device ms of the launch (timed)."""
    ms = ctypes.c_float(0.0)
    _check(lib().g3_bfs_batch(batch.handle, _ptr(roots),
                              ctypes.byref(options) if options is not None else None,
                              _ptr(parent), _ptr(level), ctypes.byref(ms) if timed else None,
                              _stream(stream)), "g3_bfs_batch")
    return ms.value


def _path(p):
    return None if p is None else os.fsencode(p)


def tune_key(kind: int, vertices: int, nnz: int, graphs: int = 1):
    sc, dc = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().g3_tune_key(kind, vertices, nnz, graphs, ctypes.byref(sc), ctypes.byref(dc)),
           "g3_tune_key")
    return sc.value, dc.value


def tune_cache_lookup(path, kind: int, size_class: int, deg_class: int):
    """The cached g3_tune_entry for the key, or None."""
    e = g3_tune_entry()
    found = ctypes.c_int32()
    _check(lib().g3_tune_cache_lookup(_path(path), kind, size_class, deg_class, ctypes.byref(e),
                                      ctypes.byref(found)), "g3_tune_cache_lookup")
    return e if found.value else None


def tune_cache_store(path, entry: g3_tune_entry):
    _check(lib().g3_tune_cache_store(_path(path), ctypes.byref(entry)), "g3_tune_cache_store")


def autotune_bfs(graph: "Graph", roots, parent, level, cache_path=None,
                 start: g3_bfs_opts | None = None, stream=None):
    """Returns (tuned g3_bfs_opts, g3_tune_entry)."""
    roots = [int(r) for r in roots]
    arr = (ctypes.c_int32 * len(roots))(*roots)
    o = start if start is not None else opts()
    rec = g3_tune_entry()
    _check(lib().g3_autotune_bfs(graph.handle, arr, len(roots), _ptr(parent), _ptr(level),
                                 _path(cache_path), ctypes.byref(o), ctypes.byref(rec),
                                 _stream(stream)), "g3_autotune_bfs")
    return o, rec


def autotune_msbfs(graph: "Graph", roots, level, cache_path=None,
                   start: g3_msbfs_opts | None = None, stream=None):
    roots = [int(r) for r in roots]
    arr = (ctypes.c_int32 * len(roots))(*roots)
    o = start if start is not None else msbfs_opts()
    rec = g3_tune_entry()
    _check(lib().g3_autotune_msbfs(graph.handle, arr, len(roots), _ptr(level),
                                   _path(cache_path), ctypes.byref(o), ctypes.byref(rec),
                                   _stream(stream)), "g3_autotune_msbfs")
    return o, rec


def autotune_batch(batch: Batch, roots, parent, level, cache_path=None,
                   start: g3_batch_opts | None = None, stream=None):
    o = start if start is not None else batch_opts()
    rec = g3_tune_entry()
    _check(lib().g3_autotune_batch(batch.handle, _ptr(roots), _ptr(parent), _ptr(level),
                                   _path(cache_path), ctypes.byref(o), ctypes.byref(rec),
                                   _stream(stream)), "g3_autotune_batch")
    return o, rec


def _optr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def g3_mlp_forward(params, x, stream=None):
    """MLP outputs (B x 4, float32 device tensor) for feature rows x (B x 12)."""
    import torch
    out = torch.empty((x.shape[0], 4), dtype=torch.float32, device=x.device)
    _check(lib().g3_mlp_forward(_ptr(params), _ptr(x), x.shape[0], _ptr(out), _stream(stream)),
           "g3_mlp_forward")
    return out


def g3_mlp_loss_grad(params, x, y, w=None, stream=None):
    import torch
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    grad = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=x.device)
    _check(lib().g3_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(y), _optr(w), x.shape[0],
                                  _ptr(loss), _ptr(grad), _stream(stream)), "g3_mlp_loss_grad")
    return loss, grad


def g3_mlp_train(params, x, y, steps: int, lr: float = 1e-2, w=None, stream=None):
    """Full-batch Adam on the GPU, params updated in place; returns the losses."""
    import torch
    losses = torch.empty(max(steps, 1), dtype=torch.float32, device=x.device)
    _check(lib().g3_mlp_train(_ptr(params), _ptr(x), _ptr(y), _optr(w), x.shape[0], int(steps),
                              float(lr), _ptr(losses), _stream(stream)), "g3_mlp_train")
    return losses[:steps]


def g3_mlp_features(stats, n_bfs: int, nnz: int, device="cuda", stream=None):
    """Feature rows (len(stats) x 12) of level records (dicts from g3_bfs) of a
    search on a graph of n_bfs vertices and nnz directed entries."""
    import torch
    arr = (g3_level_stats * max(len(stats), 1))()
    for i, d in enumerate(stats):
        for k, _ in g3_level_stats._fields_:
            v = d[k]
            if k in ("hist", "mlp_out"):
                for j, e in enumerate(v):
                    getattr(arr[i], k)[j] = e
            else:
                setattr(arr[i], k, v)
    x = torch.empty((max(len(stats), 1), 12), dtype=torch.float32, device=device)
    _check(lib().g3_mlp_features(arr, len(stats), int(n_bfs), int(nnz), _ptr(x),
                                 _stream(stream)),
           "g3_mlp_features")
    return x[:len(stats)]


def g3_graph_free(graph: "Graph"):
    graph.free()


class Graph:
    """Owner of a g3_graph*; frees it on free() or garbage collection."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle

    def free(self):
        if self.handle and self.handle.value:
            import torch
            torch.cuda.synchronize()
            lib().g3_graph_free(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            if self.handle and self.handle.value:
                lib().g3_graph_free(self.handle)
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return g3_graph_info_get(self)

    def perm(self, device="cuda"):
        import torch
        n = self.info["n"]
        a = torch.empty(n, dtype=torch.int32, device=device)
        b = torch.empty(n, dtype=torch.int32, device=device)
        g3_get_perm(self, a, b)
        return a, b

    def csr(self, device="cuda"):
        import torch
        i = self.info
        off = torch.empty(i["n_bfs"] + 1, dtype=torch.int64, device=device)
        col = torch.empty(max(i["nnz"], 1), dtype=torch.int32, device=device)
        g3_get_csr(self, off, col)
        return off, col[:i["nnz"]]
