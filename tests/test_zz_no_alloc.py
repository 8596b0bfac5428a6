"""The allocation-free BFS entry point (g3_bfs_noalloc) against the regular
one (g3_bfs). g3_bfs_noalloc serves callers that cannot allocate device
memory while they search (their framework owns the device memory, or an
allocation could synchronise the device); its scratch is a fixed static
device array shared by all calls. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import graphgen  # noqa: E402
import oracle  # noqa: E402
import paper_2012_10026_gb300 as g3  # noqa: E402


def test_noalloc_matches_g3_bfs_on_two_calls_in_a_row():
    scale, n = 14, 1 << 14
    src, dst = graphgen.kronecker_edges(scale, 16, seed=3)
    g = g3.g3_build_csr(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    off, col = g.csr()
    off_h, col_h = off.cpu().numpy(), col.cpu().numpy()
    roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 2, seed=4).tolist()
    for root in roots:  # two calls in a row share the static scratch
        p = torch.empty(n, dtype=torch.int32, device="cuda")
        l = torch.empty(n, dtype=torch.int32, device="cuda")
        g3.g3_bfs_noalloc(off, col, n, root, p, l)
        p_ref = torch.empty(n, dtype=torch.int32, device="cuda")
        l_ref = torch.empty(n, dtype=torch.int32, device="cuda")
        g3.g3_bfs(g, root, p_ref, l_ref)
        torch.cuda.synchronize()
        lv, pv = l.cpu().numpy(), p.cpu().numpy()
        # level[] is unique: equal exactly; parent[] may differ but must be valid
        assert np.array_equal(lv, l_ref.cpu().numpy()), root
        assert oracle.validate(off_h, col_h, root, pv, lv) == 0, root
    g.free()


def test_noalloc_at_its_largest_size():
    # n == G3_NOALLOC_MAX_N exactly: the visited bitmap and both queues of the
    # static array are used to their full extent
    n = g3.NOALLOC_MAX_N
    scale = n.bit_length() - 1
    src, dst = graphgen.kronecker_edges(scale, 16, seed=5)
    g = g3.g3_build_csr(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    off, col = g.csr()
    off_h, col_h = off.cpu().numpy(), col.cpu().numpy()
    root = int(graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 1, seed=6)[0])
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    l = torch.empty(n, dtype=torch.int32, device="cuda")
    g3.g3_bfs_noalloc(off, col, n, root, p, l)
    p_ref = torch.empty(n, dtype=torch.int32, device="cuda")
    l_ref = torch.empty(n, dtype=torch.int32, device="cuda")
    g3.g3_bfs(g, root, p_ref, l_ref)
    torch.cuda.synchronize()
    lv, pv = l.cpu().numpy(), p.cpu().numpy()
    assert np.array_equal(lv, l_ref.cpu().numpy())
    assert oracle.validate(off_h, col_h, root, pv, lv) == 0
    g.free()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = g3.lib()
    dummy = ctypes.c_void_p(16)  # never dereferenced: rejected on the host
    st = L.g3_bfs_noalloc(dummy, dummy, g3.NOALLOC_MAX_N + 1, 0, dummy, dummy, None)
    assert st == g3.G3_EINVAL
    assert b"static scratch" in L.g3_last_error_detail()
    assert L.g3_bfs_noalloc(dummy, dummy, 0, 0, dummy, dummy, None) == g3.G3_EINVAL
