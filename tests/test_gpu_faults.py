"""Error paths under injected faults (host-side hooks, no GPU fault): every
device allocation of a call made to fail in turn must give G3_ENOMEM, leave
nothing of the call allocated and the graph as it was, and the same call
must then succeed and agree with the oracle; an RCM relabel capped below the
hooking rounds it needs must give G3_ETIMEOUT and leave the graph usable; a
kernel's bounded wait that runs out (its data never arrives) must give
G3_ETIMEOUT and leave the device usable."""
import numpy as np
import pytest

import graphgen
import oracle
from _graphs import path_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_10026_gb300 as g3  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


@pytest.fixture(autouse=True)
def _disarm():
    yield
    g3.g3_debug_inject(g3.G3_INJECT_ALLOC, 0)
    g3.g3_debug_inject(g3.G3_INJECT_RCM_ROUNDS, 0)
    g3.g3_debug_inject(g3.G3_INJECT_STAGED_STALL, 0)


def _each_allocation_fails(call, check_clean, limit=200):
    """Runs call() with the k-th allocation failing, k = 1, 2, ... until the
    call no longer reaches a k-th allocation. Returns the number of
    allocation sites that failed cleanly and the successful result."""
    for k in range(1, limit):
        g3.g3_debug_inject(g3.G3_INJECT_ALLOC, k)
        try:
            res = call()
        except g3.G3Error as e:
            assert e.status == g3.G3_ENOMEM, (k, e)
            torch.cuda.synchronize()
            check_clean(k)
            continue
        g3.g3_debug_inject(g3.G3_INJECT_ALLOC, 0)
        return k - 1, res
    raise AssertionError("the call kept allocating")


def test_build_csr_allocation_failures_are_clean():
    scale, n = 10, 1 << 10
    src, dst = graphgen.kronecker_edges(scale, 16, seed=7)
    s, d = _dev(src), _dev(dst)
    torch.cuda.synchronize()
    base = g3.g3_debug_pool_used()

    def clean(k):
        assert g3.g3_debug_pool_used() == base, k

    sites, g = _each_allocation_fails(lambda: g3.g3_build_csr(s, d, n), clean)
    assert sites >= 5
    off, col = g.csr()
    off_o, col_o = oracle.build_csr(src, dst, n)
    assert np.array_equal(off.cpu().numpy(), off_o) and np.array_equal(col.cpu().numpy(), col_o)
    g.free()


def test_rcm_allocation_failures_leave_the_graph_as_it_was():
    scale, n = 11, 1 << 11
    src, dst = graphgen.kronecker_edges(scale, 16, seed=8)
    ref = oracle.pipeline(src, dst, n)
    g = g3.g3_build_csr(_dev(src), _dev(dst), n)
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    root = int(graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 1, seed=9)[0])
    _, lref = oracle.bfs(ref["off"], ref["col"], root)
    torch.cuda.synchronize()
    base = g3.g3_debug_pool_used()

    def clean(k):
        assert g3.g3_debug_pool_used() == base, k
        assert g.info["relabelled"] == 0
        g3.g3_bfs(g, root, parent, level)  # the unrelabelled graph still searches
        assert np.array_equal(level.cpu().numpy(), lref), k

    sites, _ = _each_allocation_fails(lambda: g3.g3_rcm_relabel(g), clean)
    assert sites >= 10
    old_of_new, _ = g.perm()
    assert np.array_equal(old_of_new.cpu().numpy(), ref["P"])
    g3.g3_bfs(g, root, parent, level)
    assert np.array_equal(level.cpu().numpy(), lref)
    g.free()


def test_bfs_and_msbfs_workspace_failures():
    scale, n = 12, 1 << 12
    src, dst = graphgen.kronecker_edges(scale, 16, seed=10)
    ref = oracle.pipeline(src, dst, n)
    roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 3, seed=11).tolist()
    want = np.stack([oracle.bfs(ref["off"], ref["col"], r)[1] for r in roots])
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    lv8 = torch.empty((len(roots), n), dtype=torch.int8, device="cuda")
    for call in ("bfs", "msbfs"):
        g = g3.g3_build_csr(_dev(src), _dev(dst), n)
        g3.g3_rcm_relabel(g)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]

        def clean(k):
            # workspaces come from cudaMalloc: what a failed call took is back
            assert abs(torch.cuda.mem_get_info()[0] - free0) < (2 << 20), k

        if call == "bfs":
            sites, _ = _each_allocation_fails(
                lambda: g3.g3_bfs(g, roots[0], parent, level), clean)
            assert np.array_equal(level.cpu().numpy(), want[0])
            assert oracle.validate(ref["off"], ref["col"], roots[0], parent.cpu().numpy(),
                                   level.cpu().numpy()) == 0
        else:
            sites, _ = _each_allocation_fails(lambda: g3.g3_msbfs(g, roots, lv8), clean)
            assert np.array_equal(lv8.cpu().numpy(), want.astype(np.int8))
        assert sites >= 8, (call, sites)
        g.free()


def test_batch_pack_allocation_failures():
    specs = graphgen.small_graph_specs(3, seed=12)
    graphs, host, voff, roots = [], [], [0], []
    for sc, gs in specs:
        s, d = graphgen.kronecker_edges(sc, 16, seed=gs)
        gg = g3.g3_build_csr(_dev(s), _dev(d), 1 << sc)
        g3.g3_rcm_relabel(gg)
        graphs.append(gg)
        r = int(graphgen.pick_roots(graphgen.nonisolated_flags(s, d, 1 << sc), 1, gs)[0])
        host.append((s, d, 1 << sc, r))
        roots.append(voff[-1] + r)
        voff.append(voff[-1] + (1 << sc))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]

    def clean(k):
        assert abs(torch.cuda.mem_get_info()[0] - free0) < (2 << 20), k

    sites, b = _each_allocation_fails(lambda: g3.g3_batch_pack(graphs), clean)
    assert sites >= 5
    for gg in graphs:
        gg.free()
    bp = torch.empty(voff[-1], dtype=torch.int32, device="cuda")
    bl = torch.empty(voff[-1], dtype=torch.int32, device="cuda")
    g3.g3_bfs_batch(b, torch.tensor(roots, dtype=torch.int32, device="cuda"), bp, bl)
    bl = bl.cpu().numpy()
    for (s, d, nn, r), vb in zip(host, voff):
        o, c = oracle.build_csr(s, d, nn)
        assert np.array_equal(bl[vb:vb + nn], oracle.bfs(o, c, r)[1])
    b.free()


def test_rcm_hooking_cap_gives_timeout_and_a_usable_graph():
    # a path with scattered IDs needs several hooking rounds; one is allowed
    n = 4096
    ids = np.random.default_rng(3).permutation(n).astype(np.int32)
    src, dst = ids[:-1], ids[1:]
    off_o, col_o = oracle.build_csr(src, dst, n)
    P, _ = oracle.rcm(off_o, col_o)
    g = g3.g3_build_csr(_dev(src), _dev(dst), n)
    torch.cuda.synchronize()
    base = g3.g3_debug_pool_used()
    g3.g3_debug_inject(g3.G3_INJECT_RCM_ROUNDS, 1)
    with pytest.raises(g3.G3Error) as e:
        g3.g3_rcm_relabel(g)
    assert e.value.status == g3.G3_ETIMEOUT
    torch.cuda.synchronize()
    assert g3.g3_debug_pool_used() == base and g.info["relabelled"] == 0
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    g3.g3_bfs(g, int(ids[0]), parent, level)
    want = np.full(n, -1, np.int32)
    want[ids] = np.arange(n)
    assert np.array_equal(level.cpu().numpy(), want)
    g3.g3_debug_inject(g3.G3_INJECT_RCM_ROUNDS, 0)
    g3.g3_rcm_relabel(g)
    assert np.array_equal(g.perm()[0].cpu().numpy(), P)
    g.free()


def test_inject_rejects_unknown_kind():
    with pytest.raises(g3.G3Error) as e:
        g3.g3_debug_inject(99, 1)
    assert e.value.status == g3.G3_EINVAL


def test_staged_kernel_wait_runs_out_and_the_device_stays_usable():
    # the staged bottom-up kernel's first tile never arrives: its bounded
    # wait ends, the search reports G3_ETIMEOUT, and the next search (hook
    # off) is exact
    scale, n = 14, 1 << 14
    src, dst = graphgen.kronecker_edges(scale, 16, seed=13)
    ref = oracle.pipeline(src, dst, n)
    g = g3.g3_build_csr(_dev(src), _dev(dst), n)
    g3.g3_rcm_relabel(g)
    root = int(graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 1, seed=14)[0])
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    o = g3.opts(controller=g3.G3_CTRL_BOTTOMUP, bu_kernel=1)
    g3.g3_debug_inject(g3.G3_INJECT_STAGED_STALL, 1000)
    for timing in (0, 1):  # the level-loop graph and the host-driven loop
        with pytest.raises(g3.G3Error) as e:
            g3.g3_bfs(g, root, parent, level, g3.opts(controller=g3.G3_CTRL_BOTTOMUP,
                                                      bu_kernel=1, timing=timing))
        assert e.value.status == g3.G3_ETIMEOUT
    g3.g3_debug_inject(g3.G3_INJECT_STAGED_STALL, 0)
    g3.g3_bfs(g, root, parent, level, o)
    _, lref = oracle.bfs(ref["off"], ref["col"], root)
    assert np.array_equal(level.cpu().numpy(), lref)
    assert oracle.validate(ref["off"], ref["col"], root, parent.cpu().numpy(),
                           level.cpu().numpy()) == 0
    g.free()
