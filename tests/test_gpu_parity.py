"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs. CSR and RCM permutation bit-exact, level[] bit-exact,
parent[] valid under the BFS-tree rules, per-level statistics and the
direction sequence equal to the oracle's."""
import numpy as np
import pytest
from conftest import read_golden_cases

import graphgen
import oracle
from oracle import direction
from _graphs import band_graph, path_graph, random_graph, star_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_10026_gb300 as g3  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def gpu_pipeline(src, dst, n, relabel=True):
    g = g3.g3_build_csr(_dev(src), _dev(dst), n)
    if relabel:
        g3.g3_rcm_relabel(g)
    return g


def gpu_csr(g):
    off, col = g.csr()
    return off.cpu().numpy(), col.cpu().numpy()


def run_bfs(g, root, n, max_stats=0, **kw):
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    st = g3.g3_bfs(g, root, parent, level, g3.opts(**kw) if kw else None, max_stats=max_stats)
    return parent.cpu().numpy(), level.cpu().numpy(), st


def small_cases():
    cases = []
    for c in read_golden_cases("rcm_bfs_cases.txt"):
        cases.append((c["name"], np.array(c["src"], np.int32), np.array(c["dst"], np.int32),
                      c["n"]))
    rng = np.random.default_rng(77)
    for i in range(12):
        n = int(rng.integers(1, 300))
        s, d = random_graph(rng, n, int(rng.integers(0, 4 * n)))
        cases.append((f"random{i}", s, d, n))
    cases.append(("path", *path_graph(50), 50))
    cases.append(("star", *star_graph(40, 7), 40))
    sigma = np.random.default_rng(5).permutation(120).astype(np.int32)
    cases.append(("band", *band_graph(120, 4, sigma), 120))
    cases.append(("empty", np.zeros(0, np.int32), np.zeros(0, np.int32), 9))
    cases.append(("loops_only", np.array([1, 2], np.int32), np.array([1, 2], np.int32), 4))
    cases.append(("single_vertex", np.zeros(0, np.int32), np.zeros(0, np.int32), 1))
    for sc, ef, seed in ((10, 16, 1), (13, 8, 9)):
        s, d = graphgen.kronecker_edges(sc, ef, seed=seed)
        cases.append((f"kron{sc}", s, d, 1 << sc))
    s, d = graphgen.chunglu_edges(3000, seed=3)
    cases.append(("chunglu3000", s, d, 3000))
    return cases


CASES = small_cases()


# ------------------------------------------------------------ generators
@pytest.mark.parametrize("scale", [10, 14])
def test_kronecker_device_twin_matches_host(scale):
    hs, hd = graphgen.kronecker_edges(scale, 16, seed=1)
    ds, dd = graphgen.kronecker_edges_dev(scale, 16, seed=1)
    assert np.array_equal(ds.cpu().numpy(), hs) and np.array_equal(dd.cpu().numpy(), hd)
    f = graphgen.nonisolated_flags_dev(ds, dd, 1 << scale).cpu().numpy()
    assert np.array_equal(f, graphgen.nonisolated_flags(hs, hd, 1 << scale))


def test_chunglu_device_twin_matches_host():
    hs, hd = graphgen.chunglu_edges(5000, seed=3)
    ds, dd = graphgen.chunglu_edges_dev(5000, seed=3)
    assert np.array_equal(ds.cpu().numpy(), hs) and np.array_equal(dd.cpu().numpy(), hd)


# ------------------------------------------------------------ CSR and RCM
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_csr_and_rcm_bit_exact(case):
    name, src, dst, n = case
    off_o, col_o = oracle.build_csr(src, dst, n)
    g = gpu_pipeline(src, dst, n, relabel=False)
    off_g, col_g = gpu_csr(g)
    assert np.array_equal(off_g, off_o) and np.array_equal(col_g, col_o)
    info = g.info
    assert info["nnz"] == len(col_o) and info["max_degree"] == (np.diff(off_o).max() if n else 0)
    g3.g3_rcm_relabel(g)
    P, n_plus = oracle.rcm(off_o, col_o)
    old_of_new, new_of_old = g.perm()
    assert np.array_equal(old_of_new.cpu().numpy(), P)
    assert np.array_equal(new_of_old.cpu().numpy(), oracle.permutation_arrays(P)[1])
    assert g.info["n_plus"] == n_plus and g.info["n_bfs"] == n_plus
    off_r, col_r = oracle.permute_csr(off_o, col_o, P, n_plus)
    off_g, col_g = gpu_csr(g)
    assert np.array_equal(off_g, off_r) and np.array_equal(col_g, col_r)
    with pytest.raises(g3.G3Error) as e:
        g3.g3_rcm_relabel(g)
    assert e.value.status == g3.G3_ESTATE
    g.free()


# ------------------------------------------------------------ BFS
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("relabel", [True, False])
def test_bfs_small_cases(case, relabel):
    name, src, dst, n = case
    off_o, col_o = oracle.build_csr(src, dst, n)
    g = gpu_pipeline(src, dst, n, relabel)
    rng = np.random.default_rng(n)
    roots = sorted(set([0, n - 1] + rng.integers(0, n, 6).tolist()))
    # bottom-up in every kernel set (word pairs, staged + word tiles, word
    # tiles, word pairs + word tiles) and both scan orders; the output pass in one pass and split over
    # label halves
    for ctrl, rev, kern, split in ((g3.G3_CTRL_HEURISTIC, 1, 0, 0),
                                   (g3.G3_CTRL_HEURISTIC, 1, 1, 2),
                                   (g3.G3_CTRL_TOPDOWN, 1, 0, 1),
                                   (g3.G3_CTRL_BOTTOMUP, 1, 0, 0), (g3.G3_CTRL_BOTTOMUP, 0, 0, 0),
                                   (g3.G3_CTRL_BOTTOMUP, 1, 1, 0), (g3.G3_CTRL_BOTTOMUP, 0, 1, 2),
                                   (g3.G3_CTRL_BOTTOMUP, 1, 2, 0), (g3.G3_CTRL_BOTTOMUP, 1, 3, 0),
                                   (g3.G3_CTRL_HEURISTIC, 0, 3, 0)):
        for root in roots:
            parent, level, _ = run_bfs(g, root, n, controller=ctrl, bu_reverse=rev,
                                       bu_kernel=kern, out_split=split)
            _, lref = oracle.bfs(off_o, col_o, root)
            assert np.array_equal(level, lref), (name, root, ctrl)
            assert oracle.validate(off_o, col_o, root, parent, level) == 0, (name, root, ctrl)
    g.free()


@pytest.fixture(scope="module")
def kron16():
    scale, n = 16, 1 << 16
    src, dst = graphgen.kronecker_edges(scale, 16, seed=1)
    ref = oracle.pipeline(src, dst, n)
    roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 64, seed=2)
    g = gpu_pipeline(src, dst, n)
    yield dict(src=src, dst=dst, n=n, ref=ref, roots=roots, g=g)
    g.free()


def _levels_new(ref, level_orig):
    return level_orig[ref["old_of_new"][:ref["n_plus"]]]


@pytest.mark.parametrize("kw", [dict(), dict(controller=g3.G3_CTRL_TOPDOWN),
                                dict(controller=g3.G3_CTRL_BOTTOMUP), dict(bu_reverse=0),
                                dict(controller=g3.G3_CTRL_BOTTOMUP, bu_reverse=0),
                                dict(t1=2, t2=4, t3=8), dict(alpha=64, beta=8),
                                dict(bu_kernel=1),
                                dict(controller=g3.G3_CTRL_BOTTOMUP, bu_kernel=1),
                                dict(out_split=2), dict(out_split=1),
                                dict(controller=g3.G3_CTRL_BOTTOMUP, bu_kernel=2),
                                dict(bu_kernel=3),
                                dict(controller=g3.G3_CTRL_BOTTOMUP, bu_kernel=3)],
                         ids=["heuristic", "topdown", "bottomup", "forward_scan",
                              "bottomup_forward", "tiny_bins", "alpha64_beta8", "staged",
                              "bottomup_staged", "out_split", "out_one_pass",
                              "bottomup_tiles", "pairs_tiles", "bottomup_pairs_tiles"])
def test_bfs_kron16_all_roots(kron16, kw):
    K = kron16
    ref = K["ref"]
    for root in K["roots"].tolist():
        parent, level, st = run_bfs(K["g"], root, K["n"], max_stats=64, **kw)
        _, lref = oracle.bfs(ref["off"], ref["col"], root)
        assert np.array_equal(level, lref), root
        assert oracle.validate(ref["off"], ref["col"], root, parent, level) == 0, root
        # per-level statistics equal the oracle's level sets
        lnew = _levels_new(ref, lref)
        ost = direction.level_stats(ref["off_r"], lnew)
        assert len(st) == len(ost)
        for L, (a, b) in enumerate(zip(st, ost)):
            assert (a["n_f"], a["m_f"], a["n_u"], a["m_u"]) == (b["n_f"], b["m_f"], b["n_u"],
                                                                b["m_u"]), (root, L)
            f = np.nonzero(lnew == L)[0]
            assert a["id_min"] == f.min() and a["id_max"] == f.max()
            if a["dir"] == g3.G3_DIR_BU:
                assert a["examined"] == oracle.bu_examined(ref["off_r"], ref["col_r"], lnew, L,
                                                           reverse=bool(kw.get("bu_reverse", 1)))
        if not kw.get("controller"):
            expect = direction.heuristic_directions(ref["off_r"], lnew, kw.get("alpha", 14),
                                                    kw.get("beta", 24))
            assert [a["dir"] for a in st] == expect, root


def test_bfs_host_outputs_equal_device_outputs(kron16):
    K = kron16
    root = int(K["roots"][0])
    pd, ld, _ = run_bfs(K["g"], root, K["n"])
    ph = np.full(K["n"], 7, np.int32)
    lh = np.full(K["n"], 7, np.int32)
    g3.g3_bfs(K["g"], root, ph, lh)
    assert np.array_equal(lh, ld)
    assert oracle.validate(K["ref"]["off"], K["ref"]["col"], root, ph, lh) == 0
    pinned_p = torch.empty(K["n"], dtype=torch.int32).pin_memory()
    pinned_l = torch.empty(K["n"], dtype=torch.int32).pin_memory()
    g3.g3_bfs(K["g"], root, pinned_p, pinned_l)
    assert np.array_equal(pinned_l.numpy(), ld)


def test_bfs_isolated_root_and_bad_root(kron16):
    K = kron16
    deg = np.diff(K["ref"]["off"])
    iso = int(np.nonzero(deg == 0)[0][0])
    parent, level, st = run_bfs(K["g"], iso, K["n"], max_stats=4)
    assert level[iso] == 0 and parent[iso] == iso
    assert (level >= 0).sum() == 1 and (parent >= 0).sum() == 1 and st == []
    with pytest.raises(g3.G3Error) as e:
        run_bfs(K["g"], K["n"], K["n"])
    assert e.value.status == g3.G3_EINVAL
    with pytest.raises(g3.G3Error):
        run_bfs(K["g"], -1, K["n"])


def test_learned_controller_random_params_stays_exact(kron16):
    from oracle import mlp
    K = kron16
    ref = K["ref"]
    from paper_2012_10026_gb300 import train_controller as tc
    params = torch.from_numpy(mlp.init_params(5).astype(np.float32)).cuda()
    seen = 0
    for root in K["roots"][:8].tolist():
        parent, level, st = run_bfs(K["g"], root, K["n"], max_stats=64,
                                    controller=g3.G3_CTRL_LEARNED, mlp_params=params)
        _, lref = oracle.bfs(ref["off"], ref["col"], root)
        assert np.array_equal(level, lref)
        assert oracle.validate(ref["off"], ref["col"], root, parent, level) == 0
        consulted = 0
        for a in st[1:]:
            prev = st[a["level"] - 1]
            if not tc.rule_near(prev["dir"], a["n_f"], a["m_f"], a["m_u"], ref["n_plus"]):
                # the rule's test is clear by a factor of 4: the network is
                # not evaluated and the rule decides
                assert list(a["mlp_out"]) == [0.0] * 4
                continue
            consulted += 1
            f = mlp.features(a["n_f"], a["m_f"], a["n_u"], a["m_u"], ref["n_plus"],
                             len(ref["col_r"]), prev["dir"], a["level"], prev["n_f"])
            o = mlp.forward(mlp.init_params(5), f[None])[0]
            assert np.allclose(a["mlp_out"], o, rtol=1e-4, atol=1e-4)
            if abs(o[0]) > 1e-3:
                assert a["dir"] == (g3.G3_DIR_BU if o[0] < 0 else g3.G3_DIR_TD)
        seen += consulted
    assert seen > 0  # some levels were the network's to decide


@pytest.mark.parametrize("margin", [0, 300, 2000, 10 ** 9])
def test_learned_controller_margin_falls_back_to_rule(kron16, margin):
    """Inside the margin the alpha/beta rule decides (from the directions
    actually taken); outside it the network's sign decides."""
    from oracle import mlp
    K = kron16
    ref = K["ref"]
    params = torch.from_numpy(mlp.init_params(5).astype(np.float32)).cuda()
    for root in K["roots"][:6].tolist():
        parent, level, st = run_bfs(K["g"], root, K["n"], max_stats=64,
                                    controller=g3.G3_CTRL_LEARNED, mlp_params=params,
                                    mlp_margin=margin)
        _, lref = oracle.bfs(ref["off"], ref["col"], root)
        assert np.array_equal(level, lref)
        assert oracle.validate(ref["off"], ref["col"], root, parent, level) == 0
        assert st[0]["dir"] == g3.G3_DIR_TD
        for L in range(1, len(st)):
            a, prev = st[L], st[L - 1]
            o0 = a["mlp_out"][0]
            if abs(abs(o0) - margin / 1000) < 1e-4:
                continue  # too close to the margin to call
            if abs(o0) > margin / 1000:
                want = g3.G3_DIR_BU if o0 < 0 else g3.G3_DIR_TD
            elif prev["dir"] == g3.G3_DIR_TD:
                want = g3.G3_DIR_BU if a["m_f"] * 14 > a["m_u"] else g3.G3_DIR_TD
            else:
                shrink = a["n_f"] < prev["n_f"] and a["n_f"] * 24 < ref["n_plus"]
                want = g3.G3_DIR_TD if shrink else g3.G3_DIR_BU
            assert a["dir"] == want, (root, L, o0)
    if margin == 10 ** 9:  # never overrides: the heuristic's directions
        lnew = _levels_new(ref, lref)
        assert [a["dir"] for a in st] == direction.heuristic_directions(ref["off_r"], lnew)


def test_bad_edge_endpoint_rejected():
    with pytest.raises(g3.G3Error) as e:
        g3.g3_build_csr(_dev([0, 1]), _dev([1, 5]), 5)
    assert e.value.status == g3.G3_EINVAL


def test_kron22_permutation_and_levels():
    scale, n = 22, 1 << 22
    src, dst = graphgen.kronecker_edges(scale, 16, seed=1)
    ref = oracle.pipeline(src, dst, n)
    g = gpu_pipeline(src, dst, n)
    old_of_new, _ = g.perm()
    assert np.array_equal(old_of_new.cpu().numpy(), ref["P"])
    off_g, col_g = gpu_csr(g)
    assert np.array_equal(off_g, ref["off_r"]) and np.array_equal(col_g, ref["col_r"])
    roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 64, seed=2)
    for i, root in enumerate(roots[:6].tolist()):
        parent, level, _ = run_bfs(g, root, n, out_split=1 + i % 2, bu_kernel=(0, 1, 3)[i // 2])
        _, lref = oracle.bfs(ref["off"], ref["col"], root)
        assert np.array_equal(level, lref)
        assert oracle.validate(ref["off"], ref["col"], root, parent, level) == 0
    g.free()


def test_record_both_mode_keeps_results_exact(kron16):
    K = kron16
    ref = K["ref"]
    sweep = {(8, 256, 8192), (16, 512, 16384), (32, 1024, 32768), (64, 2048, 65536),
             (128, 4096, 131072)}
    for root in K["roots"][:4].tolist():
        parent, level, st = run_bfs(K["g"], root, K["n"], max_stats=64, record_both=1, timing=1)
        _, lref = oracle.bfs(ref["off"], ref["col"], root)
        assert np.array_equal(level, lref)
        assert oracle.validate(ref["off"], ref["col"], root, parent, level) == 0
        assert st and all(a["t_td_ms"] > 0 and a["t_bu_ms"] > 0 for a in st)
        assert all((a["best_t1"], a["best_t2"], a["best_t3"]) in sweep for a in st)


def test_counts_only_statistics_equal_the_full_ones(kron16):
    # stats_counts_only: the same counts per level as the full statistics,
    # the histogram and label range left at zero, the same results
    K = kron16
    for root in K["roots"][:4].tolist():
        for timing in (0, 1):
            p_f, l_f, st_f = run_bfs(K["g"], root, K["n"], max_stats=64, timing=timing)
            p_c, l_c, st_c = run_bfs(K["g"], root, K["n"], max_stats=64, timing=timing,
                                     stats_counts_only=1)
            assert np.array_equal(l_f, l_c) and len(st_f) == len(st_c)
            for a, b in zip(st_f, st_c):
                for key in ("level", "dir", "n_f", "m_f", "n_u", "m_u", "examined", "n_next"):
                    assert a[key] == b[key], (root, key)
                if b["level"] > 0:
                    assert list(b["hist"]) == [0, 0, 0, 0]


def test_graph_mode_equals_host_driven_mode(kron16):
    # default searches run the level loop as one CUDA graph; per-level timing
    # switches to the host-driven loop. Both must give the same levels, the
    # same per-level statistics and the same direction sequence.
    K = kron16
    for root in K["roots"][:16].tolist():
        _, lg, sg = run_bfs(K["g"], root, K["n"], max_stats=64)
        _, lh, sh = run_bfs(K["g"], root, K["n"], max_stats=64, timing=1)
        assert np.array_equal(lg, lh)
        keys = ["level", "dir", "n_f", "m_f", "n_u", "m_u", "examined", "n_next", "id_min",
                "id_max", "hist"]
        assert [[a[k] for k in keys] for a in sg] == [[a[k] for k in keys] for a in sh]
        assert all(a["ms"] > 0 and a["ms_expand"] > 0 for a in sh)


def test_deep_graph_beyond_graph_level_cap():
    # a path longer than the 4096 levels one graph launch may run: the search
    # continues on the host-driven loop and stays exact
    n = 5000
    src, dst = path_graph(n)
    off, col = oracle.build_csr(src, dst, n)
    for relabel in (True, False):
        g = gpu_pipeline(src, dst, n, relabel)
        parent, level, st = run_bfs(g, 0, n, max_stats=8)
        assert level.tolist() == list(range(n))
        assert oracle.validate(off, col, 0, parent, level) == 0
        assert len(st) == 8 and st[7]["n_f"] == 1
        g.free()


@pytest.mark.parametrize("relabel,split", [(True, 1), (True, 2), (False, 0)])
@pytest.mark.parametrize("ctrl", ["heuristic", "topdown", "bottomup"])
def test_levels_past_the_packed_word(relabel, split, ctrl):
    # n = 2^26 leaves 6 level bits in the packed (parent, level) word, so
    # levels from 63 on come from the side table; a 300-vertex path spread
    # over the ID range, searched from its 101st vertex, reaches level 199
    n, k, mid = 1 << 26, 300, 100
    ids = ((np.arange(k, dtype=np.int64) * 223_001 + 17) % n).astype(np.int32)
    g = gpu_pipeline(ids[:-1], ids[1:], n, relabel)
    c = {"heuristic": g3.G3_CTRL_HEURISTIC, "topdown": g3.G3_CTRL_TOPDOWN,
         "bottomup": g3.G3_CTRL_BOTTOMUP}[ctrl]
    parent, level, _ = run_bfs(g, int(ids[mid]), n, controller=c, out_split=split)
    want = np.full(n, -1, np.int32)
    want[ids] = np.abs(np.arange(k) - mid)
    assert np.array_equal(level, want)
    pw = np.full(n, -1, np.int32)
    pos = np.arange(k)
    pw[ids] = ids[np.clip(np.where(pos > mid, pos - 1, pos + 1), 0, k - 1)]
    pw[ids[mid]] = ids[mid]
    assert np.array_equal(parent, pw)
    g.free()


def test_roots_in_every_component_after_stale_searches():
    # after a full relabel each component is one label range, and the output
    # pass takes "reached" from the root's range instead of the visited
    # bitmap: search the largest component first, so that every packed
    # (parent, level) word holds a stale value, then one root in each other
    # component (sizes 2 to several hundred, isolated vertices in between);
    # any vertex the range wrongly includes or leaves out shows up as a level
    # that differs from the oracle's
    rng = np.random.default_rng(31)
    parts, base = [], 0
    for k in [700, 2, 3, 5, 40, 2, 260, 9, 2, 120]:
        if k == 2:
            s, d = np.array([0], np.int32), np.array([1], np.int32)
        elif k < 10:
            s, d = path_graph(k)
        else:  # a spanning path plus random chords: connected
            ps, pd = path_graph(k)
            cs, cd = random_graph(rng, k, 2 * k, allow_loops=False)
            s, d = np.concatenate([ps, cs]), np.concatenate([pd, cd])
        parts.append((s + base, d + base, base, k))
        base += k + int(rng.integers(0, 4))  # isolated vertices between parts
    n = base + 3
    sigma = rng.permutation(n).astype(np.int32)  # scatter the original IDs
    src = sigma[np.concatenate([p[0] for p in parts])]
    dst = sigma[np.concatenate([p[1] for p in parts])]
    off, col = oracle.build_csr(src, dst, n)
    g = gpu_pipeline(src, dst, n)
    roots = [int(sigma[b + int(rng.integers(0, k))]) for _, _, b, k in parts]
    roots.append(int(sigma[n - 1]))  # an isolated root
    for root in roots:
        for ctrl in (g3.G3_CTRL_HEURISTIC, g3.G3_CTRL_BOTTOMUP):
            parent, level, _ = run_bfs(g, root, n, controller=ctrl)
            _, lref = oracle.bfs(off, col, root)
            assert np.array_equal(level, lref), root
            assert oracle.validate(off, col, root, parent, level) == 0, root
    g.free()


@pytest.mark.parametrize("pm", [0, 1, 250, 500, 999, 1000])
def test_partial_rcm_permutation_and_bfs_equal_oracle(pm):
    cases = [graphgen.kronecker_edges(14, 16, seed=21) + (1 << 14,)]
    rng = np.random.default_rng(pm)
    for _ in range(4):
        n = int(rng.integers(2, 3000))
        cases.append(random_graph(rng, n, int(rng.integers(n // 2, 4 * n))) + (n,))
    for src, dst, n in cases:
        off, col = oracle.build_csr(src, dst, n)
        P, n_plus = oracle.rcm_partial(off, col, pm)
        g = g3.g3_build_csr(_dev(src), _dev(dst), n)
        g3.g3_rcm_relabel_partial(g, pm)
        assert g.info["n_plus"] == n_plus
        old_of_new, _ = g.perm()
        assert np.array_equal(old_of_new.cpu().numpy(), P), (n, pm)
        roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 3, 5).tolist()
        for r in roots:
            parent, level, _ = run_bfs(g, r, n)
            _, lref = oracle.bfs(off, col, r)
            assert np.array_equal(level, lref)
            assert oracle.validate(off, col, r, parent, level) == 0
        g.free()


def test_partial_rcm_bad_fraction():
    src, dst = path_graph(10)
    g = g3.g3_build_csr(_dev(src), _dev(dst), 10)
    for bad in (-1, 1001):
        with pytest.raises(g3.G3Error) as e:
            g3.g3_rcm_relabel_partial(g, bad)
        assert e.value.status == g3.G3_EINVAL
    g3.g3_rcm_relabel_partial(g, 500)
    with pytest.raises(g3.G3Error) as e:
        g3.g3_rcm_relabel_partial(g, 500)
    assert e.value.status == g3.G3_ESTATE
    g.free()
