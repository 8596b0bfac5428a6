"""Autotuner cache file and size classes (host only, no GPU)."""
import pytest

g3 = pytest.importorskip("paper_2012_10026_gb300")


def _entry(kind, sc, dc, p, ms=1.5, points=7):
    e = g3.g3_tune_entry()
    e.kind, e.size_class, e.deg_class = kind, sc, dc
    for i, v in enumerate(p):
        e.p[i] = v
    e.points, e.ms, e.ms_default = points, ms, 2 * ms
    return e


def test_tune_key_classes():
    assert g3.tune_key(g3.G3_TUNE_BFS, 1 << 20, 1 << 24) == (20, 4)
    assert g3.tune_key(g3.G3_TUNE_BFS, (1 << 20) + 5, 3 << 24) == (20, 5)
    # a batch is keyed by its mean graph size
    assert g3.tune_key(g3.G3_TUNE_BATCH, 4096 * 3000, 4096 * 3000 * 20, 4096) == (11, 4)
    assert g3.tune_key(g3.G3_TUNE_BFS, 0, 0) == (0, 0)
    with pytest.raises(g3.G3Error):
        g3.tune_key(g3.G3_TUNE_BFS, 10, 10, 0)


def test_cache_roundtrip_and_replace(tmp_path):
    path = str(tmp_path / "tune.txt")
    assert g3.tune_cache_lookup(path, g3.G3_TUNE_BFS, 20, 4) is None  # no file yet
    g3.tune_cache_store(path, _entry(g3.G3_TUNE_BFS, 20, 4, [14, 24, 32, 1024, 32768, 1]))
    g3.tune_cache_store(path, _entry(g3.G3_TUNE_MSBFS, 24, 4, [8, 128]))
    e = g3.tune_cache_lookup(path, g3.G3_TUNE_BFS, 20, 4)
    assert list(e.p) == [14, 24, 32, 1024, 32768, 1] and e.points == 7
    assert abs(e.ms - 1.5) < 1e-6 and abs(e.ms_default - 3.0) < 1e-6
    # same key replaces in place; other keys stay
    g3.tune_cache_store(path, _entry(g3.G3_TUNE_BFS, 20, 4, [20, 12, 16, 512, 16384, 0], ms=1.0))
    assert list(g3.tune_cache_lookup(path, g3.G3_TUNE_BFS, 20, 4).p) == [20, 12, 16, 512,
                                                                          16384, 0]
    assert list(g3.tune_cache_lookup(path, g3.G3_TUNE_MSBFS, 24, 4).p)[:2] == [8, 128]
    assert g3.tune_cache_lookup(path, g3.G3_TUNE_BFS, 20, 5) is None
    assert g3.tune_cache_lookup(path, g3.G3_TUNE_BATCH, 20, 4) is None
    lines = open(path).read().splitlines()
    assert len(lines) == 2 and all(ln.startswith("g3tune1 ") for ln in lines)


def test_cache_skips_malformed_lines_and_last_wins(tmp_path):
    path = tmp_path / "tune.txt"
    path.write_text("garbage\n"
                    "g3tune1 3 11 4 512 0 0 0 0 0 7 2.0 3.0\n"
                    "g3tune1 3 11 4 1024\n"               # truncated
                    "g3tune9 3 11 4 64 0 0 0 0 0 7 2.0 3.0\n"  # unknown tag
                    "g3tune1 3 11 4 256 0 0 0 0 0 7 1.0 3.0\n")
    e = g3.tune_cache_lookup(str(path), g3.G3_TUNE_BATCH, 11, 4)
    assert e.p[0] == 256 and abs(e.ms - 1.0) < 1e-6
    # a store keeps only well-formed entries, one per key
    g3.tune_cache_store(str(path), _entry(g3.G3_TUNE_BATCH, 12, 4, [128]))
    lines = path.read_text().splitlines()
    assert len(lines) == 2
    assert g3.tune_cache_lookup(str(path), g3.G3_TUNE_BATCH, 11, 4).p[0] == 256


def test_cache_errors(tmp_path):
    with pytest.raises(g3.G3Error):
        g3.tune_cache_store(str(tmp_path / "no" / "such" / "dir" / "t.txt"),
                            _entry(g3.G3_TUNE_BFS, 1, 1, [1]))
    with pytest.raises(g3.G3Error):
        g3.tune_cache_store(str(tmp_path / "t.txt"), _entry(9, 1, 1, [1]))
    with pytest.raises(g3.G3Error):
        g3.tune_cache_lookup(None, g3.G3_TUNE_BFS, 1, 1)


def test_learned_controller_options_at_every_size(tmp_path):
    """The trained controller (size-free features) decides the direction at
    every graph size with the margin of its file, and its bin thresholds
    only at the trained sizes; a file trained on another feature set is
    refused."""
    import json
    pytest.importorskip("torch")
    from oracle import mlp
    from paper_2012_10026_gb300 import train_controller as tc
    path = tmp_path / "c.json"
    path.write_text(json.dumps({"params": mlp.init_params(1).tolist(), "mlp_margin": 250,
                                "mlp_bins": 1, "n_bfs_range": [1 << 19, 1 << 23],
                                "features": tc.FEATURES}))
    for nb in [1 << 19, 1 << 21, 1 << 25, (1 << 19) // 2]:
        o, _, note = tc.controller_opts(str(path), nb, device="cpu", alpha=20)
        inside = (1 << 19) <= nb <= (1 << 23)
        assert (o.controller, o.mlp_margin, o.alpha) == (g3.G3_CTRL_LEARNED, 250, 20)
        assert o.mlp_bins == (1 if inside else 0)
        assert ("inside" in note) == inside
    old = tmp_path / "old.json"
    old.write_text(json.dumps({"params": mlp.init_params(1).tolist()}))
    with pytest.raises(ValueError):
        tc.controller_opts(str(old), 1 << 20, device="cpu")


def test_rule_near_is_the_factor_four_band():
    """The levels the controller consults the network on: the rule's test
    strictly within a factor of 4 of its threshold, in integers."""
    from paper_2012_10026_gb300 import train_controller as tc
    # after a top-down level: m_f * 14 against m_u
    assert tc.rule_near(0, 1, 10, 141, 10 ** 6)          # 140 vs 141
    assert not tc.rule_near(0, 1, 10, 560, 10 ** 6)      # exactly 4x: clear
    assert tc.rule_near(0, 1, 10, 559, 10 ** 6)
    assert not tc.rule_near(0, 1, 40, 140, 10 ** 6)      # 560 vs 140: clear
    assert tc.rule_near(0, 1, 40, 141, 10 ** 6)
    # after a bottom-up level: n_f * 24 against n
    assert tc.rule_near(1, 1000, 0, 0, 24000)
    assert not tc.rule_near(1, 250, 0, 0, 24000)         # 6000 * 4 == 24000
    assert not tc.rule_near(1, 4000, 0, 0, 24000)        # 96000 == 4 * 24000
    assert tc.rule_near(1, 3999, 0, 0, 24000)


def test_pick_margin_is_the_widest_with_the_least_regret():
    """The controller's margin: the widest candidate whose held-out regret is
    the smallest reached (ties go to the wider margin, so the rule stands
    where the network is unsure); the rule everywhere when only the infinite
    margin reaches it."""
    from paper_2012_10026_gb300 import train_controller as tc
    ms = tc.MARGINS
    table = {str(m): 0.5 for m in ms}
    table[str(0.1)] = table[str(0.2)] = table[str(0.3)] = 0.1
    assert tc.pick_margin(table) == 0.3
    table = {str(m): 0.2 for m in ms}
    assert tc.pick_margin(table) == max(m for m in ms if m < 1e9)
    table = {str(m): 0.3 for m in ms}
    table[str(1e9)] = 0.1
    assert tc.pick_margin(table) == 1e9
