"""Pins for the direction rule, the float64 MLP, TEPS arithmetic and the
seeded generators."""
import numpy as np
import pytest

import graphgen
import oracle
from oracle import direction, metrics, mlp
from _graphs import path_graph, star_graph


# ---------------------------------------------------------------- direction
def test_direction_star_from_centre():
    # F_0 = {centre} top-down (Algorithm 2 starts top-down); F_1 = all leaves:
    # m_f = n-1 > m_u/alpha = 0 -> bottom-up.
    n = 10
    off, col = oracle.build_csr(*star_graph(n, 0), n)
    _, level = oracle.bfs(off, col, 0)
    st = direction.level_stats(off, level)
    assert st[0] == dict(n_f=1, m_f=n - 1, n_u=n - 1, m_u=n - 1)
    assert st[1] == dict(n_f=n - 1, m_f=n - 1, n_u=0, m_u=0)
    assert direction.heuristic_directions(off, level) == [0, 1]


def test_direction_path_stays_top_down():
    # path from an end: F_L = {L}, m_f = 2, m_u = 2(n-L-1)-1 -> bottom-up only
    # once 2*alpha > m_u, i.e. near the end of the path.
    n = 100
    off, col = oracle.build_csr(*path_graph(n), n)
    _, level = oracle.bfs(off, col, 0)
    dirs = direction.heuristic_directions(off, level, alpha=14, beta=24)
    # m_u at level L: vertices L+1..n-1, degree 2 except the last (1)
    expect = [0]
    for L in range(1, n):
        m_f = 2 if L < n - 1 else 1
        m_u = 2 * (n - L - 1) - 1 if L < n - 1 else 0
        if expect[-1] == 0:
            expect.append(1 if m_f * 14 > m_u else 0)
        else:
            # n_f = 1 never shrinks below the previous 1 -> stays bottom-up
            expect.append(1)
    assert dirs == expect
    assert dirs.index(1) == next(L for L in range(1, n) if 2 * 14 > 2 * (n - L - 1) - 1)


def test_direction_back_to_top_down_when_shrinking():
    # root 0 - {1..5}, each of 1..5 - 6; n = 7. F_1 = {1..5}: m_f = 10,
    # m_u = 5 -> bottom-up. F_2 = {6} shrank, but n_f * beta < n fails for
    # any beta >= 7, so the search stays bottom-up.
    src = np.array([0, 0, 0, 0, 0, 1, 2, 3, 4, 5], np.int32)
    dst = np.array([1, 2, 3, 4, 5, 6, 6, 6, 6, 6], np.int32)
    off, col = oracle.build_csr(src, dst, 7)
    _, level = oracle.bfs(off, col, 0)
    assert direction.heuristic_directions(off, level, 14, 24) == [0, 1, 1]
    assert direction.heuristic_directions(off, level, 14, 100) == [0, 1, 1]
    # larger graph: hub then a single vertex, n large -> back to TD
    k = 50
    src = np.concatenate([np.zeros(k, np.int32), np.arange(1, k + 1, dtype=np.int32),
                          np.array([k + 1], np.int32)])
    dst = np.concatenate([np.arange(1, k + 1, dtype=np.int32), np.full(k, k + 1, np.int32),
                          np.array([k + 2], np.int32)])
    n = k + 3
    off, col = oracle.build_csr(src, dst, n)
    _, level = oracle.bfs(off, col, 0)
    # F_0={0} TD; F_1 = 50 leaves, m_f=100 > m_u/14 -> BU; F_2={51}: 1 < 50 and
    # 1*24 < 53 -> TD; F_3={52} after TD: m_f = 1, m_u = 0 -> 14 > 0 -> BU.
    assert direction.heuristic_directions(off, level, 14, 24) == [0, 1, 0, 1]


# ---------------------------------------------------------------- MLP
def test_mlp_grad_matches_central_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(1)
    x = rng.normal(size=(17, mlp.N_IN))
    y = rng.normal(size=(17, mlp.N_OUT))
    w = np.array([1.0, 0.5, 0.25, 2.0])
    _, g = mlp.loss_and_grad(p, x, y, w)
    h = 1e-6
    for i in rng.choice(mlp.N_PARAMS, 60, replace=False):
        e = np.zeros_like(p); e[i] = h
        num = (mlp.loss_and_grad(p + e, x, y, w)[0] - mlp.loss_and_grad(p - e, x, y, w)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), i


def test_mlp_closed_forms():
    # all weights zero: output = b2, loss = mean 0.5*sum w (b2 - y)^2,
    # dW1 = db1 = dW2 = 0 (h = 0), db2 = w * mean(b2 - y)
    W1 = np.zeros((mlp.N_HID, mlp.N_IN)); b1 = np.zeros(mlp.N_HID)
    W2 = np.zeros((mlp.N_OUT, mlp.N_HID)); b2 = np.array([1.0, -2.0, 0.5, 3.0])
    p = mlp.pack(W1, b1, W2, b2)
    x = np.ones((4, mlp.N_IN)); y = np.zeros((4, mlp.N_OUT))
    loss, g = mlp.loss_and_grad(p, x, y)
    assert loss == pytest.approx(0.5 * (1 + 4 + 0.25 + 9))
    gW1, gb1, gW2, gb2 = mlp.unpack(g)
    assert not gW1.any() and not gb1.any() and not gW2.any()
    assert np.allclose(gb2, b2)
    # one active hidden unit: h0 = x0 (W1[0,0]=1), o_k = W2[k,0] h0
    W1 = np.zeros((mlp.N_HID, mlp.N_IN)); W1[0, 0] = 1.0
    W2 = np.zeros((mlp.N_OUT, mlp.N_HID)); W2[:, 0] = [2.0, 0, 0, 0]
    p = mlp.pack(W1, np.zeros(mlp.N_HID), W2, np.zeros(mlp.N_OUT))
    x = np.zeros((1, mlp.N_IN)); x[0, 0] = 3.0
    y = np.zeros((1, mlp.N_OUT))
    assert np.allclose(mlp.forward(p, x), [[6.0, 0, 0, 0]])
    loss, g = mlp.loss_and_grad(p, x, y)
    assert loss == pytest.approx(18.0)
    gW1, gb1, gW2, gb2 = mlp.unpack(g)
    assert gW2[0, 0] == pytest.approx(6.0 * 3.0)      # r0 * h0
    assert gW1[0, 0] == pytest.approx(6.0 * 2.0 * 3.0)  # r0 * W2[0,0] * x0
    # ReLU derivative 0 at z <= 0: a negative input kills the gradient
    x[0, 0] = -3.0
    _, g = mlp.loss_and_grad(p, x, y)
    assert not mlp.unpack(g)[0].any()


def test_adam_first_step_is_signed_lr():
    # first Adam step: m_hat = g, v_hat = g^2 -> step = lr * g / (|g| + eps)
    p = mlp.init_params(2)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(8, mlp.N_IN)); y = rng.normal(size=(8, mlp.N_OUT))
    _, g = mlp.loss_and_grad(p, x, y)
    p1, _ = mlp.train_adam(p, x, y, steps=1, lr=0.01)
    expect = p - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1, expect, rtol=0, atol=1e-12)


def test_adam_fits_linear_target():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(64, mlp.N_IN))
    y = np.stack([x[:, 0] - x[:, 1], x[:, 2], 0.5 * x[:, 3], np.ones(64)], 1)
    p, losses = mlp.train_adam(mlp.init_params(3), x, y, steps=1500, lr=1e-2)
    assert losses[-1] < 0.02 * losses[0]


def test_features_closed_form():
    # 8/256, 16/1024, 128/256, (128/8)/8, (16/8)/16, 16/512, 256/(32*16), 1,
    # (512/128)/16, (8/2)/8, 4/32, 128/255
    f = mlp.features(n_f=7, m_f=15, n_u=127, m_u=511, n=255, nnz=1023, prev_dir=1, level=4,
                     prev_nf=1)
    assert np.allclose(f, [-5, -6, -1, 4 / 8, 1 / 16, -5, -1, 1, 2 / 16, 2 / 8, 4 / 32,
                           128 / 255])
    # the same situation on a graph 64 times larger gives the same features:
    # every input is a ratio of the graph's own counts
    g = mlp.features(n_f=7 * 64 + 63, m_f=15 * 64 + 63, n_u=127 * 64 + 63, m_u=511 * 64 + 63,
                     n=255 * 64 + 63, nnz=1023 * 64 + 63, prev_dir=1, level=4,
                     prev_nf=1 * 64 + 63)
    keep = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10]
    assert np.allclose(f[keep], g[keep]) and abs(f[11] - g[11]) < 1e-2
    assert mlp.features(0, 0, 0, 0, 0, 0, 0, 40, 0)[10] == 1.0


# ---------------------------------------------------------------- metrics
def test_teps_arithmetic():
    assert metrics.harmonic_mean_teps([10, 20], [1, 4]) == pytest.approx(2 / (0.1 + 0.2))
    src = np.array([0, 1, 2, 3, 3], np.int32)
    level = np.array([0, 1, -1, 2], np.int32)
    assert metrics.edges_traversed(src, level) == 4
    off = np.array([0, 1, 3, 3, 4])
    assert metrics.unique_edges_traversed(off, level) == 2


# ---------------------------------------------------------------- generators
def test_kronecker_deterministic_and_chunked():
    a = graphgen.kronecker_edges(12, 16, seed=1)
    b = graphgen.kronecker_edges(12, 16, seed=1)
    c = graphgen.kronecker_edges(12, 16, seed=2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    part = graphgen.kronecker_edges(12, 16, seed=1, e0=1000, count=500)
    assert np.array_equal(part[0], a[0][1000:1500]) and np.array_equal(part[1], a[1][1000:1500])
    assert a[0].min() >= 0 and a[0].max() < 4096


def test_kronecker_self_loop_rate():
    # both endpoint bits agree with probability A + D = 0.62 per level, so a
    # tuple is a self-loop with probability 0.62^scale (relabelling keeps it)
    scale, ef = 8, 64
    src, dst = graphgen.kronecker_edges(scale, ef, seed=11)
    m = ef << scale
    p = 0.62 ** scale
    mu, sd = m * p, np.sqrt(m * p * (1 - p))
    assert abs(int((src == dst).sum()) - mu) < 4 * sd


def test_kronecker_quadrant_frequencies_at_scale_one():
    # scale 1: the tuple is the quadrant itself, relabelled by a bijection on
    # {0, 1}; quadrant frequencies must match (A, B, C, D) within 4 sigma
    m = 1 << 16
    src, dst = graphgen.kronecker_edges(1, m >> 1, seed=5)
    inv = {graphgen.perm_value(5, 2, x): x for x in (0, 1)}
    u = np.array([inv[x] for x in src[:4096]]); v = np.array([inv[x] for x in dst[:4096]])
    counts = np.array([np.sum((u == a) & (v == b)) for a, b in ((0, 0), (0, 1), (1, 0), (1, 1))])
    probs = np.array([0.57, 0.19, 0.19, 0.05])
    sd = np.sqrt(4096 * probs * (1 - probs))
    assert np.all(np.abs(counts - 4096 * probs) < 4 * sd), counts


@pytest.mark.parametrize("n", [1 << 10, 1000, 7])
def test_perm_is_bijection(n):
    vals = [graphgen.perm_value(9, n, x) for x in range(n)]
    assert sorted(vals) == list(range(n))


def test_chunglu_table_and_edges():
    n = 1 << 14
    w = graphgen.chunglu_weights(n)
    assert w.mean() == pytest.approx(20.0, rel=1e-9)
    assert w.max() <= 2 ** 16 and np.all(np.diff(w) <= 0)
    cum = graphgen.chunglu_table(n)
    assert np.all(np.diff(cum.astype(np.float64)) >= 0)
    src, dst = graphgen.chunglu_edges(n, seed=3)
    assert len(src) == n * 10
    # endpoint frequencies follow w: relabelled vertex perm(0) has weight w0
    v0 = graphgen.perm_value(3, n, 0)
    cnt = int((src == v0).sum() + (dst == v0).sum())
    exp = 2 * len(src) * w[0] / w.sum()
    assert abs(cnt - exp) < 5 * np.sqrt(exp)


def test_roots_uniform_non_isolated_distinct():
    src, dst = graphgen.kronecker_edges(10, 16, seed=1)
    flags = graphgen.nonisolated_flags(src, dst, 1 << 10)
    r = graphgen.pick_roots(flags, 64, seed=2)
    assert len(r) == 64 and len(set(r.tolist())) == 64 and np.all(flags[r] == 1)
    assert np.array_equal(r, graphgen.pick_roots(flags, 64, seed=2))
    few = np.zeros(50, np.uint8); few[[3, 7]] = 1
    assert sorted(graphgen.pick_roots(few, 64, seed=1).tolist()) == [3, 7]


def test_small_graph_specs():
    specs = graphgen.small_graph_specs(4096, seed=5)
    scales = np.array([s for s, _ in specs])
    assert scales.min() == 8 and scales.max() == 14
    assert specs[3][1] == 5 * (1 << 20) + 3
    counts = np.bincount(scales - 8, minlength=7)
    assert np.all(np.abs(counts - 4096 / 7) < 4 * np.sqrt(4096 / 7))
