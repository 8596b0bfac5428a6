"""GPU MLP kernels (forward, loss/gradient, Adam training, features) against
the float64 oracle of oracle/mlp.py."""
import numpy as np
import pytest

import graphgen
import oracle
from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_10026_gb300 as g3  # noqa: E402


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _data(B, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 3, size=(B, mlp.N_IN)).astype(np.float32)
    y = rng.normal(0, 2, size=(B, mlp.N_OUT)).astype(np.float32)
    return x, y


def test_forward_matches_oracle():
    p = mlp.init_params(7).astype(np.float32)
    x, _ = _data(1000, 1)
    out = g3.g3_mlp_forward(_t(p), _t(x)).cpu().numpy()
    ref = mlp.forward(p.astype(np.float64), x.astype(np.float64))
    assert np.allclose(out, ref, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("B", [1, 31, 257, 4096])
def test_loss_grad_matches_oracle_within_1e4(B):
    p = mlp.init_params(3).astype(np.float32)
    x, y = _data(B, B)
    w = np.array([1.0, 0.1, 0.2, 0.3], np.float32)
    loss, grad = g3.g3_mlp_loss_grad(_t(p), _t(x), _t(y), _t(w))
    rl, rg = mlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64),
                               y.astype(np.float64), w.astype(np.float64))
    g = grad.cpu().numpy()
    assert abs(loss.item() - rl) <= 1e-4 * abs(rl)
    # relative error of the gradient vector, and elementwise with a floor
    assert np.linalg.norm(g - rg) <= 1e-4 * np.linalg.norm(rg)
    assert np.all(np.abs(g - rg) <= 1e-4 * np.maximum(np.abs(rg), np.abs(rg).max() * 1e-2))


def test_loss_grad_is_deterministic():
    p = mlp.init_params(4).astype(np.float32)
    x, y = _data(3000, 9)
    a = g3.g3_mlp_loss_grad(_t(p), _t(x), _t(y))[1].cpu().numpy()
    b = g3.g3_mlp_loss_grad(_t(p), _t(x), _t(y))[1].cpu().numpy()
    assert np.array_equal(a, b)


def test_adam_training_follows_oracle():
    p0 = mlp.init_params(5)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(300, mlp.N_IN)).astype(np.float32)
    y = np.stack([x[:, 0] - x[:, 1], x[:, 2], 0.5 * x[:, 3], np.ones(300)], 1).astype(np.float32)
    pt = _t(p0)
    losses = g3.g3_mlp_train(pt, _t(x), _t(y), steps=30, lr=1e-2).cpu().numpy()
    rp, rlosses = mlp.train_adam(p0, x.astype(np.float64), y.astype(np.float64), 30, lr=1e-2)
    assert np.allclose(losses, rlosses, rtol=2e-3)
    assert np.allclose(pt.cpu().numpy(), rp, atol=2e-3)
    # longer run fits the target
    losses = g3.g3_mlp_train(pt, _t(x), _t(y), steps=1500, lr=1e-2).cpu().numpy()
    assert losses[-1] < 0.05 * rlosses[0]


def test_features_match_oracle_on_real_levels():
    scale, n = 14, 1 << 14
    src, dst = graphgen.kronecker_edges(scale, 16, seed=2)
    g = g3.g3_build_csr(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    g3.g3_rcm_relabel(g)
    nb, nnz = g.info["n_bfs"], g.info["nnz"]
    roots = graphgen.pick_roots(graphgen.nonisolated_flags(src, dst, n), 4, seed=3)
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in roots.tolist():
        st = g3.g3_bfs(g, r, parent, level, max_stats=64)
        x = g3.g3_mlp_features(st, nb, nnz).cpu().numpy()
        for a, row in zip(st, x):
            prev = st[a["level"] - 1]["dir"] if a["level"] > 0 else 0
            pnf = st[a["level"] - 1]["n_f"] if a["level"] > 0 else 0
            ref = mlp.features(a["n_f"], a["m_f"], a["n_u"], a["m_u"], nb, nnz, prev,
                               a["level"], pnf)
            assert np.allclose(row, ref, rtol=1e-5, atol=1e-5)
    g.free()
