"""Float64 oracle of the 12-32-4 MLP direction/binning controller --
TEST INFRASTRUCTURE ONLY.

The paper has no learned part; this restates the network the library trains
(ReLU hidden layer of 32 units, 4 linear outputs) in plain numpy float64:
forward, loss, backward and the Adam update (Kingma and Ba, ICLR 2015).

Loss over a batch of B samples with per-output weights w_k:
    L = 1/(2B) * sum_b sum_k w_k (o_bk - y_bk)^2
ReLU derivative is taken as 0 at z == 0.

Features of a level (inputs), from the frontier sizes and degree sums of the
searched graph (n vertices, nnz directed entries):
    0 log2((1+n_f)/(1+n))    1 log2((1+m_f)/(1+nnz))
    2 log2((1+n_u)/(1+n))    3 log2((1+n_u)/(1+n_f)) / 8 (unvisited
      vertices per frontier vertex)
    4 log2((1+m_f)/(1+n_f)) / 16 (mean frontier degree)
    5 log2((1+m_f)/(1+m_u))  6 log2((1+n) / (32 (1+m_f)))
    7 previous direction (0 TD, 1 BU)
    8 log2((1+m_u)/(1+n_u)) / 16 (mean unvisited degree)
    9 log2((1+n_f)/(1+n_f of the previous level)) / 8 (frontier growth)
   10 min(level, 32) / 32   11 1 - n_u / n (fraction visited)
Outputs: o0 ~ ln(t_BU / t_TD) (bottom-up when o0 < 0), o1..o3 ~ log2 of the
top-down bin thresholds T1 < T2 < T3.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 12, 32, 4
N_PARAMS = N_HID * N_IN + N_HID + N_OUT * N_HID + N_OUT  # 548


def unpack(p):
    p = np.asarray(p, np.float64)
    i = 0
    W1 = p[i:i + N_HID * N_IN].reshape(N_HID, N_IN); i += N_HID * N_IN
    b1 = p[i:i + N_HID]; i += N_HID
    W2 = p[i:i + N_OUT * N_HID].reshape(N_OUT, N_HID); i += N_OUT * N_HID
    b2 = p[i:i + N_OUT]
    return W1, b1, W2, b2


def pack(W1, b1, W2, b2):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2]).astype(np.float64)


def init_params(seed: int = 0):
    """Seeded initial parameters (He-uniform); passed to both sides as input."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (N_HID, N_IN)) * np.sqrt(6.0 / N_IN)
    W2 = rng.uniform(-1, 1, (N_OUT, N_HID)) * np.sqrt(6.0 / N_HID)
    return pack(W1, np.zeros(N_HID), W2, np.zeros(N_OUT))


def forward(p, x):
    W1, b1, W2, b2 = unpack(p)
    x = np.asarray(x, np.float64)
    z = x @ W1.T + b1
    h = np.maximum(z, 0.0)
    return h @ W2.T + b2


def loss_and_grad(p, x, y, w=None):
    W1, b1, W2, b2 = unpack(p)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    B = x.shape[0]
    w = np.ones(N_OUT) if w is None else np.asarray(w, np.float64)
    z = x @ W1.T + b1
    h = np.maximum(z, 0.0)
    o = h @ W2.T + b2
    r = o - y
    loss = 0.5 * np.sum(w * r * r) / B
    go = w * r / B
    dW2 = go.T @ h
    db2 = go.sum(0)
    gh = go @ W2
    gz = gh * (z > 0)
    dW1 = gz.T @ x
    db1 = gz.sum(0)
    return loss, pack(dW1, db1, dW2, db2)


def train_adam(p, x, y, steps: int, lr: float = 1e-2, w=None, beta1: float = 0.9,
               beta2: float = 0.999, eps: float = 1e-8):
    """Full-batch Adam for `steps` steps; returns (params, losses)."""
    p = np.array(p, np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for t in range(1, steps + 1):
        loss, g = loss_and_grad(p, x, y, w)
        losses.append(loss)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p = p - lr * mh / (np.sqrt(vh) + eps)
    return p, np.array(losses)


def features(n_f, m_f, n_u, m_u, n, nnz, prev_dir, level, prev_nf):
    """Feature vector of one level (see the module docstring)."""
    return np.array([
        np.log2((1.0 + n_f) / (1.0 + n)), np.log2((1.0 + m_f) / (1.0 + nnz)),
        np.log2((1.0 + n_u) / (1.0 + n)), np.log2((1.0 + n_u) / (1.0 + n_f)) / 8.0,
        np.log2((1.0 + m_f) / (1.0 + n_f)) / 16.0, np.log2((1.0 + m_f) / (1.0 + m_u)),
        np.log2((1.0 + n) / (32.0 * (1.0 + m_f))), float(prev_dir),
        np.log2((1.0 + m_u) / (1.0 + n_u)) / 16.0,
        np.log2((1.0 + n_f) / (1.0 + prev_nf)) / 8.0, min(level, 32) / 32.0,
        (1.0 - n_u / n) if n > 0 else 0.0,
    ], dtype=np.float64)
