"""Float64 reference of the scheduling MLP -- TEST INFRASTRUCTURE ONLY.

The paper names deep-learning models as a direction for choosing the Boolean
operation sequence from data characteristics (Section I, adaptive strategy;
Section V, future work) but specifies no network.  The miner's learned
scheduler fixes one:

    h1 = relu(W1 x + b1)      W1: 64x8,  b1: 64
    h2 = relu(W2 h1 + b2)     W2: 64x64, b2: 64
    y  = W3 h2 + b3           W3: 2x64,  b3: 2
    y[0] predicts log2(1 + subtree work), y[1] is the logit of "store as diffset"

    loss = mean_b [ 0.5 (y0 - t0)^2 + softplus(y1) - t1 * y1 ]

Parameters in the order W1, b1, W2, b2, W3, b3 (4,866 values).  Adam uses the
usual bias-corrected first and second moments (Kingma & Ba 2015).
Parity: pinned by central finite differences and closed forms in
tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

SHAPES = [(64, 8), (64,), (64, 64), (64,), (2, 64), (2,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def split(flat: np.ndarray) -> list[np.ndarray]:
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(flat[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def join(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def forward(params: np.ndarray, x: np.ndarray):
    """x: [B, 8] -> (y [B, 2], cache)."""
    W1, b1, W2, b2, W3, b3 = split(params)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (x, z1, h1, z2, h2)


def loss(y: np.ndarray, t: np.ndarray) -> float:
    y = np.asarray(y, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    sq = 0.5 * (y[:, 0] - t[:, 0]) ** 2
    z = y[:, 1]
    bce = np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z))) - t[:, 1] * z
    return float(np.mean(sq + bce))


def backward(params: np.ndarray, cache, y: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Gradient of ``loss`` with respect to the flat parameter vector."""
    W1, b1, W2, b2, W3, b3 = split(params)
    x, z1, h1, z2, h2 = cache
    B = y.shape[0]
    t = np.asarray(t, dtype=np.float64)
    dy = np.empty_like(y)
    dy[:, 0] = (y[:, 0] - t[:, 0]) / B
    dy[:, 1] = (1.0 / (1.0 + np.exp(-y[:, 1])) - t[:, 1]) / B
    dW3 = dy.T @ h2
    db3 = dy.sum(0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    dW1 = dz1.T @ x
    db1 = dz1.sum(0)
    return join([dW1, db1, dW2, db2, dW3, db3])


def loss_and_grad(params, x, t):
    y, cache = forward(params, x)
    return loss(y, t), backward(params, cache, y, t)


def adam_step(params, grad, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; ``step`` counts from 1.  Returns (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v

