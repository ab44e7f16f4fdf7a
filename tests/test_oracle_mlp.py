"""Pins for the float64 scheduling-MLP reference (oracle/mlp.py)."""
import numpy as np
import pytest

from oracle import mlp
from paper_2412_19420_gb300 import datagen


def _data(B=17, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, 8))
    t = np.stack([rng.normal(3.0, 2.0, B), (rng.random(B) < 0.4).astype(float)], 1)
    return x, t


def test_param_count():
    assert mlp.N_PARAMS == 4866
    assert datagen.mlp_init_weights(0).shape == (4866,)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    p = datagen.mlp_init_weights(seed).astype(np.float64)
    p += np.random.default_rng(seed).normal(0, 0.05, p.shape)  # non-zero biases
    x, t = _data(seed=seed)
    _, g = mlp.loss_and_grad(p, x, t)
    rng = np.random.default_rng(100 + seed)
    idx = rng.choice(mlp.N_PARAMS, 300, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(mlp.forward(p + e, x)[0], t) - mlp.loss(mlp.forward(p - e, x)[0], t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_network_closed_form():
    # all parameters zero: y = 0, loss = mean(0.5 t0^2) + log 2 - 0,
    # only b3 has a gradient: (mean(-t0), mean(1/2 - t1))
    p = np.zeros(mlp.N_PARAMS)
    x, t = _data()
    y, _ = mlp.forward(p, x)
    assert np.all(y == 0)
    L, g = mlp.loss_and_grad(p, x, t)
    assert L == pytest.approx(np.mean(0.5 * t[:, 0] ** 2) + np.log(2.0), rel=1e-14)
    assert np.all(g[:-2] == 0)
    assert g[-2] == pytest.approx(-np.mean(t[:, 0]), rel=1e-14)
    assert g[-1] == pytest.approx(np.mean(0.5 - t[:, 1]), rel=1e-14)


def test_positive_regime_is_a_matrix_product():
    # with every pre-activation positive the network is y = W3 W2 W1 x + (...)
    rng = np.random.default_rng(3)
    parts = [np.abs(rng.normal(size=s)) for s in mlp.SHAPES]
    p = mlp.join(parts)
    x = np.abs(rng.normal(size=(5, 8)))
    W1, b1, W2, b2, W3, b3 = parts
    want = ((x @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    assert np.allclose(mlp.forward(p, x)[0], want, rtol=1e-13)


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    assert np.allclose(p[:3], -0.01 * np.sign(g[:3]), rtol=1e-4)
    assert p[3] == 0.0


def test_training_reduces_loss():
    p = datagen.mlp_init_weights(1).astype(np.float64)
    x, t = _data(B=64, seed=5)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = mlp.loss(mlp.forward(p, x)[0], t)
    for s in range(1, 201):
        _, g = mlp.loss_and_grad(p, x, t)
        p, m, v = mlp.adam_step(p, g, m, v, s, 1e-2)
    assert mlp.loss(mlp.forward(p, x)[0], t) < 0.3 * L0
