"""Pins of the surrogate network's fp64 oracle (oracle/mlp.py) against
values it does not compute: central finite differences of the loss (exact
arithmetic), closed forms of special networks, and the bfloat16 format."""
import numpy as np

from oracle import mlp


def _init(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, mlp.N_PARAMS)


def test_bf16_rounding_matches_the_format():
    # bfloat16 keeps 8 significand bits: 1 + 2^-8 is a tie and rounds to even (1)
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert mlp.bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7
    assert mlp.bf16(-2.5) == -2.5 and mlp.bf16(0.0) == 0.0
    x = np.random.default_rng(1).normal(size=1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= np.abs(x) * 2.0 ** -8 * 1.0001)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    p = _init(3)
    X = rng.normal(size=(7, 3))
    T = rng.normal(size=(7, 4))
    mask = (rng.random((7, 4)) < 0.8).astype(float)
    _, g = mlp.loss_and_grads(p, X, T, mask, rounding=False)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 191, 192, 255, 8575, 8835]])
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[k] = h
        lp, _ = mlp.loss_and_grads(p + e, X, T, mask, rounding=False)
        lm, _ = mlp.loss_and_grads(p - e, X, T, mask, rounding=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 + 1e-5 * abs(fd), (k, fd, g[k])


def test_special_networks():
    X = np.random.default_rng(4).normal(size=(5, 3))
    T = np.random.default_rng(5).normal(size=(5, 4))
    # all weights zero: the output is the last bias; its gradient is the mean residual
    p = np.zeros(mlp.N_PARAMS)
    b4 = np.array([0.5, -1.0, 2.0, 0.25])
    p[-4:] = b4
    y, _ = mlp.forward(p, X, rounding=False)
    assert np.allclose(y, b4)
    loss, g = mlp.loss_and_grads(p, X, T, rounding=False)
    assert np.isclose(loss, ((b4 - T) ** 2).sum() / 20)
    assert np.allclose(g[-4:], 2 * (b4 - T).sum(0) / 20)
    assert np.allclose(g[:-4], 0.0)


def test_adam_first_step_is_sign_times_lr():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    w, m, v = mlp.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(w[:3], -0.01 * np.sign(g[:3]), rtol=1e-4) and w[3] == 0.0
