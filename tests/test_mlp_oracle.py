"""Pins of the FP64 MLP reference: analytic gradient vs central finite differences,
softmax/cross-entropy closed forms, Adam's first step."""
import numpy as np
import pytest

from oracle import mlp


def _data(n=64, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, mlp.N_IN))
    y = rng.integers(0, 3, size=n)
    return X, y


def test_gradient_matches_central_differences():
    X, y = _data()
    th = mlp.init(3)
    w = np.array([1.0, 7.0, 5.0])
    g = mlp.grad(th, X, y, w)
    rng = np.random.default_rng(0)
    h = 1e-3

    def pattern(t):
        _, (_, a1, _, a2, _) = mlp.forward(t, X)
        return np.concatenate([(a1 > 0).ravel(), (a2 > 0).ravel()])
    base = pattern(th)
    checked = 0
    for k in rng.permutation(mlp.N_PARAMS):
        e = np.zeros_like(th)
        e[k] = h
        # central differences are exact to O(h^2) only where no ReLU switches within +-h
        if not (np.array_equal(pattern(th + e), base) and np.array_equal(pattern(th - e), base)):
            continue
        fd = (mlp.loss(th + e, X, y, w) - mlp.loss(th - e, X, y, w)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-8, (k, fd, g[k])
        checked += 1
        if checked == 150:
            break
    assert checked == 150


def test_zero_network_loss_is_log3():
    X, y = _data()
    th = np.zeros(mlp.N_PARAMS)
    assert mlp.loss(th, X, y, [1, 1, 1]) == pytest.approx(np.log(3.0), abs=1e-12)
    # and the output bias gradient is the mean of (1/3 - onehot)
    g = mlp.unpack(mlp.grad(th, X, y, [1, 1, 1]))
    want = (1.0 / 3.0 - np.eye(3)[y]).mean(0)
    np.testing.assert_allclose(g["b3"], want, atol=1e-15)


def test_layer_sizes():
    assert mlp.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 3 * 64 + 3 == 5443


def test_adam_first_step_is_lr_times_sign():
    th = np.zeros(4)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    new, m, v = mlp.adam_step(th, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> lr * g / (|g| + eps)
    np.testing.assert_allclose(new[:3], -0.01 * np.sign(g[:3]), rtol=1e-5)
    assert new[3] == 0.0
