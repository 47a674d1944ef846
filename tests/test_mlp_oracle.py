"""Pins of the FP64 warm-start network reference (oracle/mlp.py) against what
the mathematics fixes: finite differences of the loss, closed forms of gelu,
of the first Adam step and of the loss at uniform logits, and the features on
a hand-checked example."""
import math

import numpy as np
import pytest

import datagen
from oracle import mlp


def _toy(seed, n=12):
    rng = np.random.default_rng(seed)
    F = rng.normal(size=(n, mlp.IN))
    labels = rng.integers(0, 3, n).astype(np.int32)
    cw = np.array([0.5, 3.0, 1.5])
    theta = datagen.mlp_init(seed).astype(np.float64)
    theta[-3:] = rng.normal(size=3) * 0.1          # nonzero output bias
    return theta, F, labels, cw


def test_parameter_count_and_layout():
    assert mlp.NPARAM == 132 * 256 + 256 + 256 * 256 + 256 + 256 * 3 + 3 == 100611
    theta = datagen.mlp_init(0)
    assert theta.shape == (mlp.NPARAM,) and theta.dtype == np.float32
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(theta)), theta.astype(np.float64))


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    theta, F, labels, cw = _toy(seed)
    g = mlp.grad(theta, F, labels, cw)
    rng = np.random.default_rng(100 + seed)
    # every block of the layout is sampled (weights and biases of each layer)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SIZES])
    idx = np.concatenate([rng.choice(np.arange(offs[k], offs[k + 1]), size=min(24, offs[k + 1] - offs[k]),
                                     replace=False) for k in range(len(mlp.SIZES))])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, F, labels, cw) - mlp.loss(tm, F, labels, cw)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, g[i])


def test_gelu_closed_forms():
    x = np.linspace(-6, 6, 121)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)   # x Phi(x) + x Phi(-x) = x
    assert mlp.gelu(0.0) == 0.0
    np.testing.assert_allclose(mlp.gelu(np.array([30.0])), [30.0])
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_prime(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)
    assert mlp.gelu_prime(0.0) == pytest.approx(0.5)


def test_loss_at_uniform_logits_is_log3():
    theta, F, labels, cw = _toy(3)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta)
    theta0 = mlp.pack([W1, b1, W2, b2, 0 * W3, 0 * b3])
    assert mlp.loss(theta0, F, labels, cw) == pytest.approx(np.mean(cw[labels]) * math.log(3.0), rel=1e-14)


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(5)
    th, g = rng.normal(size=50), rng.normal(size=50)
    t1, m, v = mlp.adam_step(th, np.zeros(50), np.zeros(50), g, 1, 1e-3, eps=1e-8)
    np.testing.assert_allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # decoupled decay: the first step moves by lr (sign-like step + wd theta)
    t2, _, _ = mlp.adam_step(th, np.zeros(50), np.zeros(50), g, 1, 1e-3, eps=1e-8, wd=0.01)
    np.testing.assert_allclose(t2, th - 1e-3 * (g / (np.abs(g) + 1e-8) + 0.01 * th), rtol=1e-12)
    # second step with a constant gradient: m_hat = g, v_hat = g^2 again
    t3, _, _ = mlp.adam_step(t1, *mlp.adam_step(th, np.zeros(50), np.zeros(50), g, 1, 1e-3)[1:], g, 2, 1e-3)
    np.testing.assert_allclose(t3, th - 2e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_features_hand_example():
    X = np.array([[1.0, 0.0], [3.0, 0.0], [-1.0, 0.0], [-3.0, 0.0]])
    y = np.array([1, 1, -1, -1], np.int8)
    F = mlp.features(X, y, 10.0)
    # mu+ = (2, 0), mu- = (-2, 0): w = (4, 0), b = 0; margins y (w.x + b)/|w|
    # columns: x (q = 2), y, |x|/sqrt(q), margin, log10 C
    np.testing.assert_allclose(F[:, 2], [1, 1, -1, -1])
    np.testing.assert_allclose(F[:, 3], [1 / math.sqrt(2), 3 / math.sqrt(2)] * 2)
    np.testing.assert_allclose(F[:, 4], [1, 3, 1, 3])
    np.testing.assert_allclose(F[:, 5], 1.0)


def test_classes_and_start_point():
    C = 0.5
    np.testing.assert_array_equal(mlp.classes_of([0.0, 0.2, 0.5, 0.5 - 1e-12], C), [0, 1, 2, 1])
    logits = np.array([[3, 0, 0], [0, 3, 0], [0, 0, 3]], float)
    np.testing.assert_array_equal(mlp.start_point(logits, C), [0.0, 0.25, 0.5])


def test_warm_instance_recipe():
    X, y, C = datagen.warm_instance(3, n=2000)
    assert X.shape == (2000, 128) and X.dtype == np.float32
    assert 0.01 <= C <= 10.0 and set(np.unique(y)) == {-1, 1}
