"""Pins for the FP64 MLP oracle: GELU against its definition, gradients
against central finite differences of the loss, one Adam step against its
closed form, and a training run that learns a smooth function."""
import math

import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def test_gelu_is_x_times_normal_cdf():
    z = np.linspace(-4, 4, 41)
    np.testing.assert_allclose(mlp.gelu(z), z * norm.cdf(z), rtol=1e-13, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(3)
    X = rng.normal(size=(40, 2))
    y = rng.normal(size=40)
    loss, g = mlp.loss_and_grads(p, X, y)
    h = 1e-6
    for name in mlp.ORDER:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss_and_grads(p, X, y)[0]
            flat[idx] = old - h
            lm = mlp.loss_and_grads(p, X, y)[0]
            flat[idx] = old
            assert g[name].reshape(-1)[idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_first_adam_step_closed_form():
    # at t = 1 the bias-corrected moments are g and g^2, so the step is
    # -lr * g / (|g| + eps) = -lr * sign(g) (up to eps)
    p = {k: np.ones(s) for k, s in mlp.SHAPES.items()}
    g = {k: np.full(s, 0.3) * (1 if i % 2 else -1) for i, (k, s) in enumerate(mlp.SHAPES.items())}
    m = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    v = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    mlp.adam_step(p, g, m, v, 1, lr=0.01)
    for k in mlp.ORDER:
        expect = 1.0 - 0.01 * g[k] / (np.abs(g[k]) + 1e-8)
        np.testing.assert_allclose(p[k], expect, rtol=1e-12)


def test_training_fits_a_smooth_function():
    rng = np.random.default_rng(1)
    X = np.column_stack([rng.uniform(6, 18, 300), rng.uniform(-0.05, 0.05, 300)])
    y = -X[:, 0] ** 2 * X[:, 1] * 4.0
    p, s, losses = mlp.train(X, y, epochs=400, lr=3e-3, seed=2)
    assert losses[-1] < 0.05 * losses[0]
    pred = mlp.predict(p, s, X)
    assert np.sqrt(np.mean((pred - y) ** 2)) < 0.25 * y.std()


def test_adam_moment_recursions_by_hand():
    # Steps 1-3 with beta1 = 0.5, beta2 = 0.75 and gradients 1, -2, 0.5, by
    # hand (Kingma & Ba 2015: m_t = b1 m + (1 - b1) g, v_t = b2 v + (1 - b2) g^2,
    # step -lr m_t / (1 - b1^t) / (sqrt(v_t / (1 - b2^t)) + eps)):
    #   t = 1: m = 1/2,   v = 1/4,     m^ = 1,    v^ = 1
    #   t = 2: m = -3/4,  v = 19/16,   m^ = -1,   v^ = (19/16) / (7/16) = 19/7
    #   t = 3: m = -1/8,  v = 61/64,   m^ = -1/7, v^ = (61/64) / (37/64) = 61/37
    lr, eps = 0.1, 1e-8
    steps = [1.0 / (1.0 + eps), -1.0 / (math.sqrt(19.0 / 7.0) + eps), -1.0 / 7.0 / (math.sqrt(61.0 / 37.0) + eps)]
    p = {k: np.ones(s) for k, s in mlp.SHAPES.items()}
    m = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    v = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    expect = 1.0
    for t, (g, st) in enumerate(zip((1.0, -2.0, 0.5), steps), start=1):
        grads = {k: np.full(s, g) for k, s in mlp.SHAPES.items()}
        mlp.adam_step(p, grads, m, v, t, lr=lr, b1=0.5, b2=0.75, eps=eps)
        expect -= lr * st
        for k in mlp.ORDER:
            np.testing.assert_allclose(p[k], expect, rtol=1e-14)
