"""FP64 reference of the learned prior mean: an MLP 2 -> 64 -> 64 -> 1 with
exact (erf) GELU, mean-squared-error loss and Adam.

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and bench.py's CPU-baseline
leg may import this module; the product package never does.

The paper's GP has a zero prior mean (Sec. 2.2, Eq. GPEq with mu = 0); the
learned mean is the benchmark's addition: the GP then models y - mu(x).
Readings (the benchmark is silent on them): inputs and output standardised
with the training set's mean and standard deviation; exact erf GELU; Adam with
beta = (0.9, 0.999), eps = 1e-8; full-batch steps.

Parameters are a dict of arrays: W1 (64 x 2), b1 (64), W2 (64 x 64), b2 (64),
W3 (1 x 64), b3 (1); a layer computes z = a W^T + b.
"""
import math

import numpy as np
from scipy.special import erf

SHAPES = {"W1": (64, 2), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (1, 64), "b3": (1,)}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3"]


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    # d/dz [z Phi(z)] = Phi(z) + z phi(z)
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    p = {}
    for name in ORDER:
        shp = SHAPES[name]
        fan_in = SHAPES["W" + name[1]][1]
        bound = 1.0 / math.sqrt(fan_in)
        p[name] = rng.uniform(-bound, bound, shp)
    return p


def forward(p, X):
    """Activations of every layer for the standardised inputs X (n x 2)."""
    z1 = X @ p["W1"].T + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = gelu(z2)
    out = a2 @ p["W3"].T + p["b3"]
    return dict(X=X, z1=z1, a1=a1, z2=z2, a2=a2, out=out[:, 0])


def loss_and_grads(p, X, y):
    """Mean squared error (1/n) sum (out - y)^2 and its gradients by the
    chain rule, layer by layer."""
    c = forward(p, X)
    n = len(y)
    r = c["out"] - y
    loss = float((r * r).mean())
    d_out = (2.0 / n) * r[:, None]                 # n x 1
    g = {}
    g["W3"] = d_out.T @ c["a2"]                    # 1 x 64
    g["b3"] = d_out.sum(axis=0)
    d_a2 = d_out @ p["W3"]                         # n x 64
    d_z2 = d_a2 * gelu_grad(c["z2"])
    g["W2"] = d_z2.T @ c["a1"]                     # 64 x 64
    g["b2"] = d_z2.sum(axis=0)
    d_a1 = d_z2 @ p["W2"]
    d_z1 = d_a1 * gelu_grad(c["z1"])
    g["W1"] = d_z1.T @ c["X"]                      # 64 x 2
    g["b1"] = d_z1.sum(axis=0)
    return loss, g


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of every parameter; t counts from 1."""
    for k in ORDER:
        m[k] = b1 * m[k] + (1.0 - b1) * g[k]
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k]
        mh = m[k] / (1.0 - b1 ** t)
        vh = v[k] / (1.0 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


class Standardiser:
    def __init__(self, X, y):
        self.xm = X.mean(axis=0)
        self.xs = X.std(axis=0)
        self.xs[self.xs == 0] = 1.0
        self.ym = float(y.mean())
        self.ys = float(y.std()) or 1.0

    def x(self, X):
        return (X - self.xm) / self.xs

    def y(self, y):
        return (y - self.ym) / self.ys

    def y_back(self, z):
        return z * self.ys + self.ym


def train(X, y, epochs=500, lr=1e-3, seed=0):
    """Full-batch Adam on standardised data; returns (params, standardiser, losses)."""
    s = Standardiser(X, y)
    Xs, ys = s.x(X), s.y(y)
    p = init_params(seed)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    losses = []
    for t in range(1, epochs + 1):
        loss, g = loss_and_grads(p, Xs, ys)
        losses.append(loss)
        adam_step(p, g, m, v, t, lr)
    return p, s, losses


def predict(p, s, X):
    return s.y_back(forward(p, s.x(X))["out"])
