"""GPU MLP (BF16 tensor-core products, FP32 elsewhere) against the FP64
oracle.  Bounds: forward output and each gradient tensor within 2e-2 of the
reference in relative L2 norm (BF16 keeps 8 significant bits); one Adam step
within 1e-5 relative (FP32 arithmetic on identical inputs)."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu
BF16_TOL = 2e-2


@pytest.fixture(scope="module")
def ctx():
    from paper_1603_04628_gb300 import build, native
    build.build()
    c = native.Context(0, native.PREC_FP64)
    yield c
    c.close()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("n", [1, 63, 64, 65, 1000])
def test_loss_and_gradients_match_oracle(ctx, n):
    from paper_1603_04628_gb300 import native
    rng = np.random.default_rng(n)
    params = omlp.init_params(seed=n)
    # round the reference weights to the FP32 the GPU stores
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in params.items()}
    X = rng.normal(size=(n, 2))
    y = rng.normal(size=n)
    net = native.MLP(ctx, params)
    loss, g = net.loss_grad(X, y)
    loss_ref, g_ref = omlp.loss_and_grads(params, X, y)
    assert loss == pytest.approx(loss_ref, rel=BF16_TOL)
    for k in omlp.ORDER:
        assert _rel(g[k], g_ref[k]) <= BF16_TOL, k
    net.close()


def test_adam_step_matches_oracle(ctx):
    from paper_1603_04628_gb300 import native
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in omlp.init_params(seed=4).items()}
    rng = np.random.default_rng(5)
    grads = {k: rng.normal(size=v.shape).astype(np.float32).astype(np.float64) for k, v in params.items()}
    net = native.MLP(ctx, params)
    ref = {k: v.copy() for k, v in params.items()}
    m = {k: np.zeros_like(v) for k, v in ref.items()}
    v = {k: np.zeros_like(x) for k, x in ref.items()}
    for t in (1, 2, 3):
        net.adam_step(grads, lr=0.01)
        omlp.adam_step(ref, grads, m, v, t, lr=0.01)
    got, _ = net.get()
    for k in omlp.ORDER:
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-5, atol=1e-6)
    net.close()


def test_training_learns_the_flow_law(ctx):
    from paper_1603_04628_gb300 import native
    rng = np.random.default_rng(7)
    X = np.column_stack([rng.uniform(6, 18, 800), rng.uniform(-0.05, 0.05, 800)])
    y = -X[:, 0] ** 2 * X[:, 1] * 4.0 + 0.05 * rng.normal(size=800)
    net = native.MLP(ctx, seed=3)
    train, hold = net.train(X, y, epochs=1500, lr=3e-3, eval_every=25)
    pred = net.predict(X)
    rms = np.sqrt(np.mean((pred - y) ** 2))
    assert hold < 0.05                      # standardised units
    assert rms < 0.25 * y.std()
    # the same network reproduces in the oracle (BF16 forward vs FP64)
    params, st = net.get()
    Xs = (X - st[0:2]) / st[2:4]
    ref = omlp.forward(params, Xs)["out"] * st[5] + st[4]
    assert _rel(pred, ref) <= BF16_TOL
    net.close()
