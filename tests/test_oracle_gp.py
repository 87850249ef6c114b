"""Pins for the dense FP64 GP oracle (oracle/gp.py): closed forms on 1- and
3-point databases, the empty-database case, interpolation as sigma_n -> 0,
and independent library implementations of the posterior and the evidence."""
import math

import numpy as np
import pytest
import scipy.stats

from oracle import gp
from tests.conftest import read_golden


def test_scales_mean_pairwise_separation():
    X = np.array([[0.0, 5.0], [1.0, 5.0], [3.0, 5.0]])
    # pairs along dim 0: |0-1|, |0-3|, |1-3| -> mean 2; dim 1 has no spread -> fallback
    np.testing.assert_allclose(gp.scales(X, fallback=0.7), [2.0, 0.7], rtol=0, atol=0)
    np.testing.assert_allclose(gp.scales(X[:1], fallback=1.0), [1.0, 1.0])
    # per-dimension fallbacks apply only where the separation is undefined
    np.testing.assert_allclose(gp.scales(X, fallback=[0.7, 0.3]), [2.0, 0.3], rtol=0, atol=0)
    np.testing.assert_allclose(gp.scales(X[:1], fallback=[0.7, 0.3]), [0.7, 0.3])


def test_channel_fallback_scales_are_h0_half_and_forcing_gradient():
    from oracle import hybrid
    ch = hybrid.Channel(n_sections=8, dx=50.0, h0=12.0, dP_amp=400.0)
    np.testing.assert_allclose(ch.fallback, [6.0, 400.0 / (8 * 50.0)])
    # the first step's inputs share one G: that dimension takes dP_amp / L
    X = np.column_stack([ch.h, np.full(ch.N, -0.01)])
    d = gp.scales(X, fallback=ch.fallback)
    assert d[1] == pytest.approx(1.0)
    assert d[0] > 0 and d[0] != 6.0


def test_one_point_golden():
    vals = {k: float(v) for k, v in read_golden("gp_one_point.txt")}
    # query at normalised distance 1: put the scale at 1 explicitly
    g = gp.GP(np.array([[0.0]]), np.array([1.0]), 1.0, 1.0, 0.0025, dbar=np.array([1.0]))
    mean, var = g.predict(np.array([[1.0]]))
    assert mean[0] == pytest.approx(vals["mean_coefficient"], rel=1e-11)
    assert var[0] == pytest.approx(vals["variance"], rel=1e-11)


def _inv3(C):
    """3x3 inverse by the adjugate (Cramer's rule)."""
    a, b, c = C[0]
    d, e, f = C[1]
    g, h, i = C[2]
    det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g)
    adj = np.array([[e * i - f * h, c * h - b * i, b * f - c * e],
                    [f * g - d * i, a * i - c * g, c * d - a * f],
                    [d * h - e * g, b * g - a * h, a * e - b * d]])
    return adj / det


def test_three_point_closed_form():
    X = np.array([[6.0, -0.01], [9.0, 0.02], [14.0, 0.0]])
    y = np.array([0.4, -0.9, 0.1])
    sf2, l2, sn2 = 1.7, 0.8, 0.01
    g = gp.GP(X, y, sf2, l2, sn2)
    # scales by hand: dim 0 pairs 3, 8, 5 -> 16/3; dim 1 pairs .03, .01, .02 -> .02
    dbar = np.array([16.0 / 3.0, 0.02])
    np.testing.assert_allclose(g.dbar, dbar, rtol=1e-14)
    Xs = np.array([[7.0, 0.0], [12.0, 0.01], [30.0, 0.5]])

    def k(p, q):
        d2 = (((p - q) / dbar) ** 2).sum()
        return sf2 * math.exp(-d2 / (2 * l2))

    C = np.array([[k(X[i], X[j]) + (sn2 if i == j else 0.0) for j in range(3)] for i in range(3)])
    Ci = _inv3(C)
    mean, var = g.predict(Xs)
    for s in range(3):
        ks = np.array([k(Xs[s], X[j]) for j in range(3)])
        assert mean[s] == pytest.approx(ks @ Ci @ y, rel=1e-11, abs=1e-13)
        assert var[s] == pytest.approx(sf2 - ks @ Ci @ ks, rel=1e-11, abs=1e-13 * sf2)


def test_empty_database_returns_prior():
    g = gp.GP(np.zeros((0, 2)), np.zeros(0), 2.5, 1.0, 0.1, mu=lambda X: 3.0 * X[:, 0])
    mean, var = g.predict(np.array([[1.0, 0.0], [2.0, 1.0]]))
    np.testing.assert_array_equal(mean, [3.0, 6.0])
    np.testing.assert_array_equal(var, [2.5, 2.5])
    # a threshold above sigma_f never asks for MD (paper Sec. 3.1)
    assert not gp.gate(np.sqrt(var), 1.01 * math.sqrt(2.5)).any()


def test_interpolates_as_noise_vanishes():
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, (12, 2))
    y = np.sin(4 * X[:, 0]) + X[:, 1]
    g = gp.GP(X, y, 1.0, 0.3, 1e-10)
    mean, var = g.predict(X)
    np.testing.assert_allclose(mean, y, atol=1e-5)
    assert (var < 1e-6).all()


def test_variance_invariants():
    X, y = np.random.default_rng(3).uniform(0, 1, (20, 3)), np.arange(20.0)
    g = gp.GP(X, y, 1.3, 1.0, 0.02)
    assert np.allclose(g.C, g.C.T)
    assert np.linalg.eigvalsh(g.C).min() > 0
    mean, var = g.predict(np.vstack([X, X + 100.0]))
    assert (var >= 0).all()
    assert (var[:20] <= 0.02 + 1e-12).all()          # at a datum: below the noise variance
    np.testing.assert_allclose(var[20:], 1.3, rtol=1e-12)  # far away: the signal variance


def test_posterior_matches_scikit_learn():
    skl = pytest.importorskip("sklearn.gaussian_process")
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 3, (30, 2))
    y = np.cos(X[:, 0]) * X[:, 1]
    sf2, l2, sn2 = 0.9, 1.2, 0.004
    g = gp.GP(X, y, sf2, l2, sn2)
    Xs = rng.uniform(-1, 4, (17, 2))
    mean, var = g.predict(Xs)
    k = kern.ConstantKernel(sf2, "fixed") * kern.RBF(math.sqrt(l2), "fixed")
    ref = skl.GaussianProcessRegressor(kernel=k, alpha=sn2, optimizer=None, normalize_y=False)
    ref.fit(X / g.dbar, y)
    m2, s2 = ref.predict(Xs / g.dbar, return_std=True)
    np.testing.assert_allclose(mean, m2, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(var, s2 ** 2, rtol=1e-8, atol=1e-10)


def test_evidence_matches_multivariate_normal():
    rng = np.random.default_rng(5)
    X = rng.uniform(0, 1, (15, 2))
    y = rng.normal(size=15)
    g = gp.GP(X, y, 1.1, 0.7, 0.05)
    ref = scipy.stats.multivariate_normal(mean=np.zeros(15), cov=g.C).logpdf(y)
    assert g.log_marginal_likelihood() == pytest.approx(ref, rel=1e-12)


def test_prior_mean_is_added_back():
    rng = np.random.default_rng(6)
    X = rng.uniform(0, 1, (10, 2))
    y = 2.0 + X[:, 0]
    mu = lambda Z: 2.0 + Z[:, 0]
    g = gp.GP(X, y, 1.0, 1.0, 0.01, mu=mu)
    Xs = rng.uniform(0, 1, (5, 2))
    mean, var = g.predict(Xs)
    np.testing.assert_allclose(mean, mu(Xs), atol=1e-14)   # residuals are all zero
    g0 = gp.GP(X, y, 1.0, 1.0, 0.01)
    np.testing.assert_allclose(var, g0.predict(Xs)[1], rtol=1e-14)  # variance ignores mu


def test_gate_is_strict():
    assert list(gp.gate([0.5, 0.5000001, 0.4], 0.5)) == [False, True, False]


def _gp_draw(M, sf2, l2, sn2, seed):
    # inputs in the benchmark's (h, dp/dx) box; outputs drawn from the GP
    # prior with the same normalised squared-exponential covariance
    rng = np.random.default_rng(seed)
    X = np.column_stack([rng.uniform(6.0, 18.0, M), rng.uniform(-0.05, 0.05, M)])
    d = gp.scales(X)
    Z = X / d
    r2 = ((Z[:, None, :] - Z[None, :, :]) ** 2).sum(-1)
    C = sf2 * np.exp(-r2 / (2.0 * l2)) + sn2 * np.eye(M)
    y = np.linalg.cholesky(C) @ rng.standard_normal(M)
    return X, y


def test_optimize_recovers_generating_hyperparameters():
    X, y = _gp_draw(300, 2.0, 0.5, 0.01, seed=3)
    sf2, l2, sn2, f = gp.optimize(X, y, 1.0, 1.0, 0.1)
    assert 0.5 < sf2 / 2.0 < 2.0
    assert 0.5 < l2 / 0.5 < 2.0
    assert 0.5 < sn2 / 0.01 < 2.0
    assert f > gp.GP(X, y, 1.0, 1.0, 0.1).log_marginal_likelihood()


def test_optimize_ends_at_a_coordinate_maximum():
    X, y = _gp_draw(120, 1.0, 1.0, 0.05, seed=4)
    h = list(gp.optimize(X, y, 0.3, 3.0, 0.3)[:3])
    f = gp.GP(X, y, *h).log_marginal_likelihood()
    for k in range(3):
        for fac in (1.1, 1 / 1.1):
            t = list(h)
            t[k] *= fac
            assert gp.GP(X, y, *t).log_marginal_likelihood() <= f + 1e-6 * abs(f)


# ---------------------------------------------------------------- App. B periodic kernel
def test_periodic_kernel_one_point_by_hand():
    # one sample y1 = 2 at t = 0, period T = 4, l = 1, sf2 = 1, sn2 = 0.25: at
    # t = 1 the kernel is exp(-2 sin^2(pi/4)) = exp(-1), so the posterior mean
    # is exp(-1) / 1.25 * 2 and the latent variance 1 - exp(-2) / 1.25
    g = gp.GP(np.array([[0.0]]), np.array([2.0]), 1.0, 1.0, 0.25, period=4.0)
    m, v = g.predict(np.array([[1.0], [4.0], [2.0]]))
    e1 = 0.36787944117144233          # exp(-1)
    assert m[0] == pytest.approx(e1 / 1.25 * 2.0, rel=1e-14)
    assert v[0] == pytest.approx(1.0 - e1 * e1 / 1.25, rel=1e-13)
    # one period later the input is the sample itself; half a period away the
    # kernel is exp(-2 sin^2(pi/2)) = exp(-2)
    assert m[1] == pytest.approx(2.0 / 1.25, rel=1e-13)
    assert m[2] == pytest.approx(0.1353352832366127 / 1.25 * 2.0, rel=1e-13)


def test_periodic_posterior_is_periodic_and_matches_sklearn():
    from sklearn.gaussian_process import GaussianProcessRegressor
    from sklearn.gaussian_process.kernels import ConstantKernel, ExpSineSquared, WhiteKernel
    rng = np.random.default_rng(3)
    T = 7.3
    t = np.sort(rng.uniform(0.0, 3 * T, 60)).reshape(-1, 1)
    y = 1.5 * np.sin(2 * np.pi * t[:, 0] / T) + 0.2 * rng.standard_normal(60)
    sf2, l2, sn2 = 1.7, 0.8, 0.04
    g = gp.GP(t, y, sf2, l2, sn2, period=T)
    ts = np.linspace(0.0, T, 23).reshape(-1, 1)
    m, v = g.predict(ts)
    m2, v2 = g.predict(ts + 2 * T)
    np.testing.assert_allclose(m2, m, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(v2, v, rtol=1e-9, atol=1e-12)
    # scikit-learn's ExpSineSquared is exp(-2 sin^2(pi d / p) / l^2)
    k = ConstantKernel(sf2, "fixed") * ExpSineSquared(math.sqrt(l2), T, "fixed", "fixed") + WhiteKernel(sn2, "fixed")
    sk = GaussianProcessRegressor(kernel=k, optimizer=None, normalize_y=False).fit(t, y)
    ms, ss = sk.predict(ts, return_std=True)
    np.testing.assert_allclose(m, ms, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(v + sn2, ss ** 2, rtol=1e-7, atol=1e-10)   # sklearn adds the white noise


def test_periodic_kernel_long_length_scale_limit():
    # l -> infinity: every pair fully correlated, K = sf2 everywhere, so the
    # posterior mean is the constant sf2 sum(y) / (M sf2 + sn2)
    t = np.array([[0.1], [1.3], [2.9], [4.4]])
    y = np.array([1.0, -0.5, 2.0, 0.25])
    g = gp.GP(t, y, 2.0, 1e12, 0.5, period=5.0)
    m, _ = g.predict(np.array([[0.7], [3.3]]))
    np.testing.assert_allclose(m, 2.0 * y.sum() / (4 * 2.0 + 0.5), rtol=1e-9)


def test_periodic_filter_recovers_a_sinusoid_with_held_signal_variance():
    # App. B procedure: (l2, sn2) by maximum evidence on the samples up to the
    # first peak with sf2 held, then regression over the whole series
    rng = np.random.default_rng(8)
    T = 10.0
    t = np.linspace(0.0, 2 * T, 201)
    truth = 0.8 * np.sin(2 * np.pi * t / T)
    q = truth + 0.15 * rng.standard_normal(len(t))
    mean, var, l2, sn2 = gp.periodic_filter(t, q, T, 1.0, 1.0, 0.01, fit_until=T / 4)
    assert np.sqrt(np.mean((mean - truth) ** 2)) < 0.5 * np.sqrt(np.mean((q - truth) ** 2))
    assert 0.005 < sn2 < 0.1
    # the held signal variance stayed put: the search moved only l2 and sn2
    _, l2b, sn2b, _ = gp.optimize(t[t <= T / 4].reshape(-1, 1), q[t <= T / 4], 1.0, 1.0, 0.01, period=T, hold=1)
    assert (l2b, sn2b) == (l2, sn2)
