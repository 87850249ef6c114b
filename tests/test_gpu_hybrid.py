"""Algorithm 1 on the GPU (batched gate, one MD launch per step) against the
oracle's literal sequential Algorithm 1 with the oracle's MD.  FP64 forces
and short MD runs keep the two trajectories equal to rounding, so every gate
decision must agree and the flow rates and densities must match closely."""
import numpy as np
import pytest

from oracle import hybrid as ohy
from oracle import md as omd

pytestmark = pytest.mark.gpu

CASE = dict(n_sections=8, dx=50.0, h0=12.0, Lx=10.0, Lz=10.0, K=10.0, n0=0.8, dP_amp=8.0, period=400.0,
            dt=20.0, T=1.1, steps_eq=20, steps_sample=40, seed=11, sf2=4.0, l2=1.0, sn2_default=0.25)


def gpu_params(c):
    return dict(n_sections=c["n_sections"], dx=c["dx"], h0=c["h0"], Lx=c["Lx"], Lz=c["Lz"], eos_K=c["K"],
                eos_n0=c["n0"], dP_amp=c["dP_amp"], period=c["period"], dt=c["dt"], T=c["T"],
                md_steps_eq=c["steps_eq"], md_steps_sample=c["steps_sample"], seed=c["seed"], sf2=c["sf2"],
                l2=c["l2"], sn2=c["sn2_default"], sn2_from_data=0)


def oracle_md(el):
    return omd.element(omd.make_params(el))


# cache_mb -1 keeps none of the gate's factors, so every run of non-MD
# sections takes its means from a refit of the same inputs
@pytest.mark.parametrize("sigma_t,cache_mb", [(0.5, 0), (1.2, 0), (0.5, -1)])
def test_hybrid_steps_match_sequential_oracle(sigma_t, cache_mb):
    from paper_1603_04628_gb300 import build, native
    build.build()
    ctx = native.Context(0, native.PREC_FP64)
    hy = native.Hybrid(ctx, factor_cache_mb=cache_mb, **gpu_params(CASE))
    ref = ohy.Channel(**CASE)
    total = 0
    for step in range(4):
        st = hy.step(sigma_t)
        r = ref.step_sequential(sigma_t, oracle_md)
        s = hy.state()
        assert (s["from_md"] == r["from_md"]).all(), step
        np.testing.assert_allclose(s["G"], r["G"], rtol=1e-9, atol=1e-14)
        np.testing.assert_allclose(s["sd"], r["sd"], rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose(s["q"], r["q"], rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(s["density"], ref.n, rtol=1e-9)
        assert st["md_runs"] == r["from_md"].sum()
        total += st["md_runs"]
    X, y, se = hy.database()
    np.testing.assert_allclose(X, ref.X, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(y, ref.y, rtol=1e-6, atol=1e-8)
    assert total == ref.md_calls > 0
    hy.close()
    ctx.close()


def test_learned_mean_leaves_gate_unchanged():
    # Eq. predVarEq: the prior mean does not enter the variance, so from the
    # same state the same MD sections are chosen; only the means move (and
    # with them the densities, so later steps see different inputs)
    from paper_1603_04628_gb300 import native
    ctx = native.Context(0, native.PREC_FP64)
    a = native.Hybrid(ctx, **gpu_params(CASE))
    b = native.Hybrid(ctx, **gpu_params(CASE))
    b.set_mean(lambda X: -0.5 * X[:, 0] ** 2 * X[:, 1] + 0.3)
    a.step(0.8)
    b.step(0.8)
    sa, sb = a.state(), b.state()
    assert sa["from_md"].any() and not sa["from_md"].all()
    assert (sa["from_md"] == sb["from_md"]).all()
    np.testing.assert_allclose(sa["sd"], sb["sd"], rtol=1e-12)
    gp_only = ~sa["from_md"]
    assert np.abs(sb["q"] - sa["q"])[gp_only].max() > 0.05    # the mean moved the predictions
    a.close(); b.close(); ctx.close()


def test_paper_inputs_with_pressure_gp_match_sequential_oracle():
    # the paper's form (Sec. 2.4): q-GP on (h, n, F), pressure from a p-GP on
    # pre-simulation data; the same decisions and values as the sequential
    # oracle with the same pressure database
    from paper_1603_04628_gb300 import native
    hs = np.linspace(6.0, 18.0, 4)
    ns = np.linspace(0.6, 1.0, 5)
    Xp = np.array([[h, n] for h in hs for n in ns])
    yp = 10.0 * (Xp[:, 1] - 0.8) + 0.02 * np.cos(5.0 * Xp[:, 0] + 17.0 * Xp[:, 1])
    pdb = (Xp, yp, 1.0, 1.0, 1e-4)
    ctx = native.Context(0, native.PREC_FP64)
    hy = native.Hybrid(ctx, inputs=1, **gpu_params(CASE))
    hy.set_pressure(Xp, yp, 1.0, 1.0, 1e-4)
    ref = ohy.Channel(inputs=1, pressure_db=pdb, **CASE)
    for step in range(3):
        hy.step(0.5)
        r = ref.step_sequential(0.5, oracle_md)
        s = hy.state()
        assert (s["from_md"] == r["from_md"]).all(), step
        np.testing.assert_allclose(s["G"], r["G"], rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(s["sd"], r["sd"], rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose(s["q"], r["q"], rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(s["density"], ref.n, rtol=1e-9)
    X, y, se = hy.database()
    assert X.shape[1] == 3 and len(y) == ref.md_calls > 0
    np.testing.assert_allclose(X, ref.X, rtol=1e-8, atol=1e-12)
    hy.close()
    ctx.close()
