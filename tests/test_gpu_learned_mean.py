"""What the learned prior mean gains: trained on an MD database of the
channel's inputs, the MLP carries the flow law, the residual GP gets a smaller
signal variance, and the hybrid needs fewer MD runs at the same threshold."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_learned_mean_hybrid_needs_fewer_md_runs():
    from paper_1603_04628_gb300 import build, cases, native
    build.build()
    ctx = native.Context(0, native.PREC_FP32)
    sn = 0.5
    X, y, se = cases.md_database(ctx, 96, seed=5, steps_eq=600, steps_sample=1200)
    assert np.isfinite(y).all()
    net, sf_res, info = cases.learned_mean(ctx, X, y, sn, epochs=1500)
    sf_plain = 20 * sn
    assert sf_res < sf_plain
    params = dict(n_sections=24, dx=50.0, h0=12.0, Lx=10.0, Lz=10.0, eos_K=10.0, eos_n0=0.8, dP_amp=48.0,
                  period=300.0, dt=20.0, T=1.1, md_steps_eq=600, md_steps_sample=1200, seed=17, l2=1.0,
                  sn2=sn ** 2, sn2_from_data=0)
    rows = cases.mlp_comparison(ctx, [1.0], 8, net, sf_res, sf_plain, **params)
    r = rows[0]
    print(info, r)
    assert r["md_runs_mlp"] < r["md_runs_plain"]
    net.close()
    ctx.close()
