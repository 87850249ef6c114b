"""The learned prior mean (benchmark addition to Algorithm 1) against the
plain GP under the same rule: both arms' q-GP hyperparameters maximise the
evidence (Sec. 2.3, Eq. evidenceEq) with sigma_n^2 held at the database's
mean squared standard error -- on the flow rates for the plain GP, on the
residuals of the MLP for the learned mean -- so the arms differ only by the
prior mean.  Judged against MD at every section and step, with the thermal
noise of two such runs as the band."""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_mean_cuts_md_runs_within_the_noise_band():
    from paper_1603_04628_gb300 import build, cases, native
    build.build()
    ctx = native.Context(0, native.PREC_FP32)
    params = dict(n_sections=24, dx=400.0, h0=12.0, Lx=10.0, Lz=10.0, eos_K=10.0, eos_n0=0.8, dP_amp=400.0,
                  period=1000.0, dt=20.0, T=1.1, md_steps_eq=2000, md_steps_sample=3000, seed=17, sn2_from_data=0,
                  inputs=0)
    rows, info, net = cases.learned_mean_comparison(ctx, [2.0], 25, db_elements=128, db_seed=23, **params)
    r = rows[0]
    noise = info["noise_error"]
    print(info, r)
    assert r["md_runs_mlp"] < r["md_runs_plain"]
    # the learned-mean hybrid's flow error stays within the thermal-noise band
    assert r["error_mlp"] <= 2.0 * noise, (r["error_mlp"], noise)
    net.close()
    ctx.close()
