"""Warm starts (paper Sec. 2.4, Algorithm 1): an MD run that starts from the
final snapshot of an earlier run, adapted to the new element, through the C
ABI (mdgp_micro_plan_from) and inside the hybrid (warm_start)."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    from paper_1603_04628_gb300 import build, native as nat
    build.build()
    return nat


def _snapshot(ctx, el):
    ctx.micro_plan([el])
    ctx.micro_launch()
    r = ctx.micro_results()[0]
    x, v = ctx.micro_state()
    return dict(xv=np.hstack([x, v]).astype(np.float32), n_fluid=r["n_fluid"], n_wall=r["n_wall"],
                h=el["h"], Lx=el["Lx"], Lz=el["Lz"])


def _min_image(d, Lx, Lz):
    d = d.copy()
    d[..., 0] -= Lx * np.round(d[..., 0] / Lx)
    d[..., 2] -= Lz * np.round(d[..., 2] / Lz)
    return d


def test_start_state_from_a_snapshot(native):
    # the device starts from the state the host prepares (mdgp_start_state):
    # denser (atoms inserted), sparser (atoms removed), and a cold start for
    # another channel height
    ctx = native.Context(0, native.PREC_FP64)
    base = synth.element_plain(steps_eq=200, steps_sample=0)
    snap = _snapshot(ctx, base)
    nf0 = snap["n_fluid"]
    for density, more in ((0.84, True), (0.76, False)):
        el = dict(base, density=density, steps_eq=0, steps_sample=0, id=77)
        want, kind = native.start_state(el, snap)
        assert kind == 1
        ctx.micro_plan_from([el], [snap])
        ctx.micro_launch()
        r = ctx.micro_results()[0]
        x, v = ctx.micro_state()
        assert r["start"] == 1 and (r["n_fluid"] > nf0) == more and r["n_fluid"] != nf0
        assert len(x) == len(want)
        d = _min_image(x - want[:, :3], el["Lx"], el["Lz"])
        assert np.abs(d).max() < 1e-9
        np.testing.assert_allclose(v, want[:, 3:], rtol=0, atol=1e-12)
    # another height or lateral box cannot take the snapshot: the lattice
    for el in (dict(base, h=base["h"] * 1.1, steps_eq=0, steps_sample=0),
               dict(base, Lx=base["Lx"] + 1.0, steps_eq=0, steps_sample=0)):
        ctx.micro_plan_from([el], [snap])
        ctx.micro_launch()
        assert ctx.micro_results()[0]["start"] == 0
        x_warm, _ = ctx.micro_state()
        ctx.micro_plan([el])
        ctx.micro_launch()
        x_cold, _ = ctx.micro_state()
        np.testing.assert_array_equal(x_warm, x_cold)
    ctx.close()


def test_warm_started_flow_rate_matches_a_cold_ensemble(native):
    # sixteen driven runs from the lattice (2000 + 3000 steps) against sixteen
    # started from the final snapshots of runs at the same height and other
    # densities (half denser: atoms removed; half sparser: atoms inserted),
    # equilibrated for 500 steps only: the mean flow rates, temperatures and
    # pressures agree within two combined standard errors
    ctx = native.Context(0, native.PREC_FP32)
    src = [synth.element_plain(seed=600 + k, g=0.05, elem_id=k, steps_eq=1500, steps_sample=0) for k in range(16)]
    src = [dict(e, density=e["density"] + (0.02 if k % 2 else -0.02)) for k, e in enumerate(src)]
    ctx.micro_plan(src)
    ctx.micro_launch()
    rs = ctx.micro_results()
    x, v = ctx.micro_state()
    snaps, off = [], 0
    for e, r in zip(src, rs):
        m = r["n_fluid"] + r["n_wall"]
        snaps.append(dict(xv=np.hstack([x[off:off + m], v[off:off + m]]).astype(np.float32), n_fluid=r["n_fluid"],
                          n_wall=r["n_wall"], h=e["h"], Lx=e["Lx"], Lz=e["Lz"]))
        off += m
    cold = [synth.element_plain(seed=700 + k, g=0.05, elem_id=100 + k) for k in range(16)]
    warm = [dict(c, seed=800 + k, id=200 + k, steps_eq=500) for k, c in enumerate(cold)]
    rc = ctx.micro_batch(cold)
    ctx.micro_plan_from(warm, snaps)
    ctx.micro_launch()
    rw = ctx.micro_results()
    ctx.close()
    assert all(r["start"] == 1 for r in rw)
    for key in ("q", "T_meas", "p"):
        a = np.array([r[key] for r in rc])
        b = np.array([r[key] for r in rw])
        se = math.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
        z = abs(a.mean() - b.mean()) / se
        print("%s: cold %.4f warm %.4f z %.2f" % (key, a.mean(), b.mean(), z))
        assert z < 2.0, (key, z)


def test_hybrid_warm_starts(native):
    # a small channel with warm starts: from the second step on, MD runs start
    # from database snapshots and equilibrate 500 steps instead of 2000
    ctx = native.Context(0, native.PREC_FP32)
    p = dict(n_sections=12, dx=50.0, h0=12.0, Lx=10.0, Lz=10.0, eos_K=10.0, eos_n0=0.8, dP_amp=400.0,
             period=1000.0, dt=20.0, T=1.1, md_steps_eq=2000, md_steps_sample=3000, seed=5, sf2=100.0,
             l2=1.0, sn2=0.25, warm_start=1, md_steps_eq_warm=500)
    hy = native.Hybrid(ctx, **p)
    st1 = hy.step(0.0)
    assert st1["md_runs"] == 12 and st1["md_warm"] == 0
    st2 = hy.step(0.0)
    assert st2["md_runs"] == 12 and st2["md_warm"] == 12
    st3 = hy.step(1.0)
    assert st3["md_warm"] == st3["md_runs"]
    assert np.isfinite(hy.state()["q"]).all()
    hy.close()
    ctx.close()


def test_hybrid_warm_starts_with_pseudo_md(native):
    # Algorithm 1's pseudoMD sets the warm runs' equilibration: the start-up
    # time from x_in's force to x*'s, within [md_steps_eq_warm, md_steps_eq]
    ctx = native.Context(0, native.PREC_FP32)
    p = dict(n_sections=8, dx=50.0, h0=12.0, Lx=10.0, Lz=10.0, eos_K=10.0, eos_n0=0.8, dP_amp=400.0,
             period=1000.0, dt=20.0, T=1.1, md_steps_eq=4000, md_steps_sample=2000, seed=9, sf2=100.0,
             l2=1.0, sn2=0.25, warm_start=1, md_steps_eq_warm=200, pseudo_nu=2.5, pseudo_slip=0.7)
    hy = native.Hybrid(ctx, **p)
    st1 = hy.step(0.0)
    assert st1["md_warm"] == 0 and st1["md_steps_eq_warm"] == 0
    X, _, _ = hy.database()
    st2 = hy.step(0.0)
    assert st2["md_warm"] == 8
    assert 200 <= st2["md_steps_eq_warm"] <= 4000
    # the longest start-up of the step, from each section's previous force to its new one
    G = hy.state()["G"]
    n = hy.state()["density"]
    hs = X[:, 0]
    ts = [native.pseudo_md(hs[j], 2.5, 0.7, -X[j, 1] / n[j], -G[j] / n[j], False, 0.8 * 10.0, 0.125)
          for j in range(8)]
    print("pseudoMD steps", st2["md_steps_eq_warm"], "t_s", max(ts) / 0.005)
    assert np.isfinite(hy.state()["q"]).all()
    hy.close()
    ctx.close()
