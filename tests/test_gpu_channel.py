"""A whole converging-diverging channel as one MD element (walls that follow
h(x) = h (1 - a cos(2 pi x / Lx)): the full MD the hybrid is judged against,
Sec. 3) and continued runs (mdgp_micro_continue: the same state carried into
the next window with new forcing), against the FP64 oracle through the C ABI.

Tolerances as in test_gpu_md: FP64 path positions <= 1e-6 sigma after 100
steps and time averages to 1e-7 relative; FP32 forces 2e-5 relative; FP32
trajectories within 1e-4 sigma of the oracle over 100 steps."""
import math

import numpy as np
import pytest

from oracle import md as omd

pytestmark = pytest.mark.gpu

CH = dict(h=8.0, Lx=36.0, Lz=9.0, density=0.8, T=1.1, g_ext=0.03, wall_amp=0.4, seed=5, id=3)


@pytest.fixture(scope="module")
def native():
    from paper_1603_04628_gb300 import build, native as nat
    build.build()
    return nat


def _dx(a, b, el):
    d = a - b
    d[:, 0] -= el["Lx"] * np.round(d[:, 0] / el["Lx"])
    d[:, 2] -= el["Lz"] * np.round(d[:, 2] / el["Lz"])
    return float(np.abs(d).max())


def test_profiled_channel_trajectory_and_averages_fp64(native):
    el = dict(CH, steps_eq=40, steps_sample=60)
    ctx = native.Context(0, native.PREC_FP64)
    r = ctx.micro_batch([el])[0]
    ctx.micro_plan([el])
    ctx.micro_launch()
    xg, vg = ctx.micro_state()
    ctx.close()
    p = omd.make_params(el)
    x, v, a, sp = omd.init(p)
    acc, st = omd.simulate(p, x, v, a, sp, 0, 100)
    ref = omd.finalize(p, acc)
    assert r["status"] == 0 and (r["n_fluid"], r["n_wall"]) == (ref["n_fluid"], ref["n_wall"])
    assert _dx(xg, x, el) <= 1e-6
    assert np.abs(vg - v).max() <= 1e-5
    for k in ("q", "p", "T_meas", "e_drift"):
        assert r[k] == pytest.approx(ref[k], rel=1e-7, abs=1e-9), k


@pytest.mark.parametrize("prec", [0, 1])
def test_profiled_channel_forces(native, prec):
    el = dict(CH, Lx=30.0)
    p = omd.make_params(el)
    x, v, a, sp = omd.init(p)
    x = x + np.random.default_rng(4).uniform(-0.08, 0.08, x.shape)
    fr, wr, er = omd.lj_forces(p, x, sp, "cells")
    ctx = native.Context(0, prec)
    f, w, e = ctx.md_forces(el, x)
    ctx.close()
    d = np.linalg.norm(f - fr, axis=1)
    mag = np.linalg.norm(fr, axis=1)
    rel = d / np.maximum(mag, math.sqrt((mag ** 2).mean()))
    # atoms with a pair within 1e-6 of r_c (the truncated force jumps there)
    lo = omd.lj_forces(omd.make_params(el, rc=2.5 - 1e-6), x, sp, "cells")[0]
    hi = omd.lj_forces(omd.make_params(el, rc=2.5 + 1e-6), x, sp, "cells")[0]
    amb = (np.abs(lo - fr).max(axis=1) > 0) | (np.abs(hi - fr).max(axis=1) > 0)
    assert rel[~amb].max() <= (1e-12 if prec == 0 else 2e-5)
    assert e.sum() == pytest.approx(er.sum(), rel=1e-11 if prec == 0 else 2e-5)


def test_continued_run_follows_the_oracle_fp64(native):
    # 50 steps, then 50 more with another body force: the continued window's
    # averages and the final state against the oracle run straight through
    # (the Langevin noise of the second window uses steps 50-99)
    el = dict(CH, steps_eq=0, steps_sample=50)
    ctx = native.Context(0, native.PREC_FP64)
    ctx.micro_plan([el])
    ctx.micro_launch()
    r1 = ctx.micro_results()[0]
    ctx.micro_continue(g_ext=[0.05])
    r2 = ctx.micro_results()[0]
    xg, vg = ctx.micro_state()
    ctx.close()
    p = omd.make_params(el)
    x, v, a, sp = omd.init(p)
    acc1, _ = omd.simulate(p, x, v, a, sp, 0, 50)
    ref1 = omd.finalize(p, acc1)
    p2 = omd.make_params(dict(el, g_ext=0.05, steps_eq=50, steps_sample=50))
    acc2, _ = omd.simulate(p2, x, v, a, sp, 50, 100)
    ref2 = omd.finalize(p2, acc2)
    assert r1["status"] == 0 and r2["status"] == 0
    for k in ("q", "p", "T_meas"):
        assert r1[k] == pytest.approx(ref1[k], rel=1e-7, abs=1e-9), k
        assert r2[k] == pytest.approx(ref2[k], rel=1e-7, abs=1e-9), k
    # the continued window's drift starts from the energy the first one ended with
    drift2 = (acc2.e_last - acc1.e_last) / (ref2["n_fluid"] + ref2["n_wall"])
    assert r2["e_drift"] == pytest.approx(drift2, rel=1e-6, abs=1e-9)
    assert _dx(xg, x, el) <= 1e-6
    assert np.abs(vg - v).max() <= 1e-5


def test_continued_run_fp32_persistent(native):
    # the timed configuration: FP32 pair forces, double-float state, the
    # persistent step loop; two windows of 50 steps against the oracle
    el = dict(CH, steps_eq=0, steps_sample=50)
    ctx = native.Context(0, native.PREC_FP32)
    ctx.micro_plan([el])
    assert ctx.path() == "persistent-graph"
    ctx.micro_launch()
    ctx.micro_continue(g_ext=[0.05])
    r2 = ctx.micro_results()[0]
    xg, _ = ctx.micro_state()
    ctx.close()
    p = omd.make_params(el)
    x, v, a, sp = omd.init(p)
    omd.simulate(p, x, v, a, sp, 0, 50)
    p2 = omd.make_params(dict(el, g_ext=0.05, steps_eq=50, steps_sample=50))
    acc2, _ = omd.simulate(p2, x, v, a, sp, 50, 100)
    ref2 = omd.finalize(p2, acc2)
    assert r2["status"] == 0
    assert _dx(xg, x, el) < 1e-4
    assert r2["q"] == pytest.approx(ref2["q"], rel=1e-3, abs=1e-3)


def test_continue_needs_a_launch(native):
    ctx = native.Context(0, native.PREC_FP32)
    ctx.micro_plan([dict(CH, steps_eq=0, steps_sample=10)])
    with pytest.raises(native.MdgpError):
        ctx.micro_continue()
    ctx.close()
