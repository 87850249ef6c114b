"""GPU micro-element MD against the FP64 oracle, through the C ABI.

Tolerances:
  - pair forces, FP64 path: max_i |dF_i| <= 1e-12 * max(|F_i|, F_rms);
  - pair forces, FP32 path: max_i |dF_i| <= 2e-5 * max(|F_i|, F_rms);
    atoms with a pair within 1e-6 of r_c (where the truncated force is
    discontinuous) are held to |dF_i| <= 2 |F(r_c)| instead;
  - positions after the first 100 steps, FP64 path: <= 1e-6 sigma;
  - long-run flow rate, FP32 forces: within the ensemble z-score bound below.
"""
import math
import multiprocessing as mp

import numpy as np
import pytest

import synth
from oracle import md as omd

pytestmark = pytest.mark.gpu

FP_TOL = {0: 1e-12, 1: 2e-5}


@pytest.fixture(scope="module")
def native():
    from paper_1603_04628_gb300 import build, native as nat
    build.build()
    return nat


def _force_err(f, ref, skip=None):
    d = np.linalg.norm(f - ref, axis=1)
    mag = np.linalg.norm(ref, axis=1)
    frms = math.sqrt((mag ** 2).mean())
    rel = d / np.maximum(mag, frms)
    if skip is not None:
        rel = rel[~skip]
    return float(rel.max())


def _cutoff_ambiguous(el, x, sp, ref):
    """Atoms with a pair within 1e-6 of r_c: the truncated force jumps by
    |F(r_c)| there, so which side a finite-precision r^2 lands on is arbitrary.
    Returned with the bound their error must still meet."""
    lo = omd.lj_forces(omd.make_params(el, rc=2.5 - 1e-6), x, sp, "cells")[0]
    hi = omd.lj_forces(omd.make_params(el, rc=2.5 + 1e-6), x, sp, "cells")[0]
    amb = (np.abs(lo - ref).max(axis=1) > 0) | (np.abs(hi - ref).max(axis=1) > 0)
    return amb, 2.0 * abs(omd.lj_force(2.5))


def _wrap_dx(dx, p):
    dx = dx.copy()
    dx[:, 0] -= p.Lx * np.round(dx[:, 0] / p.Lx)
    dx[:, 2] -= p.Lz * np.round(dx[:, 2] / p.Lz)
    return dx


def _configs():
    rng = np.random.default_rng(17)
    out = []
    el = synth.element_plain()
    p = omd.make_params(el)
    x, v, a, sp = omd.init(p)
    out.append(("lattice+jitter", el, x + rng.uniform(-0.1, 0.1, x.shape), sp))
    x2, v2 = x.copy(), v.copy()
    omd.simulate(p, x2, v2, a, sp, 0, 300)
    out.append(("liquid after 300 steps", el, x2, sp))
    el3 = synth.batch_uneven(3, seed=5, steps=100)[2]
    p3 = omd.make_params(el3)
    x3, v3, a3, sp3 = omd.init(p3)
    omd.simulate(p3, x3, v3, a3, sp3, 0, 100)
    out.append(("uneven element", el3, x3, sp3))
    return out


CONFIGS = None


def configs():
    global CONFIGS
    if CONFIGS is None:
        CONFIGS = _configs()
    return CONFIGS


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("which", [0, 1, 2])
def test_pair_forces_match_oracle(native, prec, which):
    name, el, x, sp = configs()[which]
    p = omd.make_params(el)
    fr, wr, er = omd.lj_forces(p, x, sp, "cells")
    amb, jump = _cutoff_ambiguous(el, x, sp, fr)
    ctx = native.Context(0, prec)
    f, w, e = ctx.md_forces(el, x)
    err = _force_err(f, fr, amb)
    assert err <= FP_TOL[prec], (name, err)
    assert np.abs(f - fr)[amb].max(initial=0.0) <= jump
    # fluid atoms' x-virial shares (the pressure measurement's input) and energies
    tol = 1e-11 if prec == 0 else 2e-5
    fl = sp == 0
    assert np.abs(w[fl] - wr[fl]).max() <= tol * max(np.abs(wr[fl]).max(), 1.0)
    assert (w[~fl] == 0).all()
    assert e.sum() == pytest.approx(er.sum(), rel=tol)
    ctx.close()


def test_pair_forces_at_maximum_element_size(native):
    # the tallest, widest and densest element of the stress workload
    el = dict(h=40.0, Lx=31.0, Lz=31.0, density=0.9, T=1.1, g_ext=0.0, seed=3, id=9)
    p = omd.make_params(el)
    x, v, a, sp = omd.init(p)
    x = x + np.random.default_rng(1).uniform(-0.08, 0.08, x.shape)
    fr, wr, er = omd.lj_forces(p, x, sp, "cells")
    amb, jump = _cutoff_ambiguous(el, x, sp, fr)
    for prec in (0, 1):
        ctx = native.Context(0, prec)
        f, w, e = ctx.md_forces(el, x)
        assert _force_err(f, fr, amb) <= FP_TOL[prec], prec
        assert np.abs(f - fr)[amb].max(initial=0.0) <= jump
        ctx.close()


def test_first_100_steps_positions_fp64(native):
    el = synth.element_plain(steps_eq=100, steps_sample=0)
    ctx = native.Context(0, native.PREC_FP64)
    ctx.micro_plan([el])
    ctx.micro_launch()
    res = ctx.micro_results()[0]
    xg, vg = ctx.micro_state()
    p = omd.make_params(el)
    x, v, a, sp = omd.init(p)
    omd.simulate(p, x, v, a, sp, 0, 100)
    assert res["status"] == 0
    assert np.abs(_wrap_dx(xg - x, p)).max() <= 1e-6
    assert np.abs(vg - v).max() <= 1e-5
    ctx.close()


def test_short_run_measurements_fp64(native):
    # 150 steps, 100 sampled: identical trajectories give identical averages
    el = synth.element_plain(steps_eq=50, steps_sample=100, g=0.05)
    ctx = native.Context(0, native.PREC_FP64)
    res = ctx.micro_batch([el])[0]
    ref = omd.element(omd.make_params(el))
    for k in ("q", "p", "T_meas", "q_se", "p_se", "e_drift"):
        assert res[k] == pytest.approx(ref[k], rel=1e-7, abs=1e-9), k
    assert (res["n_fluid"], res["n_wall"]) == (ref["n_fluid"], ref["n_wall"])
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_batch_matches_each_element(native, prec):
    els = synth.batch_uneven(5, seed=11, steps=60)
    els[2] = dict(els[2], dpdx=0.01)          # pressure-gradient input (Eq. momentumEq)
    ctx = native.Context(0, prec)
    ctx.micro_plan(els)
    ctx.micro_launch()
    res = ctx.micro_results()
    xg, vg = ctx.micro_state()
    off = 0
    for el, r in zip(els, res):
        p = omd.make_params(el)
        x, v, a, sp = omd.init(p)
        acc, st = omd.simulate(p, x, v, a, sp, 0, 60)
        ref = omd.finalize(p, acc)
        n = len(sp)
        dx = np.abs(_wrap_dx(xg[off:off + n] - x, p)).max()
        off += n
        assert r["status"] == 0
        if prec == 0:
            assert dx <= 1e-6
            assert r["q"] == pytest.approx(ref["q"], rel=1e-7, abs=1e-9)
        else:
            assert dx <= 1e-3          # FP32 forces: trajectories stay close over 60 steps
            assert r["q"] == pytest.approx(ref["q"], rel=1e-2, abs=0.05)
    assert off == len(xg)
    ctx.close()


def test_edge_cases(native):
    ctx = native.Context(0, native.PREC_FP64)
    with pytest.raises(native.MdgpError):
        ctx.micro_batch([dict(synth.element_plain(), Lx=7.0)])       # fewer than 3 cells along x
    with pytest.raises(native.MdgpError):
        ctx.micro_batch([])
    # no sampling steps: no averages
    r = ctx.micro_batch([synth.element_plain(steps_eq=10, steps_sample=0)])[0]
    assert r["status"] == 0 and math.isnan(r["q"])
    # walls only
    r = ctx.micro_batch([dict(synth.element_plain(steps_eq=5, steps_sample=20), density=0.0)])[0]
    assert r["status"] == 0 and r["n_fluid"] == 0 and r["n_wall"] > 0
    # fewer samples than blocks
    r = ctx.micro_batch([synth.element_plain(steps_eq=0, steps_sample=3)])[0]
    ref = omd.element(omd.make_params(synth.element_plain(steps_eq=0, steps_sample=3)))
    assert r["q"] == pytest.approx(ref["q"], rel=1e-8)
    assert r["q_se"] == pytest.approx(ref["q_se"], rel=1e-6)
    # a neighbour-list capacity that is too small is reported, never written past
    ctx.set_md_params(list_capacity=8)
    ctx.micro_plan([synth.element_plain(steps_eq=2, steps_sample=2)])
    ctx.micro_launch()
    assert ctx.micro_results()[0]["status"] == -8
    ctx.close()


def test_uneven_step_counts_split_into_groups(native):
    els = [synth.element_plain(steps_eq=10, steps_sample=20, elem_id=0),
           synth.element_plain(steps_eq=5, steps_sample=40, elem_id=1, seed=9)]
    ctx = native.Context(0, native.PREC_FP64)
    res = ctx.micro_batch(els)
    for el, r in zip(els, res):
        ref = omd.element(omd.make_params(el))
        assert r["q"] == pytest.approx(ref["q"], rel=1e-7, abs=1e-9)
    ctx.close()


def _oracle_run(el):
    return omd.element(omd.make_params(el))


def test_long_run_flow_rate_fp32_within_oracle_ensemble(native):
    # the plain element (2000 + 3000 steps) with body force 0.05, sixteen seeds
    # on each side; the standard error of each ensemble mean is the spread
    # across seeds / sqrt(16) (independent runs), the bound is two combined
    # standard errors, |z| < 2.  Both sides are deterministic (the oracle, and
    # the GPU's fixed in-cell order and summation orders), so for these
    # seeds the outcome is the same on every run.
    seeds = [301 + k for k in range(16)]
    els = [synth.element_plain(seed=s, g=0.05, elem_id=k) for k, s in enumerate(seeds)]
    ctx_pool = mp.get_context("spawn")
    with ctx_pool.Pool(16) as pool:
        refs = pool.map(_oracle_run, els)
    ctx = native.Context(0, native.PREC_FP32)
    res = ctx.micro_batch(els)
    ctx.close()
    for key in ("q", "p", "T_meas"):
        g = np.array([r[key] for r in res])
        o = np.array([r[key] for r in refs])
        se = math.sqrt(g.var(ddof=1) / len(g) + o.var(ddof=1) / len(o))
        z = abs(g.mean() - o.mean()) / se
        print("%s: gpu %.4f oracle %.4f z %.2f" % (key, g.mean(), o.mean(), z))
        assert z < 2.0, (key, z)


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_conservation_without_thermostat_or_forcing(native, prec):
    # NVE (gamma = 0, g = 0): velocity Verlet conserves energy up to O(dt^2)
    # fluctuations; a pair missed by the neighbour lists would show as a jump
    el = synth.element_plain(steps_eq=1500, steps_sample=500, g=0.0)
    ctx = native.Context(0, prec, gamma_wall=0.0)
    r = ctx.micro_batch([el])[0]
    ctx.close()
    ref = omd.element(omd.make_params(el, gamma_wall=0.0))
    assert r["status"] == 0
    assert abs(ref["e_drift"]) < 2e-3
    assert abs(r["e_drift"]) < 2e-3 + 2 * abs(ref["e_drift"])


def test_ballot_build_multi_pass_matches_oracle(native):
    # dense walls (wall density 4) and r_c = 4 put far more than one shared
    # buffer of candidates around each cell and more than 32 atoms in a cell:
    # the ballot build sweeps in several passes
    el = dict(h=8.0, Lx=13.5, Lz=13.5, density=0.75, T=2.44, g_ext=0.0, dpdx=0.0, steps_eq=0, steps_sample=0,
              seed=3, id=0)
    p = omd.make_params(el, **PAPER_MODE)
    x, v, a, sp = omd.init(p)
    rng = np.random.default_rng(5)
    x = x + rng.normal(0.0, 0.05, x.shape) * (sp[:, None] == 0)
    fr, wr, er = omd.lj_forces(p, x, sp, "cells")
    ctx = native.Context(0, native.PREC_FP64, list_capacity=1600, **PAPER_MODE)
    f, w, e = ctx.md_forces(el, x)
    ctx.close()
    assert _force_err(f, fr) <= FP_TOL[0]
    fl = sp == 0
    assert np.abs(w[fl] - wr[fl]).max() <= 1e-11 * max(np.abs(wr[fl]).max(), 1.0)


def test_autotune_keeps_results_exact(native):
    els = synth.batch_uneven(6, seed=13, steps=60)
    ctx = native.Context(0, native.PREC_FP64)
    chosen, rate = ctx.autotune(els, probe_steps=40)
    assert chosen["skin"] in (0.3, 0.4, 0.5, 0.6)
    assert rate > 0
    res = ctx.micro_batch(els)
    for el, r in zip(els, res):
        ref = omd.element(omd.make_params(el))
        assert r["q"] == pytest.approx(ref["q"], rel=1e-7, abs=1e-9)
    ctx.close()


PAPER_MODE = dict(mode=1, eps_wf=0.2, sig_wf=0.75, wall_density=4.0, rc=4.0, dt=0.0025, tau_T=0.5)


def test_paper_mode_frozen_walls_berendsen_fp64(native):
    # App. A parameters: frozen dense walls, wall-fluid (0.2, 0.75), r_c = 4,
    # dt = 0.0025, T = 2.44, Berendsen on the fluid's v_z
    el = dict(h=10.0, Lx=15.0, Lz=15.0, density=0.75, T=2.44, g_ext=0.02, dpdx=0.0, steps_eq=60,
              steps_sample=40, seed=77, id=5)
    ctx = native.Context(0, native.PREC_FP64, list_capacity=640, **PAPER_MODE)
    ctx.micro_plan([el])
    ctx.micro_launch()
    r = ctx.micro_results()[0]
    xg, vg = ctx.micro_state()
    ctx.close()
    p = omd.make_params(el, **PAPER_MODE)
    x, v, a, sp = omd.init(p)
    acc, st = omd.simulate(p, x, v, a, sp, 0, 100)
    ref = omd.finalize(p, acc)
    assert r["status"] == 0
    assert np.abs(_wrap_dx(xg - x, p)).max() <= 1e-6
    assert np.abs(_wrap_dx(xg[sp == 1] - a[sp == 1], p)).max() <= 1e-12   # walls did not move
    for k in ("q", "p", "T_meas", "e_drift"):
        assert r[k] == pytest.approx(ref[k], rel=1e-7, abs=1e-9), k


@pytest.mark.parametrize("mode", [0, 1])
def test_persistent_step_loop_matches_per_step_launches(native, mode):
    # the persistent step kernel (grid barriers between steps, rebuilds in a
    # graph WHILE loop) and one launch per step do the same arithmetic; the
    # order of atoms inside a cell (binning atomics) may differ, so the
    # trajectories agree to FP32 summation order over a short run
    els = synth.batch_uneven(6, seed=21, steps=80)
    kw = PAPER_MODE if mode == 1 else {}
    if mode == 1:
        # r_c = 4: the box must hold three cells of r_c + skin along x and z
        els = [dict(e, T=2.44, density=0.75, Lx=15.0, Lz=15.0) for e in els]
    out = []
    for persistent in (1, 0):
        ctx = native.Context(0, native.PREC_FP32, persistent=persistent, list_capacity=640 if mode else 128, **kw)
        ctx.micro_plan(els)
        ctx.micro_launch()
        res = ctx.micro_results()
        x, v = ctx.micro_state()
        out.append((res, x, v, ctx.rebuild_count()))
        ctx.close()
    (ra, xa, va, na), (rb, xb, vb, nb) = out
    assert all(r["status"] == 0 for r in ra + rb)
    assert na > 1 and nb > 1
    off = 0
    for el, r in zip(els, ra):
        n = r["n_fluid"] + r["n_wall"]
        d = xa[off:off + n] - xb[off:off + n]
        d[:, 0] -= el["Lx"] * np.round(d[:, 0] / el["Lx"])
        d[:, 2] -= el["Lz"] * np.round(d[:, 2] / el["Lz"])
        assert np.abs(d).max() < 1e-3
        off += n
    assert off == len(xa)
    assert np.abs(va - vb).max() < 1e-2
    for a, b in zip(ra, rb):
        assert a["q"] == pytest.approx(b["q"], rel=1e-2, abs=1e-3)


@pytest.mark.parametrize("tpa", [1, 2, 4, 8])
def test_threads_per_atom_against_the_oracle(native, tpa):
    # several threads sharing an atom's pair loop (small batches): each
    # element of a ragged batch after 100 persistent FP32 steps against its
    # own FP64 oracle run, as for the full benchmark batch
    import os
    els = synth.batch_uneven(4, seed=23, steps=100)
    with mp.get_context("spawn").Pool(min(4, os.cpu_count() or 1)) as pool:
        refs = pool.map(_oracle_positions, els)
    ctx = native.Context(0, native.PREC_FP32, threads_per_atom=tpa)
    n = ctx.micro_plan(els)
    shape = ctx.launch_shape()
    ctx.micro_launch()
    res = ctx.micro_results()
    xg, _ = ctx.micro_state()
    ctx.close()
    assert shape["threads_per_atom"] == tpa
    assert shape["atoms_per_block"] * tpa <= shape["threads"] <= 256
    assert shape["blocks"] * shape["atoms_per_block"] >= n
    assert all(r["status"] == 0 for r in res)
    off, worst = 0, 0.0
    for el, r, xr in zip(els, res, refs):
        m = r["n_fluid"] + r["n_wall"]
        d = xg[off:off + m] - xr
        d[:, 0] -= el["Lx"] * np.round(d[:, 0] / el["Lx"])
        d[:, 2] -= el["Lz"] * np.round(d[:, 2] / el["Lz"])
        worst = max(worst, float(np.abs(d).max()))
        off += m
    assert off == n
    assert worst < 1e-4


def test_threads_per_atom_paper_mode_and_auto_choice(native):
    # frozen walls, Berendsen and mixed pair types (the non-uniform pair
    # loop) with four threads per atom follow the one-thread run to FP32
    # summation order; a two-element batch gets several threads per atom by
    # default, the 64-element benchmark batch one
    els = [dict(e, T=2.44, density=0.75, Lx=15.0, Lz=15.0) for e in synth.batch_uneven(3, seed=21, steps=80)]
    out = []
    for tpa in (1, 4):
        ctx = native.Context(0, native.PREC_FP32, threads_per_atom=tpa, list_capacity=640, **PAPER_MODE)
        ctx.micro_plan(els)
        ctx.micro_launch()
        out.append((ctx.micro_results(), ctx.micro_state()[0]))
        ctx.close()
    (ra, xa), (rb, xb) = out
    assert all(r["status"] == 0 for r in ra + rb)
    off = 0
    for el, r in zip(els, ra):
        m = r["n_fluid"] + r["n_wall"]
        d = xa[off:off + m] - xb[off:off + m]
        d[:, 0] -= el["Lx"] * np.round(d[:, 0] / el["Lx"])
        d[:, 2] -= el["Lz"] * np.round(d[:, 2] / el["Lz"])
        assert np.abs(d).max() < 1e-3
        off += m
    for a, b in zip(ra, rb):
        assert a["q"] == pytest.approx(b["q"], rel=1e-2, abs=1e-3)
    ctx = native.Context(0, native.PREC_FP32)
    ctx.micro_plan([synth.element_plain(steps_eq=10, steps_sample=10)] * 2)
    assert ctx.launch_shape()["threads_per_atom"] == 8
    ctx.micro_plan(synth.batch_uneven(64, steps=10))
    assert ctx.launch_shape()["threads_per_atom"] == 1
    ctx.close()


@pytest.mark.parametrize("tpa,persistent,cap", [(8, 1, 128), (4, 1, 128), (2, 2, 128), (2, 1, 256)])
def test_resident_kernel_matches_the_general_one_bit_for_bit(native, tpa, persistent, cap):
    # the small-batch kernel that keeps each atom's state in registers and
    # its list in shared memory for a rebuild interval runs the same
    # arithmetic in the same order as the general persistent kernel: after
    # 300 steps (~30 rebuilds, each a fresh launch that reloads and writes
    # back the state) positions and velocities are identical bit for bit.  The
    # measurements are not part of the state: their per-atom terms are formed
    # in FP32 (the compiler may fuse their multiply-adds differently in the
    # two kernels) and summed by FP64 atomics in arbitrary order, so q, P_xx
    # and T are held to 1e-6 relative, far inside their standard errors.  A
    # list capacity of 256 puts the shared memory above the default 48 KB per
    # block.
    els = synth.batch_uneven(3, seed=29, steps=300)
    out = []
    for resident in (0, 1):
        ctx = native.Context(0, native.PREC_FP32, threads_per_atom=tpa, persistent=persistent,
                             list_capacity=cap, resident=resident)
        ctx.micro_plan(els)
        shape = ctx.launch_shape()
        ctx.micro_launch()
        res = ctx.micro_results()
        x, v = ctx.micro_state()
        out.append((shape, res, x, v, ctx.rebuild_count()))
        ctx.close()
    (sa, ra, xa, va, na), (sb, rb, xb, vb, nb) = out
    assert sa["resident"] == 0 and sb["resident"] == 1
    assert sa["threads_per_atom"] == sb["threads_per_atom"] == tpa
    assert all(r["status"] == 0 for r in ra + rb)
    assert na == nb > 10
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    for a, b in zip(ra, rb):
        for key in ("q", "p", "T_meas"):
            assert a[key] == pytest.approx(b[key], rel=1e-6, abs=1e-12)


def test_resident_kernel_only_where_it_applies(native):
    # frozen walls (two phases per step), one thread per atom and batches
    # whose blocks would stride over several chunks keep the general kernel
    els = [dict(e, T=2.44, density=0.75, Lx=15.0, Lz=15.0) for e in synth.batch_uneven(2, seed=21, steps=20)]
    ctx = native.Context(0, native.PREC_FP32, list_capacity=640, **PAPER_MODE)
    ctx.micro_plan(els)
    assert ctx.launch_shape()["threads_per_atom"] > 1
    assert ctx.launch_shape()["resident"] == 0
    ctx.close()
    ctx = native.Context(0, native.PREC_FP32)
    ctx.micro_plan([synth.element_plain(steps_eq=10, steps_sample=10)] * 2)
    assert ctx.launch_shape()["resident"] == 1
    ctx.micro_plan(synth.batch_uneven(64, steps=10))
    assert ctx.launch_shape()["resident"] == 0
    ctx.close()


def test_full_uneven_batch_in_bench_configuration():
    # the 64-element batch exactly as bench.py launches it (FP32 pair forces,
    # double-float state, persistent step loop, default parameters), 100
    # steps: every element finishes cleanly, and sampled elements (smallest,
    # largest, a middle one) run alone follow the same trajectories to FP32
    # summation order: batching couples nothing
    from paper_1603_04628_gb300 import native
    els = synth.batch_uneven(64, steps=100)
    ctx = native.Context(0, native.PREC_FP32)
    n = ctx.micro_plan(els)
    ctx.micro_launch()
    res = ctx.micro_results()
    xb, vb = ctx.micro_state()
    assert all(r["status"] == 0 for r in res)
    assert ctx.rebuild_count() >= 2
    sizes = [r["n_fluid"] + r["n_wall"] for r in res]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    assert offs[-1] == n == len(xb)
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 31})
    for k in picks:
        c1 = native.Context(0, native.PREC_FP32)
        c1.micro_plan([els[k]])
        c1.micro_launch()
        r1 = c1.micro_results()[0]
        x1, v1 = c1.micro_state()
        c1.close()
        d = xb[offs[k]:offs[k + 1]] - x1
        d[:, 0] -= els[k]["Lx"] * np.round(d[:, 0] / els[k]["Lx"])
        d[:, 2] -= els[k]["Lz"] * np.round(d[:, 2] / els[k]["Lz"])
        assert np.abs(d).max() < 1e-3, k
        assert r1["q"] == pytest.approx(res[k]["q"], rel=2e-2, abs=2e-2), k
    ctx.close()


def test_fp32_forces_dense_walls_paper_mode(native):
    # FP32 pair forces with the paper's parameters: frozen dense walls (wall
    # density 4), wall-fluid (0.2, 0.75), r_c = 4 -- crowded cells, several
    # candidate passes per cell, three pair types
    el = dict(h=8.0, Lx=13.5, Lz=13.5, density=0.75, T=2.44, g_ext=0.0, dpdx=0.0, steps_eq=0, steps_sample=0,
              seed=3, id=0)
    p = omd.make_params(el, **PAPER_MODE)
    x, v, a, sp = omd.init(p)
    rng = np.random.default_rng(5)
    x = x + rng.normal(0.0, 0.05, x.shape) * (sp[:, None] == 0)
    fr, wr, er = omd.lj_forces(p, x, sp, "cells")
    amb, jump = _cutoff_ambiguous_rc(el, x, sp, fr, 4.0, PAPER_MODE)
    ctx = native.Context(0, native.PREC_FP32, list_capacity=1600, **PAPER_MODE)
    f, w, e = ctx.md_forces(el, x)
    ctx.close()
    assert _force_err(f, fr, amb) <= FP_TOL[1]
    fl = sp == 0
    assert np.abs(w[fl] - wr[fl]).max() <= 2e-5 * max(np.abs(wr[fl]).max(), 1.0)
    assert e.sum() == pytest.approx(er.sum(), rel=2e-5)


def _cutoff_ambiguous_rc(el, x, sp, ref, rc, phys):
    lo = omd.lj_forces(omd.make_params(el, **dict(phys, rc=rc - 1e-6)), x, sp, "cells")[0]
    hi = omd.lj_forces(omd.make_params(el, **dict(phys, rc=rc + 1e-6)), x, sp, "cells")[0]
    return (np.abs(lo - ref).max(axis=1) > 0) | (np.abs(hi - ref).max(axis=1) > 0), None


@pytest.mark.parametrize("prec", [0, 1])
def test_runs_are_reproducible(native, prec):
    # the in-cell order follows the atoms' original indices and every
    # per-atom sum runs in a fixed order, so the same batch gives the same
    # trajectory bit for bit (FP32: the persistent step loop)
    els = synth.batch_uneven(4, seed=31, steps=120)
    out = []
    for _ in range(2):
        ctx = native.Context(0, prec)
        ctx.micro_plan(els)
        ctx.micro_launch()
        res = ctx.micro_results()
        x, v = ctx.micro_state()
        out.append((res, x, v, ctx.rebuild_count()))
        ctx.close()
    (ra, xa, va, na), (rb, xb, vb, nb) = out
    assert na == nb > 1
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    for a, b in zip(ra, rb):
        assert a["status"] == b["status"] == 0
        assert a["q"] == pytest.approx(b["q"], rel=1e-12, abs=1e-14)   # FP64 atomics add the samples


@pytest.mark.parametrize("resident", [0, 1])
def test_barrier_timeout_is_reported_and_context_recovers(native, resident):
    # failure detection without a fault: one block of the persistent step
    # kernel (the general one and the resident-atom one) leaves out its first
    # grid-barrier arrival (test-only switch), so every other block's bounded
    # wait runs out after 50 ms of the GPU's global timer; the launch ends
    # with MDGP_E_TIMEOUT on every element and the same context then runs the
    # batch cleanly
    els = synth.batch_uneven(3, seed=41, steps=40)
    ctx = native.Context(0, native.PREC_FP32, inject_barrier_skip=1, wait_timeout_ms=50, resident=resident)
    ctx.micro_plan(els)
    assert ctx.launch_shape()["resident"] == resident
    ctx.micro_launch()
    res = ctx.micro_results()
    assert [r["status"] for r in res] == [-6] * len(els)
    ctx.set_md_params(wait_timeout_ms=50, resident=resident)
    ctx.micro_plan(els)
    assert ctx.launch_shape()["resident"] == resident
    ctx.micro_launch()
    res = ctx.micro_results()
    assert all(r["status"] == 0 for r in res)
    ref = native.Context(0, native.PREC_FP32, resident=resident).micro_batch(els)
    for a, b in zip(res, ref):
        assert a["q"] == pytest.approx(b["q"], rel=1e-12, abs=1e-14)
    ctx.close()


def test_double_float_state_against_fp64_over_20000_steps(native):
    # The FP32-force path keeps positions and velocities as double-float
    # pairs (~44-bit significand) instead of FP64.  Over 20 000 steps of an
    # element of the uneven batch's kind (h = 10, 12 x 12, n = 0.8):
    #  - NVE (no thermostat, no forcing): the energy drift per atom stays at
    #    the FP64 run's level -- a state rounded like plain FP32 would walk;
    #  - driven (g = 0.02, thermostatted walls): the ensemble-mean flow rate
    #    of sixteen seeds matches the FP64 ensemble within two standard
    #    errors (the runs are chaotic, so seeds, not trajectories, compare).
    base = dict(h=10.0, Lx=12.0, Lz=12.0, density=0.8, T=1.1, g_ext=0.0, dpdx=0.0, steps_eq=4000,
                steps_sample=16000, seed=7, id=0)
    drift = {}
    for prec in (0, 1):
        ctx = native.Context(0, prec, gamma_wall=0.0)
        drift[prec] = ctx.micro_batch([base])[0]["e_drift"]
        ctx.close()
    print("NVE e_drift per atom: FP64 %.3g, FP32 forces + double-float state %.3g" % (drift[0], drift[1]))
    assert abs(drift[1]) <= 2.0 * abs(drift[0]) + 2e-4
    els = [dict(base, g_ext=0.02, seed=900 + k, id=k) for k in range(16)]
    q = {}
    for prec in (0, 1):
        ctx = native.Context(0, prec)
        res = ctx.micro_batch(els)
        ctx.close()
        assert all(r["status"] == 0 for r in res)
        q[prec] = np.array([r["q"] for r in res])
    se = math.sqrt(q[0].var(ddof=1) / 16 + q[1].var(ddof=1) / 16)
    z = abs(q[0].mean() - q[1].mean()) / se
    print("q over 16 seeds: FP64 %.4f, FP32 + double-float %.4f, combined SE %.4f, z %.2f"
          % (q[0].mean(), q[1].mean(), se, z))
    assert z < 2.0


def _oracle_positions(el):
    p = omd.make_params(el)
    x, v, a, sp = omd.init(p)
    omd.simulate(p, x, v, a, sp, 0, el["steps_eq"] + el["steps_sample"])
    return x


def test_full_uneven_batch_against_the_oracle():
    # every element of the 64-element batch exactly as bench.py launches it
    # (FP32 pair forces, double-float state, the persistent step loop), 100
    # steps, against its own FP64 oracle run:
    # positions agree to FP32 order (the force error, ~1e-5 relative, grows
    # through the chaotic dynamics to well under 1e-4 sigma in 100 steps)
    import os
    from paper_1603_04628_gb300 import native
    els = synth.batch_uneven(64, steps=100)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        refs = pool.map(_oracle_positions, els)
    ctx = native.Context(0, native.PREC_FP32)
    n = ctx.micro_plan(els)
    ctx.micro_launch()
    res = ctx.micro_results()
    xg, vg = ctx.micro_state()
    ctx.close()
    assert all(r["status"] == 0 for r in res)
    off, worst = 0, 0.0
    for el, r, xr in zip(els, res, refs):
        m = r["n_fluid"] + r["n_wall"]
        assert m == len(xr)
        d = xg[off:off + m] - xr
        d[:, 0] -= el["Lx"] * np.round(d[:, 0] / el["Lx"])
        d[:, 2] -= el["Lz"] * np.round(d[:, 2] / el["Lz"])
        worst = max(worst, float(np.abs(d).max()))
        off += m
    assert off == n
    print("64-element batch, 100 steps: max |dx| against the oracle %.3g sigma" % worst)
    assert worst < 1e-4
