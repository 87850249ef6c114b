"""The converging-diverging channel case (paper Sec. 3; Algorithm 1) driven
through the library's C ABI.

run_channel() advances one hybrid case for n_steps macro steps at a given
uncertainty threshold and returns the section-averaged flow-rate history, the
MD call count and wall times.  full_channel_md() runs the full MD of the
whole channel (one element whose walls follow the profile, Sec. 3's judge).
channel_sweep() runs a threshold sweep plus the sigma_t = 0 case that runs MD
at every section and step, and reports for each threshold:
  - Eq. error: sum_i |qbar_i - Q_i| / sum_i |Q_i| against the sigma_t = 0 run
    and, given the full MD, against its App. B filtered history;
  - the same quantity between two sigma_t = 0 runs with different MD seeds
    (the thermal noise of the reference);
  - Eq. speedup: t_end N_af / (tbar_sim N_sim Nbar_ah), with N_af the atoms a
    full MD of the whole channel holds (estimated, or the full MD's own);
  - the measured wall time against the sigma_t = 0 run's and the full MD's.
"""
import math
import time

import numpy as np

from . import native


def channel_atoms(params):
    """Atoms of a full MD of the whole channel: fluid at the initial density
    over every section's cross-section plus the two tethered walls."""
    N, dx, h0, Lz, n0 = params["n_sections"], params["dx"], params["h0"], params["Lz"], params["eos_n0"]
    x = np.arange(N) * dx
    h = h0 * (1.0 - params.get("h_amp", 0.5) * np.cos(2.0 * math.pi * x / (N * dx)))
    fluid = float((n0 * h * Lz * dx).sum())
    a0 = 4.0 ** (1.0 / 3.0)
    walls = 2 * 3 * 2 * (N * dx / a0) * (Lz / a0)
    return fluid + walls


def run_channel(ctx, sigma_t, n_steps, mlp=None, sf2=None, pressure_db=None, **params):
    p = dict(params)
    if sf2 is not None:
        p["sf2"] = sf2
    hy = native.Hybrid(ctx, **p)
    if mlp is not None:
        hy.set_mlp_mean(mlp)
    if pressure_db is not None:
        hy.set_pressure(*pressure_db)
    qbar, md_runs, md_atoms = [], 0, 0
    t0 = time.perf_counter()
    gp_s = md_s = 0.0
    for _ in range(n_steps):
        st = hy.step(sigma_t)
        qbar.append(st["q_mean"])
        md_runs += st["md_runs"]
        md_atoms += st["md_atoms"]
        gp_s += st["gp_seconds"]
        md_s += st["md_seconds"]
    wall = time.perf_counter() - t0
    X, y, se = hy.database()
    hy.close()
    return dict(sigma_t=sigma_t, qbar=np.array(qbar), md_runs=md_runs, md_atoms=md_atoms, wall_s=wall,
                gp_s=gp_s, md_s=md_s, db=(X, y, se))


def fit_pseudo_md(ctx, hs=(8.0, 12.0, 16.0), g=0.02, n_seeds=8, density=0.8, T=1.1, Lx=10.0, Lz=10.0,
                  steps_eq=10000, steps_sample=10000, seed=1, mass=1.0):
    """The viscosity and slip length pseudoMD needs (Algorithm 1's t_s), from
    the library's own MD: steady driven elements at several heights, the
    steady flow rate q = m n Lz g (h^3 / 6 + slip h^2) / (2 nu) fitted by
    least squares in (1/nu, slip/nu) with weights 1/SE^2.  A negative slip
    (the fluid next to the walls at rest) is refitted as no-slip planes
    -slip inside the walls, q = m n Lz g (h + 2 slip)^3 / (12 nu), by a
    scan over slip.  Returns dict(nu, slip, h, q, q_se)."""
    els = [dict(h=float(h), Lx=Lx, Lz=Lz, density=density, T=T, g_ext=float(g), dpdx=0.0, steps_eq=steps_eq,
                steps_sample=steps_sample, seed=int(seed) + k, id=1000 * i + k)
           for i, h in enumerate(hs) for k in range(n_seeds)]
    res = ctx.micro_batch(els)
    q = np.array([r["q"] for r in res]).reshape(len(hs), n_seeds)
    qm = q.mean(1)
    qse = q.std(1, ddof=1) / math.sqrt(n_seeds)
    hv = np.array(hs, dtype=np.float64)
    scale = mass * density * Lz * g / 2.0
    A = np.column_stack([scale * hv ** 3 / 6.0, scale * hv ** 2]) / qse[:, None]
    a, b = np.linalg.lstsq(A, qm / qse, rcond=None)[0]
    nu, slip = 1.0 / a, b / a
    if slip < 0.0:
        best = None
        for d in np.linspace(0.0, 0.45 * hv.min(), 901):
            col = scale * (hv - 2.0 * d) ** 3 / 6.0 / qse
            inv_nu = float(col @ (qm / qse) / (col @ col))
            chi2 = float(((col * inv_nu - qm / qse) ** 2).sum())
            if best is None or chi2 < best[0]:
                best = (chi2, 1.0 / inv_nu, -d)
        nu, slip = best[1], best[2]
    return dict(nu=float(nu), slip=float(slip), h=hv.tolist(), q=qm.tolist(), q_se=qse.tolist())


def warm_start_comparison(ctx, sigma_t, n_steps, reference, pseudo=None, eq_warm=(500,), pressure_db=None,
                          **params):
    """Algorithm 1 with cold starts against warm starts (Sec. 2.4) at one
    threshold: MD runs, MD seconds, equilibration steps and Eq. error
    against the reference flow-rate history, for each fixed warm
    equilibration in eq_warm and, with pseudo = (nu, slip), with pseudoMD's
    start-up time (floor eq_warm[0])."""
    rows = []
    arms = [("cold", dict(warm_start=0))]
    arms += [("warm %d" % e, dict(warm_start=1, md_steps_eq_warm=int(e))) for e in eq_warm]
    if pseudo is not None:
        arms.append(("warm pseudoMD", dict(warm_start=1, md_steps_eq_warm=int(eq_warm[0]),
                                           pseudo_nu=float(pseudo[0]), pseudo_slip=float(pseudo[1]))))
    for name, kw in arms:
        hy = native.Hybrid(ctx, **dict(params, **kw))
        if pressure_db is not None:
            hy.set_pressure(*pressure_db)
        qbar, runs, warm, md_s, eq_steps = [], 0, 0, 0.0, 0
        for _ in range(n_steps):
            st = hy.step(sigma_t)
            qbar.append(st["q_mean"])
            runs += st["md_runs"]
            warm += st["md_warm"]
            md_s += st["md_seconds"]
            eq_steps += st["md_warm"] * (st["md_steps_eq_warm"] if st["md_warm"] else 0) + \
                (st["md_runs"] - st["md_warm"]) * params["md_steps_eq"]
        hy.close()
        rows.append(dict(arm=name, md_runs=runs, md_warm=warm, md_s=md_s,
                         mean_eq_steps=eq_steps / runs if runs else 0.0, error=error(qbar, reference)))
    return rows


def error(q, Q):
    return float(np.abs(np.asarray(q) - np.asarray(Q)).sum() / np.abs(np.asarray(Q)).sum())


def pressure_sweep(ctx, hs, densities, T=1.1, steps_eq=2000, steps_sample=3000, Lx=10.0, Lz=10.0, seed=1):
    """Pre-simulations for the p-GP (paper Sec. 2.4): one MD element per
    (h, n) pair with no flow forcing; returns inputs (M x 2: h, n), the
    measured pressures and their standard errors."""
    pairs = [(float(h), float(n)) for h in hs for n in densities]
    els = [dict(h=h, Lx=Lx, Lz=Lz, density=n, T=T, g_ext=0.0, dpdx=0.0, steps_eq=steps_eq,
                steps_sample=steps_sample, seed=int(seed), id=k) for k, (h, n) in enumerate(pairs)]
    res = ctx.micro_batch(els)
    return (np.array(pairs), np.array([r["p"] for r in res]), np.array([r["p_se"] for r in res]))


def channel_sweep(ctx, thresholds, n_steps=100, seed_noise=None, pressure_db=None, full_md=None, **params):
    """The threshold sweep: per threshold, MD runs, Eq. error against the
    sigma_t = 0 run (MD at every section), Eq. speedup and wall times; with
    full_md (the dict of full_channel_md plus its App. B filtered history
    under "Q_filtered") also Eq. error against the full MD, Eq. speedup with
    its own atom and step counts, and the wall time against it."""
    ref = run_channel(ctx, 0.0, n_steps, pressure_db=pressure_db, **params)
    out = {"reference": ref}
    if seed_noise is not None:
        noise = run_channel(ctx, 0.0, n_steps, pressure_db=pressure_db, **dict(params, seed=seed_noise))
        out["noise_error"] = error(noise["qbar"], ref["qbar"])
        out["noise"] = noise
    md_steps = params["md_steps_eq"] + params["md_steps_sample"]
    t_end_steps = n_steps * params["dt"] / 0.005
    n_af = channel_atoms(params)
    rows = []
    for s in thresholds:
        r = run_channel(ctx, s, n_steps, pressure_db=pressure_db, **params)
        mean_atoms = r["md_atoms"] / r["md_runs"] if r["md_runs"] else 0.0
        rows.append(dict(
            sigma_t=s, md_runs=r["md_runs"], error=error(r["qbar"], ref["qbar"]),
            speedup_eq=(t_end_steps * n_af / (md_steps * r["md_runs"] * mean_atoms)) if r["md_runs"] else math.inf,
            wall_s=r["wall_s"], wall_vs_reference=ref["wall_s"] / r["wall_s"] if r["wall_s"] > 0 else math.inf,
            gp_s=r["gp_s"], md_s=r["md_s"], result=r))
        if full_md is not None and r["md_runs"]:
            rows[-1].update(error_vs_full_md=error(r["qbar"], full_md["Q_filtered"]),
                            speedup_eq_full_md=full_md["md_steps"] * full_md["n_atoms"] /
                            (md_steps * r["md_runs"] * mean_atoms),
                            wall_vs_full_md=full_md["wall_s"] / r["wall_s"])
    if full_md is not None:
        out["reference_error_vs_full_md"] = error(ref["qbar"], full_md["Q_filtered"])
        out["full_md_noise"] = error(full_md["Q"], full_md["Q_filtered"])
    out["rows"] = rows
    return out


def subdomain_refinement(ctx, sigma_t, n_steps, levels=4, pressure_db=None, **params):
    """Sec. 3.3's cases S1-S4: the same channel with the number of sections
    doubled at each level (the new sections bisect the old ones, dx halved),
    each case starting from the database the previous one ended with.
    Returns per level: sections, MD runs, database size at the start and
    the end, and the section-averaged flow-rate history."""
    rows, db = [], None
    n0, dx0 = params.pop("n_sections"), params.pop("dx")
    for k in range(levels):
        p = dict(params, n_sections=n0 * 2 ** k, dx=dx0 / 2 ** k)
        hy = native.Hybrid(ctx, **p)
        if pressure_db is not None:
            hy.set_pressure(*pressure_db)
        if db is not None:
            hy.set_database(*db)
        start = len(hy.database()[1])
        runs, qbar = 0, []
        for _ in range(n_steps):
            st = hy.step(sigma_t)
            runs += st["md_runs"]
            qbar.append(st["q_mean"])
        db = hy.database()
        hy.close()
        rows.append(dict(n_sections=p["n_sections"], md_runs=runs, db_start=start, db_end=len(db[1]),
                         qbar=np.array(qbar)))
    return rows


def periodic_filter(ctx, t, q, period, sf2=1.0, l2=1.0, sn2=0.01, fit_until=None, max_evals=200):
    """App. B: filter the noise out of a periodic flow-rate time series q(t)
    with a GP on time alone and the periodic kernel of Eq. periodicKernel.
    The length scale and the noise variance maximise the log marginal
    likelihood (Sec. 2.3, Eq. evidenceEq) of the samples up to fit_until (the
    paper fits up to the first peak) with sf2 held; then the regression
    (Eqs. predMeanEq, predVarEq, zero prior mean) runs over the whole series.
    Returns (mean, var, l2, sn2)."""
    t = np.asarray(t, dtype=np.float64).reshape(-1, 1)
    q = np.asarray(q, dtype=np.float64)
    sel = np.ones(len(q), bool) if fit_until is None else t[:, 0] <= fit_until
    best = native.gp_optimize(ctx, t[sel], q[sel], sf2, l2, sn2, max_evals=max_evals, period=period, hold=1)
    g = native.GP(ctx, t, q, sf2, best["l2"], best["sn2"], period=period)
    mean, var = g.predict(t)
    g.close()
    return mean, var, best["l2"], best["sn2"]


def full_channel_md(ctx, n_steps, n_sections=200, dx=50.0, h0=12.0, Lz=10.0, eos_n0=0.8, dP_amp=400.0,
                    period=1000.0, dt=20.0, T=1.1, seed=1, h_amp=0.5, md_dt=0.005, sub_steps=400,
                    eq_steps=10000, log=None, **_):
    """The full MD of the channel (Sec. 3: the ground truth of Eqs. error and
    speedup): one element of length L = n_sections dx whose walls follow
    h(x) = h0 (1 - h_amp cos(2 pi x / L)), fluid at n0, every fluid atom
    driven by the external force F_ext(t) = dP_amp sin(2 pi t / period) /
    (L n0) of the hybrid's macro model (Eq. momentumEq).  The run starts from
    the lattice at rest, equilibrates eq_steps at F = 0 (t < 0), then runs
    in windows of sub_steps MD steps, each continued from the last
    (mdgp_micro_continue) with the force at the window's midpoint; Q_i is the
    mean flow rate (m / L) sum v_x over the windows within half a macro step
    of t_i = i dt, the time the hybrid's macro step i stands for.  The
    context's MD parameters apply (dt must be md_dt).
    Returns Q (n_steps), the window series (t, q), the atom count and the
    measured MD wall time."""
    L = n_sections * dx
    per_macro = int(round(dt / md_dt))
    if per_macro % sub_steps:
        raise ValueError("a macro step must hold whole windows of sub_steps MD steps")
    f_amp = dP_amp / (L * eos_n0)
    el = dict(h=h0, Lx=L, Lz=Lz, density=eos_n0, T=T, steps_eq=0, steps_sample=sub_steps, g_ext=0.0,
              seed=int(seed), id=0, wall_amp=h_amp)
    t0 = time.perf_counter()
    n_atoms = ctx.micro_plan([el])
    n_eq = max(1, int(math.ceil(eq_steps / sub_steps)))
    ctx.micro_launch()
    for _ in range(n_eq - 1):
        ctx.micro_continue(g_ext=[0.0])
    ctx.micro_results()
    # windows from t = 0 to t_n + dt / 2
    n_win = (n_steps * per_macro + per_macro // 2) // sub_steps
    tw, qw = [], []
    for k in range(n_win):
        tm = (k + 0.5) * sub_steps * md_dt
        ctx.micro_continue(g_ext=[f_amp * math.sin(2.0 * math.pi * tm / period)])
        r = ctx.micro_results()[0]
        if r["status"] != 0:
            raise RuntimeError("full-channel MD window %d: status %d" % (k, r["status"]))
        tw.append(tm)
        qw.append(r["q"])
        if log and k % 100 == 0:
            log(dict(stage="full_md", window=k, of=n_win, t=tm, q=r["q"]))
    wall = time.perf_counter() - t0
    tw, qw = np.array(tw), np.array(qw)
    Q = np.array([qw[np.abs(tw - (i + 1) * dt) <= 0.5 * dt].mean() for i in range(n_steps)])
    return dict(Q=Q, t_windows=tw, q_windows=qw, n_atoms=int(n_atoms), wall_s=wall,
                md_steps=(n_eq + n_win) * sub_steps, f_amp=f_amp)


def md_database(ctx, n_elements, seed, h_range=(6.0, 18.0), G_range=(-0.06, 0.06), density=0.8, T=1.1,
                steps_eq=1000, steps_sample=2000, Lx=10.0, Lz=10.0):
    """A training database from the library's MD: elements drawn uniformly over
    the channel's (h, G) range; returns inputs (n x 2), flow rates, errors."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(*h_range, n_elements)
    G = rng.uniform(*G_range, n_elements)
    els = [dict(h=float(h[k]), dpdx=float(G[k]), density=density, T=T, steps_eq=steps_eq,
                steps_sample=steps_sample, Lx=Lx, Lz=Lz, g_ext=0.0, seed=int(seed), id=k)
           for k in range(n_elements)]
    res = ctx.micro_batch(els)
    X = np.column_stack([h, G])
    return X, np.array([r["q"] for r in res]), np.array([r["q_se"] for r in res])


def learned_mean(ctx, X, y, sigma_n, epochs=2000, lr=3e-3, seed=1):
    """Train the MLP prior mean on the database; the residual GP's sigma_f is
    the network's holdout RMS error, floored at twice the noise level."""
    net = native.MLP(ctx, seed=seed)
    train, hold = net.train(X, y, epochs=epochs, lr=lr, eval_every=25)
    resid = y - net.predict(X)
    _, st = net.get()
    rms_hold = math.sqrt(hold) * st[5] if hold == hold else float(np.sqrt(np.mean(resid ** 2)))
    sf_res = max(rms_hold, 2.0 * sigma_n)
    return net, sf_res, dict(train_loss=train, holdout_loss=hold, rms_holdout=rms_hold)


def evidence_hyperparameters(ctx, X, y, sn2, max_evals=200):
    """(sf2, l2) of the q-GP by maximum evidence (Sec. 2.3, Eq. evidenceEq)
    on a database (X, y), sn2 held at the given noise variance."""
    y = np.asarray(y, dtype=np.float64)
    sf2 = max(float(np.var(y)), 4.0 * sn2)
    best = native.gp_optimize(ctx, X, y, sf2, 1.0, sn2, max_evals=max_evals, hold=4)
    return best["sf2"], best["l2"]


def learned_mean_comparison(ctx, thresholds, n_steps, db_elements=256, db_seed=11, epochs=2000, reference=None,
                            log=None, full_md=None, **params):
    """The learned prior mean against the plain GP at matched thresholds
    (benchmark addition to Algorithm 1).  One MD database over the channel's
    (h, G) range trains the MLP; each arm's (sf2, l2) come from the same
    rule, maximum evidence with sn2 held at the database's mean squared
    standard error -- on y for the plain GP, on the residuals y - MLP(X) for
    the learned mean -- so the two arms differ only by the prior mean.
    reference: (q history of the sigma_t = 0 run, q history of a second one
    with other MD seeds) to judge the flow error against and to set the
    thermal-noise band; run here when not given.  full_md (optional, the
    dict of full_channel_md with its App. B filtered history in "Q_filtered")
    adds each arm's Eq. error against the full MD of the channel.  log (if
    given) receives a dict after each stage."""
    say = log or (lambda d: None)
    X, y, se = md_database(ctx, db_elements, db_seed, density=params.get("eos_n0", 0.8), T=params.get("T", 1.1),
                           Lx=params.get("Lx", 10.0), Lz=params.get("Lz", 10.0),
                           steps_eq=params.get("md_steps_eq", 2000), steps_sample=params.get("md_steps_sample", 3000))
    sn2 = float(np.mean(se)) ** 2
    sf2_p, l2_p = evidence_hyperparameters(ctx, X, y, sn2)
    net = native.MLP(ctx, seed=db_seed)
    train, hold = net.train(X, y, epochs=epochs, lr=3e-3, eval_every=25)
    sf2_m, l2_m = evidence_hyperparameters(ctx, X, y - net.predict(X), sn2)
    say(dict(stage="hyperparameters", sn2=sn2, plain=(sf2_p, l2_p), mlp=(sf2_m, l2_m), holdout=hold))
    if reference is None:
        ref = run_channel(ctx, 0.0, n_steps, **params)["qbar"]
        ref2 = run_channel(ctx, 0.0, n_steps, **dict(params, seed=params.get("seed", 0) + 1000))["qbar"]
    else:
        ref, ref2 = reference
    noise = error(ref2, ref)
    say(dict(stage="reference", noise=noise))
    rows = []
    for s in thresholds:
        a = run_channel(ctx, s, n_steps, **dict(params, sf2=sf2_p, l2=l2_p, sn2=sn2))
        b = run_channel(ctx, s, n_steps, mlp=net, **dict(params, sf2=sf2_m, l2=l2_m, sn2=sn2))
        rows.append(dict(sigma_t=s, md_runs_plain=a["md_runs"], md_runs_mlp=b["md_runs"],
                         error_plain=error(a["qbar"], ref), error_mlp=error(b["qbar"], ref),
                         wall_plain=a["wall_s"], wall_mlp=b["wall_s"]))
        if full_md is not None:
            rows[-1].update(error_plain_vs_full_md=error(a["qbar"], full_md["Q_filtered"]),
                            error_mlp_vs_full_md=error(b["qbar"], full_md["Q_filtered"]))
        say(dict(stage="threshold", **rows[-1]))
    info = dict(db_elements=db_elements, sn2=sn2, plain=dict(sf2=sf2_p, l2=l2_p), mlp=dict(sf2=sf2_m, l2=l2_m),
                mlp_train_loss=train, mlp_holdout_loss=hold, noise_error=noise)
    if full_md is not None:
        info.update(md_everywhere_vs_full_md=error(ref, full_md["Q_filtered"]),
                    full_md_noise=error(full_md["Q"], full_md["Q_filtered"]))
    return rows, info, net


def mlp_comparison(ctx, thresholds, n_steps, net, sf_res, sf_plain, reference_q=None, **params):
    """MD calls and flow error of the plain-GP hybrid against the learned-mean
    hybrid at matched thresholds."""
    rows = []
    for s in thresholds:
        a = run_channel(ctx, s, n_steps, sf2=sf_plain ** 2, **params)
        b = run_channel(ctx, s, n_steps, mlp=net, sf2=sf_res ** 2, **params)
        row = dict(sigma_t=s, md_runs_plain=a["md_runs"], md_runs_mlp=b["md_runs"])
        if reference_q is not None:
            row["error_plain"] = error(a["qbar"], reference_q)
            row["error_mlp"] = error(b["qbar"], reference_q)
        rows.append(row)
    return rows
