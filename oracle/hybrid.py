"""Algorithm 1 (hybrid scheme with on-the-fly GP learning), plain Python.

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and bench.py's CPU-baseline
leg may import this module; the product package never does.

Macro model (paper Sec. 2.1, Eqs. subsEq, continuityEq, momentumEq; readings
for the parts the paper leaves open are marked READING):
  - N periodic sections at x_j = j dx (Eq. subsEq with L = N dx); heights
    h_j = h0 (1 - a cos(2 pi x_j / L)), a = 0.5 by default (the converging-diverging channel in
    the benchmark's form; the paper's Eq. heightEq has the same shape);
  - state: fluid number density n_j (mass density m n_j, m = 1);
  - pressure from a linear equation of state p = K (n - n0) (READING), or
    as in the paper (Sec. 2.4) from a second GP, the p-GP over (h, n),
    fitted once to pressures measured in pre-simulations and evaluated at
    its posterior mean;
  - pressure gradient by periodic central differences (Alg. 1, the p' line);
  - Eq. momentumEq: every fluid atom feels F_j = F_ext - p'_j / n_j, the
    external force F_ext the same on every atom of the channel (Algorithm 1
    sets one F_ext^i per macro step).  READING: its amplitude is given as an
    inlet-outlet pressure difference dP(t) = dP_A sin(2 pi t / period) at the
    initial density, F_ext = dP / (L n0); an MD element gets
    dpdx = G_j = p'_j - n_j F_ext, so that F = -G_j / n_j; the q-GP input is
    x = (h_j, G_j), or the paper's (h_j, n_j, F_j) (inputs = 1);
  - q-GP (Eqs. quadraticKernelEq-predVarEq) on the database of (x, q) pairs,
    refit whenever the database grows; gate sd > sigma_t (strict);
  - READING: sigma_n is fixed during a macro step.  The paper measured it
    once beforehand (Sec. 2.3) and kept it; here it is the configured value,
    or optionally (sn2_from_data) the mean standard error of the database's
    MD runs as they stood at the start of the step.  Holding it fixed within
    a step keeps the gate a function of the inputs alone;
  - continuity, Eq. continuityEq discretised with central differences:
    n_j <- n_j - dt / A_j (q_{j+1} - q_{j-1}) / (2 dx), A_j = h_j L_z.
"""
import math

import numpy as np

from . import gp as ogp


class Channel:
    def __init__(self, n_sections=8, dx=50.0, h0=12.0, Lx=10.0, Lz=10.0, K=10.0, n0=0.8, dP_amp=0.0,
                 period=1000.0, dt=20.0, T=1.1, steps_eq=100, steps_sample=100, seed=7, sf2=1.0, l2=1.0,
                 sn2_default=0.0025, sn2_from_data=False, density0=None, inputs=0, pressure_db=None, h_amp=0.5):
        self.N = int(n_sections)
        self.dx, self.h0, self.Lx, self.Lz = float(dx), float(h0), float(Lx), float(Lz)
        self.K, self.n0, self.dP_amp, self.period, self.dt = float(K), float(n0), float(dP_amp), float(period), float(dt)
        self.T, self.steps_eq, self.steps_sample, self.seed = float(T), int(steps_eq), int(steps_sample), int(seed)
        self.sf2, self.l2, self.sn2_default, self.sn2_from_data = float(sf2), float(l2), float(sn2_default), bool(sn2_from_data)
        L = self.N * self.dx
        x = np.arange(self.N) * self.dx
        self.h = self.h0 * (1.0 - h_amp * np.cos(2.0 * math.pi * x / L))
        # Eq. d2Eq's mean separation is undefined for an input without spread
        # (all h equal; the uniform gradient of the first steps; a uniform
        # density): h then takes h0 / 2, G the forcing gradient amplitude
        # dP_amp / L (F that over n0), n a tenth of n0
        g = self.dP_amp / L if self.dP_amp > 0 else 1.0
        self.D = 3 if inputs == 1 else 2
        self.fallback = (np.array([0.5 * self.h0, g]) if self.D == 2 else
                         np.array([0.5 * self.h0, 0.1 * self.n0, g / self.n0]))
        # p-GP (Sec. 2.4): (X (M x 2: h, n), p, sf2, l2, sn2), or None for the linear law
        self.pgp = None
        if pressure_db is not None:
            Xp, yp, psf2, pl2, psn2 = pressure_db
            if len(yp):
                self.pgp = ogp.GP(np.asarray(Xp, dtype=np.float64).reshape(-1, 2), np.asarray(yp, dtype=np.float64),
                                  psf2, pl2, psn2, fallback=[0.5 * self.h0, 0.1 * self.n0])
        self.n = np.full(self.N, self.n0) if density0 is None else np.array(density0, dtype=np.float64)
        self.i = 0                       # macro steps taken
        self.X = np.zeros((0, self.D))
        self.y = np.zeros(0)
        self.se = np.zeros(0)
        self.md_calls = 0

    # ------------------------------------------------------------------ helpers
    def sn2(self):
        """Noise variance for the coming step."""
        if self.sn2_from_data and len(self.se) > 0:
            return float(np.mean(self.se)) ** 2
        return self.sn2_default

    def pressure(self):
        if self.pgp is not None:
            return self.pgp.predict(np.column_stack([self.h, self.n]))[0]
        return self.K * (self.n - self.n0)

    def inputs(self, j, G):
        """Section j's q-GP input row."""
        if self.D == 2:
            return np.array([[self.h[j], G[j]]])
        return np.array([[self.h[j], self.n[j], -G[j] / self.n[j]]])

    def gradients(self, t):
        p = self.pressure()
        dpdx = (np.roll(p, -1) - np.roll(p, 1)) / (2.0 * self.dx)
        dP = self.dP_amp * math.sin(2.0 * math.pi * t / self.period)
        f_ext = dP / (self.N * self.dx * self.n0)     # uniform external force per atom
        return dpdx - self.n * f_ext

    def element(self, j, G, call_id):
        return dict(h=float(self.h[j]), dpdx=float(G), density=float(self.n[j]), T=self.T,
                    steps_eq=self.steps_eq, steps_sample=self.steps_sample, Lx=self.Lx, Lz=self.Lz,
                    g_ext=0.0, seed=self.seed, id=int(call_id))

    def continuity(self, q):
        A = self.h * self.Lz
        self.n = self.n - self.dt / A * (np.roll(q, -1) - np.roll(q, 1)) / (2.0 * self.dx)

    # ------------------------------------------------------------------ Alg. 1
    def step_sequential(self, sigma_t, md_fn):
        """One macro step exactly as Algorithm 1 orders it: for each section,
        a GP prediction on the current database; an MD run (appended at once,
        covariance refit) whenever the predicted sd exceeds sigma_t."""
        self.i += 1
        t = self.i * self.dt
        G = self.gradients(t)
        sn2 = self.sn2()
        q = np.zeros(self.N); sd = np.zeros(self.N); from_md = np.zeros(self.N, bool)
        for j in range(self.N):
            x = self.inputs(j, G)
            g = ogp.GP(self.X, self.y, self.sf2, self.l2, sn2, fallback=self.fallback)
            m, v = g.predict(x)
            sd[j] = math.sqrt(v[0])
            if ogp.gate(sd[j], sigma_t):
                r = md_fn(self.element(j, G[j], self.md_calls))
                self.md_calls += 1
                self.X = np.vstack([self.X, x])
                self.y = np.append(self.y, r["q"])
                self.se = np.append(self.se, r["q_se"])
                q[j] = r["q"]
                from_md[j] = True
            else:
                q[j] = m[0]
        self.continuity(q)
        return dict(q=q, sd=sd, from_md=from_md, G=G)

    def step_batched(self, sigma_t, md_batch_fn):
        """The same step with all MD runs of the step in one batch.  The gate
        depends only on the inputs X (the posterior variance does not involve
        y, and the scales of Eq. d2Eq come from X alone), so the set of MD
        sections is decided first; the means of the other sections are then
        taken with the database as Algorithm 1 would have it at that section
        (all MD results of earlier sections appended)."""
        self.i += 1
        t = self.i * self.dt
        G = self.gradients(t)
        sn2 = self.sn2()
        X0 = self.X
        Xv = self.X
        sd = np.zeros(self.N); from_md = np.zeros(self.N, bool)
        for j in range(self.N):
            x = self.inputs(j, G)
            g = ogp.GP(Xv, np.zeros(len(Xv)), self.sf2, self.l2, sn2, fallback=self.fallback)   # y does not enter the variance
            v = g.predict(x)[1]
            sd[j] = math.sqrt(v[0])
            if ogp.gate(sd[j], sigma_t):
                from_md[j] = True
                Xv = np.vstack([Xv, x])
        md_idx = np.nonzero(from_md)[0]
        els = [self.element(j, G[j], self.md_calls + k) for k, j in enumerate(md_idx)]
        res = md_batch_fn(els) if els else []
        self.md_calls += len(els)
        q = np.zeros(self.N)
        X, y, se = X0, self.y, self.se
        k = 0
        for j in range(self.N):
            if from_md[j]:
                q[j] = res[k]["q"]
                X = np.vstack([X, self.inputs(j, G)])
                y = np.append(y, res[k]["q"])
                se = np.append(se, res[k]["q_se"])
                k += 1
            else:
                g = ogp.GP(X, y, self.sf2, self.l2, sn2, fallback=self.fallback)
                q[j] = g.predict(self.inputs(j, G))[0][0]
        self.X, self.y, self.se = X, y, se
        self.continuity(q)
        return dict(q=q, sd=sd, from_md=from_md, G=G)


def relative_error(q_hist, Q_hist):
    """Eq. error: sum_i |qbar_i - Q_i| / sum_i |Q_i| over the time history of
    the section-averaged flow rate (the stray bracket in the printed equation
    dropped)."""
    q = np.asarray(q_hist, dtype=np.float64)
    Q = np.asarray(Q_hist, dtype=np.float64)
    return float(np.abs(q - Q).sum() / np.abs(Q).sum())


def speedup(t_end_steps, n_atoms_full, steps_per_sim, n_sims, mean_atoms_per_sim):
    """Eq. speedup: t_end N_af / (tbar_sim N_sim Nbar_ah)."""
    if n_sims == 0:
        return math.inf
    return float(t_end_steps * n_atoms_full / (steps_per_sim * n_sims * mean_atoms_per_sim))


# ---------------------------------------------------------------------------
# Algorithm 1's pseudoMD (Sec. 2.4): the start-up time t_s of a new MD run,
# from the 1D Navier-Stokes (here: unsteady Stokes) solution of a channel of
# height h with Navier slip, written as its eigenfunction series.
#
#   du/dt = nu d2u/dy2 + g,   u = slip du/dn at y = 0 and y = h,
#
# started at rest or at the steady profile of force g_from, driven by g_to.
# The steady profile is u(y) = g / (2 nu) (y (h - y) + slip h); with
# s = y - h/2 the deviation from it is a sum of cos(lam_k s) exp(-nu lam_k^2 t),
# theta_k = lam_k h / 2 the roots of theta tan(theta) = h / (2 slip) in
# (k pi, k pi + pi/2) (theta_k = (2k + 1) pi / 2 without slip).  The flow
# rate is Q = q_scale * integral_0^h u dy.  READING: the paper names the
# solver but not its end criterion; t_s is the first time at which
# |Q(t) - Q_inf| <= eps_q.  A negative slip puts no-slip planes -slip inside
# each wall (the layers next to the walls at rest): the channel of width
# h + 2 slip without slip.
# ---------------------------------------------------------------------------
def _pseudo_md_width(h, slip):
    return (h + 2.0 * slip, 0.0) if slip < 0.0 else (h, slip)


def pseudo_md_roots(h, slip, n_modes):
    """theta_k, k < n_modes: roots of theta tan(theta) = h / (2 slip)."""
    from scipy.optimize import brentq
    if slip == 0.0:
        return np.array([(2 * k + 1) * math.pi / 2 for k in range(n_modes)])
    bi = h / (2.0 * slip)
    f = lambda th: th * math.sin(th) - bi * math.cos(th)
    return np.array([brentq(f, k * math.pi, k * math.pi + math.pi / 2, xtol=1e-15, rtol=1e-15)
                     for k in range(n_modes)])


def pseudo_md_steady_flow(h, nu, slip, g, q_scale):
    """Q of the steady profile g / (2 nu) (y (h - y) + slip h)."""
    h, slip = _pseudo_md_width(h, slip)
    return q_scale * g / (2.0 * nu) * (h ** 3 / 6.0 + slip * h * h)


def pseudo_md_series(h, nu, slip, g_from, g_to, from_rest, q_scale, n_modes=400):
    """(rates nu lam_k^2, weights w_k): Q(t) - Q_inf = sum_k w_k exp(-rate_k t).
    Each coefficient is the projection of the initial deviation on the
    eigenfunction cos(lam_k s) (the eigenfunctions of the Robin problem are
    orthogonal): the numerator by oscillatory quadrature (QUADPACK's QAWO,
    scipy's weight='cos'), the norm h/2 + sin(2 theta_k) / (2 lam_k); the
    eigenfunction's flow-rate integral is 2 sin(theta_k) / lam_k."""
    from scipy.integrate import quad
    h, slip = _pseudo_md_width(h, slip)
    amp = (-g_to if from_rest else g_from - g_to) / (2.0 * nu)
    dev = lambda s: amp * (h * h / 4.0 - s * s + slip * h)   # s = y - h/2
    th = pseudo_md_roots(h, slip, n_modes)
    lam = 2.0 * th / h
    w = np.zeros(n_modes)
    for k in range(n_modes):
        num = quad(dev, -h / 2.0, h / 2.0, weight="cos", wvar=lam[k], epsabs=1e-15 * abs(amp) * h ** 3,
                   epsrel=1e-12, limit=200)[0]
        den = h / 2.0 + math.sin(2.0 * th[k]) / (2.0 * lam[k])
        w[k] = q_scale * num / den * (2.0 * math.sin(th[k]) / lam[k])
    return nu * lam ** 2, w


def pseudo_md_time(h, nu, slip, g_from, g_to, from_rest, q_scale, eps_q, n_modes=400):
    """t_s: the first t with |Q(t) - Q_inf| <= eps_q (the deviation decays
    monotonically: every weight has the sign of the initial deviation)."""
    from scipy.optimize import brentq
    rate, w = pseudo_md_series(h, nu, slip, g_from, g_to, from_rest, q_scale, n_modes)
    dq = lambda t: abs(float(np.sum(w * np.exp(-rate * t))))
    if dq(0.0) <= eps_q:
        return 0.0
    hi = 1.0 / rate[0]
    while dq(hi) > eps_q:
        hi *= 2.0
    return brentq(lambda t: dq(t) - eps_q, 0.0, hi, xtol=1e-14 * hi, rtol=1e-14)
