"""Algorithm 1 oracle: the batched form takes exactly the sequential form's
decisions and values; macro-model invariants (mass conservation, the
empty-database prior, thresholds above sigma_f)."""
import math

import numpy as np
import pytest

from oracle import hybrid


def fake_md(el):
    """Deterministic stand-in for an MD run: a smooth flow law in (h, G)
    plus a hashed perturbation, with a fixed standard error."""
    h, G = el["h"], el["dpdx"]
    noise = math.sin(12.9898 * el["id"] + 78.233 * h) * 0.05
    return {"q": -0.8 * h ** 3 * G / 24.0 + noise, "q_se": 0.05}


def fake_batch(els):
    return [fake_md(e) for e in els]


def channel(**kw):
    base = dict(n_sections=16, dx=50.0, h0=12.0, K=10.0, dP_amp=400.0, period=1000.0, dt=20.0,
                sf2=1.0, l2=1.0, sn2_default=0.05 ** 2)
    base.update(kw)
    return hybrid.Channel(**base)


@pytest.mark.parametrize("sigma_t", [0.05, 0.2, 0.5])
def test_batched_step_equals_sequential(sigma_t):
    a, b = channel(), channel()
    for step in range(12):
        ra = a.step_sequential(sigma_t, fake_md)
        rb = b.step_batched(sigma_t, fake_batch)
        assert (ra["from_md"] == rb["from_md"]).all(), step
        np.testing.assert_allclose(ra["sd"], rb["sd"], rtol=1e-10, atol=1e-13)
        np.testing.assert_allclose(ra["q"], rb["q"], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(a.n, b.n, rtol=1e-12)
    assert a.md_calls == b.md_calls > 0


def test_mass_is_conserved():
    c = channel()
    mass0 = (c.n * c.h * c.Lz * c.dx).sum()
    for _ in range(10):
        c.step_batched(0.2, fake_batch)
    assert (c.n * c.h * c.Lz * c.dx).sum() == pytest.approx(mass0, rel=1e-12)


def test_threshold_above_signal_never_runs_md():
    # empty database: sd = sigma_f everywhere; sigma_t > sigma_f -> prior mean 0 (paper Sec. 3.1)
    c = channel(sf2=0.36)
    for _ in range(3):
        r = c.step_sequential(0.61, fake_md)
        assert not r["from_md"].any()
        np.testing.assert_array_equal(r["q"], 0.0)
        np.testing.assert_allclose(r["sd"], 0.6)
    assert c.md_calls == 0


def test_zero_threshold_runs_md_everywhere():
    c = channel()
    r = c.step_batched(0.0, fake_batch)
    assert r["from_md"].all() or r["sd"].min() > 0   # every sd > 0 asks for MD
    assert c.md_calls == r["from_md"].sum()


def test_error_and_speedup_definitions():
    assert hybrid.relative_error([1.0, 2.0], [1.0, 4.0]) == pytest.approx(2.0 / 5.0)
    assert hybrid.speedup(1000, 5000, 100, 5, 1000) == pytest.approx(10.0)
    assert hybrid.speedup(1000, 5000, 100, 0, 1000) == math.inf


def _pressure_db(K=10.0, n0=0.8):
    # pre-simulation stand-in: a grid over (h, n) with the linear law plus a
    # small deterministic perturbation
    hs = np.linspace(6.0, 18.0, 5)
    ns = np.linspace(0.6, 1.0, 7)
    X = np.array([[h, n] for h in hs for n in ns])
    y = K * (X[:, 1] - n0) + 0.01 * np.sin(7.0 * X[:, 0] + 31.0 * X[:, 1])
    return X, y


@pytest.mark.parametrize("sigma_t", [0.05, 0.3])
def test_paper_inputs_and_pressure_gp_batched_equals_sequential(sigma_t):
    # the paper's form: q-GP on (h, n, F), pressure from the p-GP; the gate is
    # still a function of the inputs alone, so both orders agree
    X, y = _pressure_db()
    db = (X, y, 1.0, 1.0, 1e-4)
    a = channel(inputs=1, pressure_db=db)
    b = channel(inputs=1, pressure_db=db)
    for step in range(8):
        ra = a.step_sequential(sigma_t, fake_md)
        rb = b.step_batched(sigma_t, fake_batch)
        assert (ra["from_md"] == rb["from_md"]).all(), step
        np.testing.assert_allclose(ra["q"], rb["q"], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(a.n, b.n, rtol=1e-12)
    assert a.md_calls == b.md_calls > 0
    assert a.X.shape[1] == 3


def test_paper_inputs_rows_and_pressure_gp_interpolates():
    X, y = _pressure_db()
    c = channel(inputs=1, pressure_db=(X, y, 1.0, 1.0, 1e-6))
    # at its own data the p-GP mean is K (K + sn2 I)^-1 y = y - sn2 alpha
    # exactly, so it passes through the pre-simulations as sn2 -> 0
    np.testing.assert_allclose(c.pgp.predict(X)[0], y - 1e-6 * c.pgp.alpha, rtol=0, atol=1e-9)
    assert np.abs(c.pgp.predict(X)[0] - y).max() < 0.05
    # F = -G / n: the force per unit mass an element feels (Eq. momentumEq)
    G = c.gradients(20.0)
    x = c.inputs(3, G)
    np.testing.assert_allclose(x, [[c.h[3], c.n[3], -G[3] / c.n[3]]])
    # no pre-simulation data: the linear law
    d = channel(inputs=1)
    np.testing.assert_allclose(d.pressure(), d.K * (d.n - d.n0))


def _four_sections(**kw):
    # x_j = 0, 50, 100, 150 on L = 200: h = 12 (1 - 0.5 cos(2 pi x_j / L)) = 6, 12, 18, 12,
    # so A_j = h_j L_z = 60, 120, 180, 120
    base = dict(n_sections=4, dx=50.0, h0=12.0, Lz=10.0, K=10.0, n0=0.8, dt=20.0, dP_amp=400.0, period=1000.0)
    base.update(kw)
    return hybrid.Channel(**base)


def test_continuity_update_by_hand():
    # Eq. continuityEq with central differences: flow q_1 = 1 in +x at
    # section 1 carries mass out of the region around section 0 into the
    # region around section 2:
    #   dn_0 = -dt / A_0 (q_1 - q_3) / (2 dx) = -20 / 60 / 100 = -1/300
    #   dn_2 = -dt / A_2 (q_3 - q_1) / (2 dx) = +20 / 180 / 100 = +1/900
    c = _four_sections()
    np.testing.assert_allclose(c.h, [6.0, 12.0, 18.0, 12.0], rtol=1e-15)
    c.continuity(np.array([0.0, 1.0, 0.0, 0.0]))
    np.testing.assert_allclose(c.n - 0.8, [-1.0 / 300.0, 0.0, 1.0 / 900.0, 0.0], rtol=1e-12, atol=1e-16)


def test_pressure_gradient_and_forcing_by_hand():
    # p = K (n - n0) = 0, 1, 0, -1 for n = 0.8, 0.9, 0.8, 0.7; periodic central
    # differences (p_{j+1} - p_{j-1}) / (2 dx) = 0.02, 0, -0.02, 0.  A quarter
    # period in, the inlet-outlet difference is +dP_amp = 400, so the
    # external force on every atom is F_ext = 400 / (L n0) = 400 / 160 = 2.5
    # (Eq. momentumEq's F_ext, uniform over the channel); an element gets
    # G = dp/dx - n F_ext, and its body force F = -G / n = F_ext - p' / n
    # points downstream (+x).
    c = _four_sections(density0=[0.8, 0.9, 0.8, 0.7])
    np.testing.assert_allclose(c.pressure(), [0.0, 1.0, 0.0, -1.0], rtol=0, atol=1e-14)
    G = c.gradients(250.0)
    np.testing.assert_allclose(G, [0.02 - 2.0, -2.25, -0.02 - 2.0, -1.75], rtol=1e-13)
    from oracle import md
    for j, f in enumerate([2.5 - 0.02 / 0.8, 2.5, 2.5 + 0.02 / 0.8, 2.5]):
        assert md.make_params(c.element(j, G[j], 0)).g == pytest.approx(f, rel=1e-13)
    # no forcing at t = 0 and half a period
    np.testing.assert_allclose(c.gradients(0.0), [0.02, 0.0, -0.02, 0.0], rtol=1e-13, atol=1e-15)


# --- Algorithm 1's pseudoMD (Sec. 2.4): closed forms of the start-up ---

def test_pseudo_md_no_slip_first_mode_and_weight():
    # without slip the slowest mode decays at nu pi^2 / h^2 and carries
    # 96 / pi^4 of a start-up from rest (sum over odd k of 96 / (pi k)^4 = 1)
    h, nu = 8.0, 2.5
    rate, w = hybrid.pseudo_md_series(h, nu, 0.0, 0.0, 0.02, True, 80.0)
    assert rate[0] == pytest.approx(nu * math.pi ** 2 / h ** 2, rel=1e-14)
    assert rate[1] == pytest.approx(9.0 * nu * math.pi ** 2 / h ** 2, rel=1e-14)
    assert w[0] / w.sum() == pytest.approx(96.0 / math.pi ** 4, rel=1e-8)
    assert w[1] / w.sum() == pytest.approx(96.0 / (3.0 * math.pi) ** 4, rel=1e-6)


@pytest.mark.parametrize("slip", [0.0, 0.7, 3.0])
def test_pseudo_md_series_starts_at_the_initial_flow_rate(slip):
    # completeness: at t = 0 the series gives Q(0) - Q_inf with the steady
    # flow rate q_scale g (h^3 / 6 + slip h^2) / (2 nu), from rest and from
    # another force
    h, nu, qs = 6.0, 1.7, 55.0
    for g_from, g_to, rest in ((0.0, 0.03, True), (0.01, 0.03, False), (0.05, -0.02, False)):
        _, w = hybrid.pseudo_md_series(h, nu, slip, g_from, g_to, rest, qs)
        q0 = 0.0 if rest else qs * g_from * (h ** 3 / 6 + slip * h * h) / (2 * nu)
        qinf = qs * g_to * (h ** 3 / 6 + slip * h * h) / (2 * nu)
        assert hybrid.pseudo_md_steady_flow(h, nu, slip, g_to, qs) == pytest.approx(qinf, rel=1e-15)
        assert w.sum() == pytest.approx(q0 - qinf, rel=1e-7)


def test_pseudo_md_eigenvalues_solve_the_slip_condition():
    # u = slip du/dn with u = cos(lam (y - h/2)): cos(theta) = (2 slip / h) theta sin(theta)
    h, slip = 7.0, 0.9
    th = hybrid.pseudo_md_roots(h, slip, 30)
    resid = np.cos(th) - 2 * slip / h * th * np.sin(th)
    assert np.abs(resid / (1 + th)).max() < 1e-14
    assert np.all(np.diff(th) > 0) and np.all((th > np.arange(30) * math.pi) & (th < np.arange(30) * math.pi + math.pi / 2))


def test_pseudo_md_plug_flow_limit():
    # large slip: the flow is a plug that wall friction slows, dU/dt = -2 nu U / (h slip);
    # the next order of theta tan(theta) = Bi in Bi = h / (2 slip) divides the rate by 1 + Bi / 3
    h, nu, slip = 8.0, 2.5, 400.0
    rate, w = hybrid.pseudo_md_series(h, nu, slip, 0.0, 0.02, True, 80.0)
    assert rate[0] == pytest.approx(2 * nu / (h * slip), rel=5e-3)
    assert rate[0] == pytest.approx(2 * nu / (h * slip) / (1 + h / (6 * slip)), rel=1e-4)
    assert w[0] / w.sum() == pytest.approx(1.0, abs=1e-5)


def test_pseudo_md_time_no_slip_closed_form():
    # late start-up from rest without slip: |Q - Q_inf| ~ Q_inf (96/pi^4) exp(-nu pi^2 t / h^2)
    h, nu, qs, g = 10.0, 2.0, 80.0, 0.02
    qinf = hybrid.pseudo_md_steady_flow(h, nu, 0.0, g, qs)
    eps = 1e-4 * qinf
    t = hybrid.pseudo_md_time(h, nu, 0.0, 0.0, g, True, qs, eps)
    t_first = h ** 2 / (nu * math.pi ** 2) * math.log(96 / math.pi ** 4 * qinf / eps)
    assert t == pytest.approx(t_first, rel=1e-6)
    # nothing to wait for when the forces agree
    assert hybrid.pseudo_md_time(h, nu, 0.5, g, g, False, qs, eps) == 0.0


def test_pseudo_md_negative_slip_is_a_narrower_no_slip_channel():
    # READING: slip < 0 puts the no-slip planes -slip inside each wall
    h, nu, s = 10.0, 2.0, -0.8
    rate, w = hybrid.pseudo_md_series(h, nu, s, 0.0, 0.02, True, 80.0)
    assert rate[0] == pytest.approx(nu * math.pi ** 2 / (h + 2 * s) ** 2, rel=1e-14)
    assert hybrid.pseudo_md_steady_flow(h, nu, s, 0.02, 80.0) == pytest.approx(
        80.0 * 0.02 * (h + 2 * s) ** 3 / (12 * nu), rel=1e-14)
