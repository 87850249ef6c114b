"""Seeded synthetic workload generators shared by the tests, the benchmark and
the oracle runs.

This module only draws inputs (element descriptors, GP datasets, macro-case
settings); it contains none of the method's arithmetic.  All values are in
reduced Lennard-Jones units (eps = sigma = m = 1).

Workloads (shapes follow the paper's converging-diverging channel case and
its micro-element MD, App. A, at the sizes of the benchmark configurations):
  - element_plain: one 10 x 8 x 10 element, n = 0.8, T = 1.1, g = 0.02,
    2000 equilibration + 3000 sampling steps;
  - batch_uneven: 64 elements, h ~ U[5, 20], L_x, L_z ~ U[10, 16],
    500-5000 fluid atoms (rejection sampled at n = 0.8), g ~ U[0.005, 0.05],
    20 000 steps each;
  - batch_stress: 4096 elements, h ~ U[5, 40], n ~ U[0.7, 0.9], fluid atom
    counts log-uniform in [2k, 32k], 10 000 steps each;
  - gp_dataset: inputs (h, dp/dx) over the channel's range with a smooth
    synthetic response plus noise.
"""
import numpy as np

BASE_SEED = 20160315


def element_plain(seed=BASE_SEED, steps_eq=2000, steps_sample=3000, g=0.02, elem_id=0):
    return dict(h=8.0, Lx=10.0, Lz=10.0, density=0.8, T=1.1, g_ext=float(g), dpdx=0.0,
                steps_eq=int(steps_eq), steps_sample=int(steps_sample), seed=int(seed), id=int(elem_id))


def batch_uneven(n=64, seed=BASE_SEED, steps=20000, eq_fraction=0.2, nf_range=(500, 5000)):
    rng = np.random.default_rng(seed)
    out = []
    steps_eq = int(round(steps * eq_fraction))
    while len(out) < n:
        h = rng.uniform(5.0, 20.0)
        lx = rng.uniform(10.0, 16.0)
        lz = rng.uniform(10.0, 16.0)
        g = rng.uniform(0.005, 0.05)
        if not (nf_range[0] <= 0.8 * lx * h * lz <= nf_range[1]):
            continue
        k = len(out)
        out.append(dict(h=float(h), Lx=float(lx), Lz=float(lz), density=0.8, T=1.1, g_ext=float(g),
                        dpdx=0.0, steps_eq=steps_eq, steps_sample=int(steps) - steps_eq,
                        seed=int(seed) + k, id=k))
    return out


def batch_stress(n=4096, seed=BASE_SEED + 5, steps=10000, eq_fraction=0.2):
    rng = np.random.default_rng(seed)
    out = []
    steps_eq = int(round(steps * eq_fraction))
    for k in range(n):
        h = rng.uniform(5.0, 40.0)
        dens = rng.uniform(0.7, 0.9)
        nf = np.exp(rng.uniform(np.log(2000.0), np.log(32000.0)))
        lat = max(9.0, float(np.sqrt(nf / (dens * h))))
        g = rng.uniform(0.005, 0.05)
        out.append(dict(h=float(h), Lx=lat, Lz=lat, density=float(dens), T=1.1, g_ext=float(g),
                        dpdx=0.0, steps_eq=steps_eq, steps_sample=int(steps) - steps_eq,
                        seed=int(seed) + k, id=k))
    return out


def gp_dataset(M, seed=BASE_SEED, D=2, noise=0.05):
    """Inputs over the channel's (h, dp/dx) range and a smooth response."""
    rng = np.random.default_rng(seed)
    X = np.empty((M, D))
    X[:, 0] = rng.uniform(6.0, 18.0, M)
    for k in range(1, D):
        X[:, k] = rng.uniform(-0.05, 0.05, M)
    y = -X[:, 1] * X[:, 0] ** 2 * 4.0 + 0.3 * np.sin(X[:, 0]) + noise * rng.standard_normal(M)
    return X, y


def gp_queries(m, seed=BASE_SEED + 1, D=2):
    rng = np.random.default_rng(seed)
    Xs = np.empty((m, D))
    Xs[:, 0] = rng.uniform(5.0, 19.0, m)
    for k in range(1, D):
        Xs[:, k] = rng.uniform(-0.06, 0.06, m)
    return Xs


def hybrid_channel(n_sections=200, h0=12.0, dx=10.0, n_steps=100):
    """Macro settings of the converging-diverging channel case: h(x) =
    h0 (1 - 0.5 cos(2 pi x / L)) over n_sections periodic sections."""
    return dict(n_sections=int(n_sections), h0=float(h0), dx=float(dx), n_steps=int(n_steps))
