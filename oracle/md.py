"""ctypes front end of the FP64 micro-element oracle (md_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and bench.py's CPU-baseline
leg may import this module; the product package never does.

The element follows the paper's App. A (LJ fluid between walls, periodic in x
and z, velocity Verlet, Eq. LJ truncated at r_c) with the body force of
Sec. 2.1 Eq. momentumEq and the time-averaged flow rate of Eq. continuityEq.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_md.so")

MAXB = 64


class Params(ctypes.Structure):
    _fields_ = [
        ("h", ctypes.c_double), ("Lx", ctypes.c_double), ("Lz", ctypes.c_double),
        ("density", ctypes.c_double), ("T", ctypes.c_double), ("g", ctypes.c_double),
        ("dt", ctypes.c_double), ("rc", ctypes.c_double), ("k_tether", ctypes.c_double),
        ("gamma_wall", ctypes.c_double), ("wall_density", ctypes.c_double),
        ("eps_wf", ctypes.c_double), ("sig_wf", ctypes.c_double),
        ("eps_ww", ctypes.c_double), ("sig_ww", ctypes.c_double),
        ("fluid_margin", ctypes.c_double), ("tau_T", ctypes.c_double), ("mass", ctypes.c_double),
        ("steps_eq", ctypes.c_int64), ("steps_sample", ctypes.c_int64),
        ("seed", ctypes.c_uint64), ("elem_id", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
        ("mode", ctypes.c_int32), ("wall_planes", ctypes.c_int32), ("wall_amp", ctypes.c_double),
    ]


class Accum(ctypes.Structure):
    _fields_ = [
        ("q_block", ctypes.c_double * MAXB), ("p_block", ctypes.c_double * MAXB),
        ("n_block", ctypes.c_int64 * MAXB), ("T_sum", ctypes.c_double),
        ("n_samples", ctypes.c_int64), ("e_first", ctypes.c_double), ("e_last", ctypes.c_double),
        ("status", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_double), ("q_se", ctypes.c_double), ("p", ctypes.c_double),
        ("p_se", ctypes.c_double), ("T_meas", ctypes.c_double), ("e_drift", ctypes.c_double),
        ("n_fluid", ctypes.c_int64), ("n_wall", ctypes.c_int64), ("status", ctypes.c_int32),
    ]


# Physics defaults of the tethered-wall element (reduced LJ units).
DEFAULTS = dict(dt=0.005, rc=2.5, k_tether=150.0, gamma_wall=1.0, wall_density=1.0,
                eps_wf=1.0, sig_wf=1.0, eps_ww=1.0, sig_ww=1.0, fluid_margin=0.7,
                tau_T=0.5, mass=1.0, n_blocks=10, mode=0, wall_planes=3)


def build(force=False):
    """Compile md_oracle.c with gcc (no FMA contraction) into liboracle_md.so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        L.or_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        L.or_normals4.argtypes = [ctypes.c_uint32] * 4 + [ctypes.c_uint64, dp]
        L.or_n_fluid.argtypes = [ctypes.POINTER(Params)]
        L.or_n_fluid.restype = ctypes.c_int64
        L.or_n_wall.argtypes = [ctypes.POINTER(Params)]
        L.or_n_wall.restype = ctypes.c_int64
        L.or_init.argtypes = [ctypes.POINTER(Params), dp, dp, dp, ip]
        L.or_lj_energy.argtypes = [ctypes.c_double] * 3
        L.or_lj_energy.restype = ctypes.c_double
        L.or_lj_force.argtypes = [ctypes.c_double] * 3
        L.or_lj_force.restype = ctypes.c_double
        for name in ("or_lj_brute", "or_lj_cells"):
            getattr(L, name).argtypes = [ctypes.POINTER(Params), ctypes.c_int64, dp, ip, dp, dp, dp]
        L.or_forces.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, dp, dp, ip, ctypes.c_int, dp, dp, dp]
        L.or_simulate.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, dp, dp, dp, ip,
                                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(Accum)]
        L.or_simulate.restype = ctypes.c_int
        L.or_finalize.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Accum), ctypes.c_int64,
                                  ctypes.c_int64, ctypes.POINTER(Result)]
        L.or_element.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(Result)]
        L.or_element.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def make_params(element, **physics):
    """Params from an element dict (h, Lx, Lz, density, T, g or g_ext/dpdx,
    steps_eq, steps_sample, seed, id) and physics overrides.

    The body force follows Eq. momentumEq: F = F_ext - (m / rho) dp/dx with
    rho = m * density."""
    kw = dict(DEFAULTS)
    kw.update(physics)
    if "g" in element:
        g = float(element["g"])
    else:
        g = float(element.get("g_ext", 0.0)) - float(element.get("dpdx", 0.0)) / float(element["density"])
    p = Params()
    p.h, p.Lx, p.Lz = float(element["h"]), float(element["Lx"]), float(element["Lz"])
    p.density, p.T, p.g = float(element["density"]), float(element["T"]), g
    for k in ("dt", "rc", "k_tether", "gamma_wall", "wall_density", "eps_wf", "sig_wf", "eps_ww",
              "sig_ww", "fluid_margin", "tau_T", "mass"):
        setattr(p, k, float(kw[k]))
    p.steps_eq = int(element.get("steps_eq", 0))
    p.steps_sample = int(element.get("steps_sample", 0))
    p.seed = int(element.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    p.elem_id = int(element.get("id", 0))
    p.n_blocks, p.mode, p.wall_planes = int(kw["n_blocks"]), int(kw["mode"]), int(kw["wall_planes"])
    p.wall_amp = float(element.get("wall_amp", 0.0))
    return p


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals4(a, b, c, d, seed):
    out = np.zeros(4)
    lib().or_normals4(a, b, c, d, seed, _dp(out))
    return out


def lj_energy(r, eps=1.0, sig=1.0):
    return lib().or_lj_energy(r, eps, sig)


def lj_force(r, eps=1.0, sig=1.0):
    return lib().or_lj_force(r, eps, sig)


def counts(p):
    return int(lib().or_n_fluid(ctypes.byref(p))), int(lib().or_n_wall(ctypes.byref(p)))


def init(p):
    """Initial state: x, v, anchors (N x 3) and species (0 fluid, 1 wall)."""
    nf, nw = counts(p)
    n = nf + nw
    x = np.zeros((n, 3)); v = np.zeros((n, 3)); a = np.zeros((n, 3)); sp = np.zeros(n, np.int32)
    lib().or_init(ctypes.byref(p), _dp(x), _dp(v), _dp(a), _ip(sp))
    return x, v, a, sp


def lj_forces(p, x, sp, method="cells"):
    """LJ forces (N x 3), per-atom x-virial shares and per-atom energies."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    sp = np.ascontiguousarray(sp, dtype=np.int32)
    n = len(sp)
    f = np.zeros((n, 3)); w = np.zeros(n); e = np.zeros(n)
    fn = lib().or_lj_cells if method == "cells" else lib().or_lj_brute
    fn(ctypes.byref(p), n, _dp(x), _ip(sp), _dp(f), _dp(w), _dp(e))
    return f, w, e


def forces(p, x, anchor, sp, use_cells=True):
    """Total force (LJ + tether + body force), x-virial shares and energies."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    anchor = np.ascontiguousarray(anchor, dtype=np.float64)
    sp = np.ascontiguousarray(sp, dtype=np.int32)
    n = len(sp)
    f = np.zeros((n, 3)); w = np.zeros(n); e = np.zeros(n)
    lib().or_forces(ctypes.byref(p), n, _dp(x), _dp(anchor), _ip(sp), int(use_cells), _dp(f), _dp(w), _dp(e))
    return f, w, e


def simulate(p, x, v, anchor, sp, s0, s1, use_cells=True, acc=None):
    """Advance the state (modified in place) from step s0 to s1."""
    if acc is None:
        acc = Accum()
    assert x.flags.c_contiguous and v.flags.c_contiguous
    st = lib().or_simulate(ctypes.byref(p), len(sp), _dp(x), _dp(v), _dp(np.ascontiguousarray(anchor)),
                           _ip(np.ascontiguousarray(sp, dtype=np.int32)), s0, s1, int(use_cells),
                           ctypes.byref(acc))
    return acc, st


def finalize(p, acc):
    nf, nw = counts(p)
    r = Result()
    lib().or_finalize(ctypes.byref(p), ctypes.byref(acc), nf, nw, ctypes.byref(r))
    return {k: getattr(r, k) for k, _ in Result._fields_}


def element(p, use_cells=True):
    """Run one whole element; returns the result dict."""
    r = Result()
    lib().or_element(ctypes.byref(p), int(use_cells), ctypes.byref(r))
    return {k: getattr(r, k) for k, _ in Result._fields_}
