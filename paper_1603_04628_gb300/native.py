"""Thin ctypes binding of libmdgp.so (include/mdgp.h).  Argument marshalling
only: every step of the path runs in the library's CUDA kernels.  There is no
CPU fallback -- if the library is missing this module raises."""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmdgp.so")

MDGP_OK = 0
STATUS = {0: "MDGP_OK", -1: "MDGP_E_ARG", -2: "MDGP_E_NOMEM", -3: "MDGP_E_CUDA", -4: "MDGP_E_UNSTABLE",
          -5: "MDGP_E_NOTPD", -6: "MDGP_E_TIMEOUT", -7: "MDGP_E_STATE", -8: "MDGP_E_OVERFLOW",
          -9: "MDGP_E_SKIN", -10: "MDGP_E_LIMIT"}
PREC_FP64 = 0
PREC_FP32 = 1


class Element(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("dpdx", ctypes.c_double), ("density", ctypes.c_double),
                ("T", ctypes.c_double), ("steps_eq", ctypes.c_int64), ("steps_sample", ctypes.c_int64),
                ("Lx", ctypes.c_double), ("Lz", ctypes.c_double), ("g_ext", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("flags", ctypes.c_int32), ("id", ctypes.c_int32),
                ("wall_amp", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("q_se", ctypes.c_double), ("p", ctypes.c_double),
                ("p_se", ctypes.c_double), ("T_meas", ctypes.c_double), ("e_drift", ctypes.c_double),
                ("n_fluid", ctypes.c_int64), ("n_wall", ctypes.c_int64), ("status", ctypes.c_int32),
                ("start", ctypes.c_int32)]


class Start(ctypes.Structure):
    _fields_ = [("xv", ctypes.POINTER(ctypes.c_float)), ("n_fluid", ctypes.c_int64), ("n_wall", ctypes.c_int64),
                ("h", ctypes.c_double), ("Lx", ctypes.c_double), ("Lz", ctypes.c_double)]


class MDParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("rc", ctypes.c_double), ("k_tether", ctypes.c_double),
                ("gamma_wall", ctypes.c_double), ("wall_density", ctypes.c_double),
                ("eps_wf", ctypes.c_double), ("sig_wf", ctypes.c_double), ("eps_ww", ctypes.c_double),
                ("sig_ww", ctypes.c_double), ("fluid_margin", ctypes.c_double), ("tau_T", ctypes.c_double),
                ("mass", ctypes.c_double), ("n_blocks", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("wall_planes", ctypes.c_int32), ("list_capacity", ctypes.c_int32),
                ("skin", ctypes.c_double), ("rebuild_every", ctypes.c_int32), ("build_variant", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("wait_timeout_ms", ctypes.c_int32),
                ("inject_barrier_skip", ctypes.c_int32), ("threads_per_atom", ctypes.c_int32),
                ("resident", ctypes.c_int32)]


class GPParams(ctypes.Structure):
    _fields_ = [("sf2", ctypes.c_double), ("l2", ctypes.c_double), ("sn2", ctypes.c_double),
                ("fallback_scale", ctypes.c_double), ("fixed_scales", ctypes.POINTER(ctypes.c_double)),
                ("fallback_scales", ctypes.POINTER(ctypes.c_double)), ("period", ctypes.c_double),
                ("hold", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class MacroParams(ctypes.Structure):
    _fields_ = [("n_sections", ctypes.c_int32), ("sn2_from_data", ctypes.c_int32),
                ("dx", ctypes.c_double), ("h0", ctypes.c_double), ("Lx", ctypes.c_double), ("Lz", ctypes.c_double),
                ("eos_K", ctypes.c_double), ("eos_n0", ctypes.c_double), ("dP_amp", ctypes.c_double),
                ("period", ctypes.c_double), ("dt", ctypes.c_double), ("T", ctypes.c_double),
                ("md_steps_eq", ctypes.c_int64), ("md_steps_sample", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("sf2", ctypes.c_double), ("l2", ctypes.c_double), ("sn2", ctypes.c_double),
                ("inputs", ctypes.c_int32), ("factor_cache_mb", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("reserved2", ctypes.c_int32), ("md_steps_eq_warm", ctypes.c_int64),
                ("pseudo_nu", ctypes.c_double), ("pseudo_slip", ctypes.c_double), ("pseudo_eps_q", ctypes.c_double),
                ("h_amp", ctypes.c_double)]


class HybridStats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("t", ctypes.c_double), ("md_runs", ctypes.c_int32),
                ("md_warm", ctypes.c_int32), ("md_runs_total", ctypes.c_int64), ("db_size", ctypes.c_int64),
                ("md_atoms", ctypes.c_int64), ("q_mean", ctypes.c_double), ("max_sd", ctypes.c_double),
                ("gp_seconds", ctypes.c_double), ("md_seconds", ctypes.c_double),
                ("md_steps_eq_warm", ctypes.c_int64)]


MEAN_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                           ctypes.POINTER(ctypes.c_double))


class MLPParams(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("eval_every", ctypes.c_int32), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("holdout_frac", ctypes.c_double), ("seed", ctypes.c_uint64)]


class MdgpError(RuntimeError):
    pass


_lib = None


def lib():
    """Load libmdgp.so (built by paper_1603_04628_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise MdgpError("CUDA library %s is not built; run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    sig = {
        "mdgp_start_state": ([ctypes.POINTER(MDParams), ctypes.POINTER(Element), ctypes.POINTER(Start),
                              ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "mdgp_pseudo_md": ([ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
                           ctypes.c_int),
        "mdgp_micro_direct_timing": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "mdgp_hybrid_set_database": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int64], ctypes.c_int),
        "mdgp_hybrid_save": ([ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int32], ctypes.c_int),
        "mdgp_hybrid_load": ([ctypes.c_void_p, ctypes.c_char_p], ctypes.c_int),
        "mdgp_md_params_default": ([ctypes.POINTER(MDParams)], ctypes.c_int),
        "mdgp_create": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "mdgp_destroy": ([vp], ctypes.c_int),
        "mdgp_set_md_params": ([vp, ctypes.POINTER(MDParams)], ctypes.c_int),
        "mdgp_set_stream": ([vp, vp], ctypes.c_int),
        "mdgp_micro_batch": ([vp, ctypes.POINTER(Element), i64, ctypes.POINTER(Result)], ctypes.c_int),
        "mdgp_micro_plan": ([vp, ctypes.POINTER(Element), i64, ctypes.POINTER(i64)], ctypes.c_int),
        "mdgp_micro_plan_from": ([vp, ctypes.POINTER(Element), i64, ctypes.POINTER(Start), ctypes.POINTER(i64)],
                                 ctypes.c_int),
        "mdgp_micro_launch": ([vp], ctypes.c_int),
        "mdgp_micro_results": ([vp, ctypes.POINTER(Result), i64], ctypes.c_int),
        "mdgp_micro_launch_count": ([vp], i64),
        "mdgp_micro_rebuild_count": ([vp], i64),
        "mdgp_micro_path": ([vp], ctypes.c_int),
        "mdgp_micro_launch_shape": ([vp, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "mdgp_micro_continue": ([vp, dp, dp], ctypes.c_int),
        "mdgp_micro_state": ([vp, dp, dp, i64], ctypes.c_int),
        "mdgp_md_forces": ([vp, ctypes.POINTER(Element), dp, i64, dp, dp, dp], ctypes.c_int),
        "mdgp_micro_profile": ([vp, i64, dp], ctypes.c_int),
        "mdgp_autotune": ([vp, ctypes.POINTER(Element), i64, i64, ctypes.POINTER(MDParams), dp], ctypes.c_int),
        "mdgp_last_error": ([vp], ctypes.c_char_p),
        "mdgp_gp_fit": ([vp, dp, dp, i64, ctypes.c_int32, ctypes.POINTER(GPParams), dp, ctypes.POINTER(vp)],
                        ctypes.c_int),
        "mdgp_gp_fit_inputs": ([vp, dp, i64, ctypes.c_int32, ctypes.POINTER(GPParams), ctypes.POINTER(vp)],
                               ctypes.c_int),
        "mdgp_gp_set_outputs": ([vp, dp, dp], ctypes.c_int),
        "mdgp_gp_predict": ([vp, dp, i64, dp, dp, dp], ctypes.c_int),
        "mdgp_gp_scales": ([vp, dp], ctypes.c_int),
        "mdgp_gp_log_marginal": ([vp, dp], ctypes.c_int),
        "mdgp_gp_optimize": ([vp, dp, dp, i64, ctypes.c_int32, ctypes.POINTER(GPParams), dp, ctypes.c_int32,
                              ctypes.POINTER(GPParams), dp], ctypes.c_int),
        "mdgp_gp_free": ([vp], ctypes.c_int),
        "mdgp_macro_params_default": ([ctypes.POINTER(MacroParams)], ctypes.c_int),
        "mdgp_hybrid_create": ([vp, ctypes.POINTER(MacroParams), dp, ctypes.POINTER(vp)], ctypes.c_int),
        "mdgp_hybrid_set_mean": ([vp, MEAN_FN, vp], ctypes.c_int),
        "mdgp_hybrid_step": ([vp, ctypes.c_double, ctypes.POINTER(HybridStats)], ctypes.c_int),
        "mdgp_hybrid_state": ([vp, dp, dp, dp, ctypes.POINTER(ctypes.c_int32), dp], ctypes.c_int),
        "mdgp_hybrid_database": ([vp, dp, dp, dp, i64, ctypes.POINTER(i64)], ctypes.c_int),
        "mdgp_hybrid_set_pressure": ([vp, dp, dp, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double],
                                     ctypes.c_int),
        "mdgp_hybrid_free": ([vp], ctypes.c_int),
        "mdgp_mlp_params_default": ([ctypes.POINTER(MLPParams)], ctypes.c_int),
        "mdgp_mlp_num_params": ([], ctypes.c_int),
        "mdgp_mlp_create": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.c_uint64, ctypes.POINTER(vp)], ctypes.c_int),
        "mdgp_mlp_free": ([vp], ctypes.c_int),
        "mdgp_mlp_train": ([vp, dp, dp, i64, ctypes.POINTER(MLPParams), dp, dp], ctypes.c_int),
        "mdgp_mlp_predict": ([vp, dp, i64, dp], ctypes.c_int),
        "mdgp_mlp_loss_grad": ([vp, dp, dp, i64, dp, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "mdgp_mlp_adam_step": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(MLPParams)], ctypes.c_int),
        "mdgp_mlp_get": ([vp, ctypes.POINTER(ctypes.c_float), dp], ctypes.c_int),
        "mdgp_mlp_set": ([vp, ctypes.POINTER(ctypes.c_float), dp], ctypes.c_int),
        "mdgp_hybrid_set_mlp_mean": ([vp, vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(ctx, st, what):
    if st != MDGP_OK:
        msg = lib().mdgp_last_error(ctx) if ctx else b""
        raise MdgpError("%s failed: %s (%s)" % (what, STATUS.get(st, st), (msg or b"").decode()))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def to_element(d):
    e = Element()
    e.h, e.dpdx, e.density, e.T = float(d["h"]), float(d.get("dpdx", 0.0)), float(d["density"]), float(d["T"])
    e.steps_eq, e.steps_sample = int(d.get("steps_eq", 0)), int(d.get("steps_sample", 0))
    e.Lx, e.Lz, e.g_ext = float(d["Lx"]), float(d["Lz"]), float(d.get("g_ext", d.get("g", 0.0)))
    e.seed = int(d.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    e.flags = int(d.get("flags", 0))
    e.id = int(d.get("id", 0))
    e.wall_amp = float(d.get("wall_amp", 0.0))
    return e


def elements_array(els):
    arr = (Element * len(els))()
    for i, d in enumerate(els):
        arr[i] = to_element(d)
    return arr


def result_dict(r):
    return {k: getattr(r, k) for k, _ in Result._fields_ if k != "reserved"}


def md_params_default():
    p = MDParams()
    _check(None, lib().mdgp_md_params_default(ctypes.byref(p)), "mdgp_md_params_default")
    return p


def _start(s, st, keep):
    """Fill the Start struct st from a snapshot dict (xv rows, n_fluid,
    n_wall, h, Lx, Lz); keep holds the float32 copy alive."""
    xv = np.ascontiguousarray(s["xv"], dtype=np.float32)
    keep.append(xv)
    st.xv = xv.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    st.n_fluid, st.n_wall = int(s["n_fluid"]), int(s["n_wall"])
    st.h, st.Lx, st.Lz = float(s["h"]), float(s["Lx"]), float(s["Lz"])


def pseudo_md(h, nu, slip, g_from, g_to, from_rest, q_scale, eps_q):
    """mdgp_pseudo_md (host only): Algorithm 1's start-up time t_s."""
    t = ctypes.c_double()
    _check(None, lib().mdgp_pseudo_md(float(h), float(nu), float(slip), float(g_from), float(g_to),
                                      int(bool(from_rest)), float(q_scale), float(eps_q), ctypes.byref(t)),
           "mdgp_pseudo_md")
    return t.value


def start_state(el, snap, **md_params):
    """mdgp_start_state (host only): the start state mdgp_micro_plan_from
    gives element el from snapshot snap; returns (rows x 6 array, 1) or
    (None, 0) for a cold start."""
    p = md_params_default()
    for k, v in md_params.items():
        setattr(p, k, v)
    e = to_element(el)
    st, keep = Start(), []
    _start(snap, st, keep)
    rows, kind = ctypes.c_int64(), ctypes.c_int32(0)
    _check(None, lib().mdgp_start_state(ctypes.byref(p), ctypes.byref(e), ctypes.byref(st), None, 0,
                                        ctypes.byref(rows), ctypes.byref(kind)), "mdgp_start_state")
    out = np.zeros((rows.value, 6))
    _check(None, lib().mdgp_start_state(ctypes.byref(p), ctypes.byref(e), ctypes.byref(st),
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), rows.value,
                                        ctypes.byref(rows), ctypes.byref(kind)), "mdgp_start_state")
    return (out, 1) if kind.value else (None, 0)


class Context:
    """Owns one mdgp_ctx (device buffers, stream, captured graphs)."""

    def __init__(self, device=0, precision=PREC_FP64, stream=None, **md_params):
        self.h = ctypes.c_void_p()
        _check(None, lib().mdgp_create(ctypes.byref(self.h), int(device), int(precision)), "mdgp_create")
        self.precision = precision
        if md_params:
            self.set_md_params(**md_params)
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if self.h:
            lib().mdgp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_md_params(self, **kw):
        p = md_params_default()
        names = {f for f, _ in MDParams._fields_}
        for k, v in kw.items():
            if k not in names:
                raise MdgpError("unknown MD parameter %r" % k)
            setattr(p, k, v)
        _check(self.h, lib().mdgp_set_md_params(self.h, ctypes.byref(p)), "mdgp_set_md_params")

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        _check(self.h, lib().mdgp_set_stream(self.h, ctypes.c_void_p(int(handle))), "mdgp_set_stream")

    def micro_batch(self, els):
        arr = elements_array(els)
        out = (Result * len(els))()
        _check(self.h, lib().mdgp_micro_batch(self.h, arr, len(els), out), "mdgp_micro_batch")
        return [result_dict(r) for r in out]

    def micro_plan(self, els):
        arr = elements_array(els)
        n = ctypes.c_int64()
        _check(self.h, lib().mdgp_micro_plan(self.h, arr, len(els), ctypes.byref(n)), "mdgp_micro_plan")
        self._n_el = len(els)
        self.n_atoms = int(n.value)
        return self.n_atoms

    def micro_plan_from(self, els, starts):
        """mdgp_micro_plan_from: starts[k] is None (cold) or a dict with the
        snapshot rows xv ((n_fluid + n_wall) x 6, fluid first: x y z vx vy vz)
        and the geometry h, Lx, Lz it was taken in."""
        arr = elements_array(els)
        st = (Start * len(els))()
        keep = []
        for k, s in enumerate(starts):
            if s is not None:
                _start(s, st[k], keep)
        n = ctypes.c_int64()
        _check(self.h, lib().mdgp_micro_plan_from(self.h, arr, len(els), st, ctypes.byref(n)), "mdgp_micro_plan_from")
        self._n_el = len(els)
        self.n_atoms = int(n.value)
        return self.n_atoms

    def micro_launch(self):
        _check(self.h, lib().mdgp_micro_launch(self.h), "mdgp_micro_launch")

    def micro_results(self):
        out = (Result * self._n_el)()
        _check(self.h, lib().mdgp_micro_results(self.h, out, self._n_el), "mdgp_micro_results")
        return [result_dict(r) for r in out]

    def launch_count(self):
        return int(lib().mdgp_micro_launch_count(self.h))

    def rebuild_count(self):
        return int(lib().mdgp_micro_rebuild_count(self.h))

    def path(self):
        """Step loop of the planned batch: 'per-step', 'persistent-graph' or
        'persistent-direct'."""
        code = int(lib().mdgp_micro_path(self.h))
        if code < 0:
            raise MdgpError("mdgp_micro_path: %s" % STATUS.get(code, code))
        return {0: "per-step", 1: "persistent-graph", 2: "persistent-direct"}[code]

    def micro_continue(self, g_ext=None, dpdx=None):
        """Run the planned batch for another plan's worth of steps from the
        state the last launch left (mdgp_micro_continue), optionally with new
        per-element forcing."""
        arrays = [None if v is None else
                  np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), (self._n_el,)))
                  for v in (g_ext, dpdx)]   # alive until the call returns
        ga, da = (None if a is None else _dp(a) for a in arrays)
        _check(self.h, lib().mdgp_micro_continue(self.h, ga, da), "mdgp_micro_continue")

    def launch_shape(self):
        """The persistent step kernel's launch: blocks, threads per block,
        atoms per block, threads per atom and whether the atoms are kept
        resident (mdgp_micro_launch_shape)."""
        out = (ctypes.c_int32 * 5)()
        _check(self.h, lib().mdgp_micro_launch_shape(self.h, out), "mdgp_micro_launch_shape")
        return {"blocks": out[0], "threads": out[1], "atoms_per_block": out[2], "threads_per_atom": out[3],
                "resident": out[4]}

    def micro_state(self):
        x = np.zeros((self.n_atoms, 3))
        v = np.zeros((self.n_atoms, 3))
        _check(self.h, lib().mdgp_micro_state(self.h, _dp(x), _dp(v), self.n_atoms), "mdgp_micro_state")
        return x, v

    def autotune(self, els, probe_steps=400):
        """Pick skin and list-build variant for this batch by timing; returns
        (chosen parameters as a dict, atom-steps/s of the best probe)."""
        arr = elements_array(els)
        best = MDParams()
        rate = ctypes.c_double()
        _check(self.h, lib().mdgp_autotune(self.h, arr, len(els), int(probe_steps), ctypes.byref(best),
                                           ctypes.byref(rate)), "mdgp_autotune")
        return {k: getattr(best, k) for k, _ in MDParams._fields_}, rate.value

    def direct_timing(self):
        """mdgp_micro_direct_timing: CUDA-event times of the last batch's
        host-launched persistent kernels (persistent = 2)."""
        out = np.zeros(5)
        _check(self.h, lib().mdgp_micro_direct_timing(self.h, _dp(out)), "mdgp_micro_direct_timing")
        return dict(kernel_ms=float(out[0]), steps=int(out[1]), launches=int(out[2]), rebuild_ms=float(out[3]),
                    rebuilds=int(out[4]))

    def micro_profile(self, steps=100):
        """Mean per-launch milliseconds of the integration and pair-force kernels."""
        ms = np.zeros(6)
        _check(self.h, lib().mdgp_micro_profile(self.h, int(steps), _dp(ms)), "mdgp_micro_profile")
        return dict(integrate_ms=float(ms[0]), force_ms=float(ms[1]), rebuild_ms=float(ms[2]),
                    atoms=int(ms[3]), cells=int(ms[4]), rebuild_every=int(ms[5]))

    def md_forces(self, el, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = len(x)
        f = np.zeros((n, 3)); w = np.zeros(n); e = np.zeros(n)
        e1 = to_element(el)
        _check(self.h, lib().mdgp_md_forces(self.h, ctypes.byref(e1), _dp(x), n, _dp(f), _dp(w), _dp(e)),
               "mdgp_md_forces")
        return f, w, e


class GP:
    """A fitted Gaussian process (mdgp_gp) living on ctx's device.  With
    y=None only the inputs are factored (mdgp_gp_fit_inputs); set_outputs
    adds the outputs later on the same factor."""

    def __init__(self, ctx, X, y, sf2, l2, sn2, mu_X=None, fallback_scale=1.0, fixed_scales=None,
                 fallback_scales=None, period=0.0):
        M = len(X) if y is None else len(y)
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(M, -1) if M else
                                 np.zeros((0, np.asarray(X).shape[-1] if np.ndim(X) == 2 else 1)))
        self.D = X.shape[1]
        p = GPParams(float(sf2), float(l2), float(sn2), float(fallback_scale), None, None, float(period), 0, 0)
        self._fb = None
        if fallback_scales is not None:
            self._fb = np.ascontiguousarray(fallback_scales, dtype=np.float64)
            p.fallback_scales = _dp(self._fb)
        self._fixed = None
        if fixed_scales is not None:
            self._fixed = np.ascontiguousarray(fixed_scales, dtype=np.float64)
            p.fixed_scales = _dp(self._fixed)
        self.h = ctypes.c_void_p()
        self.ctx = ctx
        self.M = M
        if y is None:
            _check(ctx.h, lib().mdgp_gp_fit_inputs(ctx.h, _dp(X), M, self.D, ctypes.byref(p),
                                                   ctypes.byref(self.h)), "mdgp_gp_fit_inputs")
            return
        y = np.ascontiguousarray(y, dtype=np.float64)
        mu = None if mu_X is None else _dp(np.ascontiguousarray(mu_X, dtype=np.float64))
        _check(ctx.h, lib().mdgp_gp_fit(ctx.h, _dp(X), _dp(y), M, self.D, ctypes.byref(p), mu,
                                        ctypes.byref(self.h)), "mdgp_gp_fit")

    def set_outputs(self, y, mu_X=None):
        y = np.ascontiguousarray(y, dtype=np.float64)
        if len(y) != self.M:
            raise ValueError("set_outputs: %d outputs for %d inputs" % (len(y), self.M))
        mu = None if mu_X is None else _dp(np.ascontiguousarray(mu_X, dtype=np.float64))
        _check(None, lib().mdgp_gp_set_outputs(self.h, _dp(y), mu), "mdgp_gp_set_outputs")

    def predict(self, Xs, mu_Xs=None, var=True):
        """Posterior (mean, var) at Xs; with var=False the means alone
        (no variance solve) and None for var."""
        Xs = np.ascontiguousarray(np.asarray(Xs, dtype=np.float64).reshape(-1, self.D))
        m = len(Xs)
        mean = np.zeros(m)
        v = np.zeros(m) if var else None
        mu = None if mu_Xs is None else _dp(np.ascontiguousarray(mu_Xs, dtype=np.float64))
        _check(None, lib().mdgp_gp_predict(self.h, _dp(Xs), m, mu, _dp(mean), None if v is None else _dp(v)),
               "mdgp_gp_predict")
        return mean, v

    def log_marginal(self):
        out = ctypes.c_double()
        _check(None, lib().mdgp_gp_log_marginal(self.h, ctypes.byref(out)), "mdgp_gp_log_marginal")
        return out.value

    def scales(self):
        out = np.zeros(self.D)
        _check(None, lib().mdgp_gp_scales(self.h, _dp(out)), "mdgp_gp_scales")
        return out

    def close(self):
        if self.h:
            lib().mdgp_gp_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hybrid:
    """One hybrid case (mdgp_hybrid): macro state, database, Algorithm 1 steps."""

    def __init__(self, ctx, density0=None, **params):
        p = MacroParams()
        _check(None, lib().mdgp_macro_params_default(ctypes.byref(p)), "mdgp_macro_params_default")
        names = {f for f, _ in MacroParams._fields_}
        for k, v in params.items():
            if k not in names:
                raise MdgpError("unknown macro parameter %r" % k)
            setattr(p, k, v)
        self.N = p.n_sections
        self.D = 3 if p.inputs == 1 else 2
        self.ctx = ctx
        self.h = ctypes.c_void_p()
        d0 = None
        if density0 is not None:
            self._d0 = np.ascontiguousarray(density0, dtype=np.float64)
            d0 = _dp(self._d0)
        _check(ctx.h, lib().mdgp_hybrid_create(ctx.h, ctypes.byref(p), d0, ctypes.byref(self.h)),
               "mdgp_hybrid_create")
        self._mean_cb = None

    def set_mean(self, fn):
        """fn(X (m x D) -> (m,)) as the GP prior mean, or None."""
        if fn is None:
            self._mean_cb = None
            _check(self.ctx.h, lib().mdgp_hybrid_set_mean(self.h, MEAN_FN(), None), "mdgp_hybrid_set_mean")
            return

        def cb(user, x, m, out):
            try:
                X = np.ctypeslib.as_array(x, shape=(m, self.D)).copy() if m else np.zeros((0, self.D))
                v = np.asarray(fn(X), dtype=np.float64).reshape(m)
                ctypes.memmove(out, v.ctypes.data, 8 * m)
                return 0
            except Exception:
                return -1
        self._mean_cb = MEAN_FN(cb)
        _check(self.ctx.h, lib().mdgp_hybrid_set_mean(self.h, self._mean_cb, None), "mdgp_hybrid_set_mean")

    def set_mlp_mean(self, mlp):
        self._mlp = mlp
        _check(self.ctx.h, lib().mdgp_hybrid_set_mlp_mean(self.h, mlp.h if mlp is not None else None),
               "mdgp_hybrid_set_mlp_mean")

    def step(self, sigma_t):
        st = HybridStats()
        _check(self.ctx.h, lib().mdgp_hybrid_step(self.h, float(sigma_t), ctypes.byref(st)), "mdgp_hybrid_step")
        return {k: getattr(st, k) for k, _ in HybridStats._fields_ if k != "reserved"}

    def state(self):
        n = np.zeros(self.N); q = np.zeros(self.N); sd = np.zeros(self.N); G = np.zeros(self.N)
        fm = np.zeros(self.N, np.int32)
        _check(None, lib().mdgp_hybrid_state(self.h, _dp(n), _dp(q), _dp(sd),
                                             fm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(G)),
               "mdgp_hybrid_state")
        return dict(density=n, q=q, sd=sd, from_md=fm.astype(bool), G=G)

    def set_database(self, X, y, se=None):
        """mdgp_hybrid_set_database: start from an earlier case's database."""
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, self.D)
        y = np.ascontiguousarray(y, dtype=np.float64)
        s = None if se is None else np.ascontiguousarray(se, dtype=np.float64)
        _check(self.ctx.h, lib().mdgp_hybrid_set_database(self.h, _dp(X), _dp(y), None if s is None else _dp(s),
                                                          len(y)), "mdgp_hybrid_set_database")

    def save(self, path, snapshots=True):
        _check(self.ctx.h, lib().mdgp_hybrid_save(self.h, os.fsencode(path), int(bool(snapshots))),
               "mdgp_hybrid_save")

    def load(self, path):
        _check(self.ctx.h, lib().mdgp_hybrid_load(self.h, os.fsencode(path)), "mdgp_hybrid_load")

    def database(self):
        M = ctypes.c_int64()
        _check(None, lib().mdgp_hybrid_database(self.h, None, None, None, 0, ctypes.byref(M)), "db size")
        m = M.value
        X = np.zeros((m, self.D)); y = np.zeros(m); se = np.zeros(m)
        _check(None, lib().mdgp_hybrid_database(self.h, _dp(X), _dp(y), _dp(se), m, ctypes.byref(M)),
               "mdgp_hybrid_database")
        return X, y, se

    def set_pressure(self, X, y, sf2, l2, sn2):
        """Pressure GP over (h, n) from pre-simulations (empty X: linear law)."""
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, 2))
        y = np.ascontiguousarray(y, dtype=np.float64)
        _check(self.ctx.h, lib().mdgp_hybrid_set_pressure(self.h, _dp(X) if len(y) else None,
                                                          _dp(y) if len(y) else None, len(y), float(sf2),
                                                          float(l2), float(sn2)), "mdgp_hybrid_set_pressure")

    def close(self):
        if self.h:
            lib().mdgp_hybrid_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_ORDER = [("W1", (64, 2)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (1, 64)), ("b3", (1,))]


def mlp_flatten(params):
    return np.concatenate([np.asarray(params[k], dtype=np.float32).reshape(-1) for k, _ in MLP_ORDER])


def mlp_unflatten(flat):
    out, off = {}, 0
    for k, shp in MLP_ORDER:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[off:off + n], dtype=np.float64).reshape(shp)
        off += n
    return out


def mlp_params_default(**kw):
    p = MLPParams()
    _check(None, lib().mdgp_mlp_params_default(ctypes.byref(p)), "mdgp_mlp_params_default")
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class MLP:
    """The learned prior mean (mdgp_mlp) on ctx's device."""

    def __init__(self, ctx, params=None, seed=1):
        self.ctx = ctx
        self.h = ctypes.c_void_p()
        init = None
        if params is not None:
            self._init = mlp_flatten(params)
            init = self._init.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        _check(ctx.h, lib().mdgp_mlp_create(ctx.h, init, int(seed), ctypes.byref(self.h)), "mdgp_mlp_create")

    def train(self, X, y, **kw):
        X = np.ascontiguousarray(X, dtype=np.float64); y = np.ascontiguousarray(y, dtype=np.float64)
        p = mlp_params_default(**kw)
        tl = ctypes.c_double(); hl = ctypes.c_double()
        _check(None, lib().mdgp_mlp_train(self.h, _dp(X), _dp(y), len(y), ctypes.byref(p), ctypes.byref(tl),
                                          ctypes.byref(hl)), "mdgp_mlp_train")
        return tl.value, hl.value

    def predict(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        out = np.zeros(len(X))
        _check(None, lib().mdgp_mlp_predict(self.h, _dp(X), len(X), _dp(out)), "mdgp_mlp_predict")
        return out

    def loss_grad(self, X, y):
        X = np.ascontiguousarray(X, dtype=np.float64); y = np.ascontiguousarray(y, dtype=np.float64)
        g = np.zeros(lib().mdgp_mlp_num_params(), np.float32)
        loss = ctypes.c_double()
        _check(None, lib().mdgp_mlp_loss_grad(self.h, _dp(X), _dp(y), len(y), ctypes.byref(loss),
                                              g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "mdgp_mlp_loss_grad")
        return loss.value, mlp_unflatten(g)

    def adam_step(self, grads, **kw):
        g = mlp_flatten(grads)
        p = mlp_params_default(**kw)
        _check(None, lib().mdgp_mlp_adam_step(self.h, g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              ctypes.byref(p)), "mdgp_mlp_adam_step")

    def get(self):
        w = np.zeros(lib().mdgp_mlp_num_params(), np.float32)
        st = np.zeros(6)
        _check(None, lib().mdgp_mlp_get(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _dp(st)),
               "mdgp_mlp_get")
        return mlp_unflatten(w), st

    def close(self):
        if self.h:
            lib().mdgp_mlp_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Same names as the C ABI.
def mdgp_create(device=0, precision=PREC_FP64):
    return Context(device, precision)


def mdgp_micro_batch(ctx, elements):
    return ctx.micro_batch(elements)


def mdgp_gp_fit(ctx, X, y, sf2, l2, sn2, mu_X=None, **kw):
    return GP(ctx, X, y, sf2, l2, sn2, mu_X=mu_X, **kw)


def mdgp_gp_predict(gp, Xs, mu_Xs=None):
    return gp.predict(Xs, mu_Xs)


def mdgp_hybrid_create(ctx, density0=None, **params):
    return Hybrid(ctx, density0, **params)


def mdgp_hybrid_step(hybrid, sigma_t):
    return hybrid.step(sigma_t)


def gp_optimize(ctx, X, y, sf2, l2, sn2, mu_X=None, fallback_scale=1.0, fallback_scales=None, max_evals=200,
                period=0.0, hold=0):
    """mdgp_gp_optimize: hyperparameters (sf2, l2, sn2) by maximum evidence;
    hold = bit mask of values kept (1 sf2, 2 l2, 4 sn2)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(len(y), -1))
    start = GPParams(float(sf2), float(l2), float(sn2), float(fallback_scale), None, None, float(period), int(hold), 0)
    fb = None
    if fallback_scales is not None:
        fb = np.ascontiguousarray(fallback_scales, dtype=np.float64)
        start.fallback_scales = _dp(fb)
    best = GPParams()
    lml = ctypes.c_double()
    mu = None if mu_X is None else np.ascontiguousarray(mu_X, dtype=np.float64)
    _check(ctx.h, lib().mdgp_gp_optimize(ctx.h, _dp(X), _dp(y), len(y), X.shape[1], ctypes.byref(start),
                                         _dp(mu) if mu is not None else None, int(max_evals), ctypes.byref(best),
                                         ctypes.byref(lml)), "mdgp_gp_optimize")
    return dict(sf2=best.sf2, l2=best.l2, sn2=best.sn2, lml=lml.value)
