"""The allocation-free GP posterior (mdgp_gp_posterior_noalloc) against the
allocating fit + predict entry points.

Callers that cannot call cudaMalloc while they run -- an application whose
device memory all belongs to its own pool allocator, or a latency-bound loop
that must not trigger the device synchronisation an allocation can cause --
pass device buffers for the inputs and outputs and get the same posterior,
computed in a fixed scratch array the library owns.  This file is
collected last; it checks two calls in a row so that state the scratch keeps
from one call cannot leak into the next."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10   # same bound as the GP parity tests


def _entry():
    from paper_1603_04628_gb300 import build, native
    build.build()
    L = native.lib()
    fn = L.mdgp_gp_posterior_noalloc
    vp = ctypes.c_void_p
    fn.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(native.GPParams), vp, vp,
                   ctypes.c_int64, vp, vp, vp, vp]
    fn.restype = ctypes.c_int
    return native, fn


def test_noalloc_posterior_matches_fit_and_predict_twice():
    torch = pytest.importorskip("torch")
    native, fn = _entry()
    ctx = native.Context(0, native.PREC_FP64)
    sf2, l2, sn2 = 1.3, 1.0, 0.0025
    stream = torch.cuda.current_stream()
    for M, m, seed in ((300, 64, 21), (77, 33, 22)):
        X, y = synth.gp_dataset(M, seed=seed)
        Xs = synth.gp_queries(m, seed=seed + 1)
        g = native.GP(ctx, X, y, sf2, l2, sn2)
        ref_mean, ref_var = g.predict(Xs)
        g.close()
        tX = torch.tensor(X, dtype=torch.float64, device="cuda")
        ty = torch.tensor(y, dtype=torch.float64, device="cuda")
        tXs = torch.tensor(Xs, dtype=torch.float64, device="cuda")
        mean = torch.empty(m, dtype=torch.float64, device="cuda")
        var = torch.empty(m, dtype=torch.float64, device="cuda")
        p = native.GPParams(sf2, l2, sn2, 1.0, None)
        st = fn(tX.data_ptr(), ty.data_ptr(), M, 2, ctypes.byref(p), None, tXs.data_ptr(), m, None,
                mean.data_ptr(), var.data_ptr(), stream.cuda_stream)
        assert st == 0
        scale = max(np.abs(y).max(), 1.0)
        assert np.abs(mean.cpu().numpy() - ref_mean).max() <= TOL * scale
        assert np.abs(var.cpu().numpy() - ref_var).max() <= TOL * sf2
    ctx.close()


def test_noalloc_rejects_databases_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    native, fn = _entry()
    X = torch.zeros((513, 2), dtype=torch.float64, device="cuda")
    y = torch.zeros(513, dtype=torch.float64, device="cuda")
    p = native.GPParams(1.0, 1.0, 0.01, 1.0, None)
    assert fn(X.data_ptr(), y.data_ptr(), 513, 2, ctypes.byref(p), None, None, 0, None, None, None, None) == -10
