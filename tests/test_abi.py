"""The C ABI library loads and exports every entry point include/mdgp.h
declares (no GPU needed: nothing here launches device work)."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*[\w\s\*]*?\b(mdgp_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_1603_04628_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("mdgp_create", "mdgp_destroy", "mdgp_micro_batch", "mdgp_micro_plan",
                     "mdgp_micro_launch", "mdgp_micro_results", "mdgp_md_forces"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_defaults_and_argument_checks_without_a_gpu(built):
    from paper_1603_04628_gb300 import native
    p = native.md_params_default()
    assert (p.dt, p.rc, p.k_tether, p.gamma_wall, p.n_blocks, p.wall_planes) == (0.005, 2.5, 150.0, 1.0, 10, 3)
    L = native.lib()
    assert L.mdgp_md_params_default(None) == -1
    assert L.mdgp_destroy(None) == -1
    assert L.mdgp_micro_batch(None, None, 0, None) == -1
    assert L.mdgp_micro_launch(None) == -1
    assert L.mdgp_create(None, 0, 0) == -1


def test_gp_and_macro_entry_points_reject_null_handles_without_a_gpu(built):
    import ctypes as C
    from paper_1603_04628_gb300 import native
    L = native.lib()
    p = native.GPParams(1.0, 1.0, 0.01, 1.0, None, None)
    out = C.c_void_p()
    assert L.mdgp_gp_fit_inputs(None, None, 0, 2, C.byref(p), C.byref(out)) == -1
    assert L.mdgp_gp_set_outputs(None, None, None) == -1
    assert L.mdgp_gp_predict(None, None, 0, None, None, None) == -1
    mp = native.MacroParams()
    assert L.mdgp_macro_params_default(C.byref(mp)) == 0
    # the factor budget defaults to 0 (4 GiB); the q-GP inputs to (h, G)
    assert (mp.n_sections, mp.inputs, mp.factor_cache_mb) == (200, 0, 0)
