"""The C-ABI library builds, loads and exports every symbol that
include/topsolve.h declares (no compute calls: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "topsolve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ts_[A-Za-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_2006_13387_gb300 import _native as N
    assert set(_declared()) == set(N.SIGNATURES)


def test_library_exports_every_symbol():
    from paper_2006_13387_gb300 import _native as N
    if not os.path.exists(N.LIB_PATH):
        from paper_2006_13387_gb300 import build
        build.build()
    L = N.lib()
    for name in _declared():
        assert hasattr(L, name), name


def test_options_default_runs_without_gpu():
    import ctypes as C
    from paper_2006_13387_gb300 import _native as N
    o = N.TsOptions()
    N.lib().ts_options_default(C.byref(o))
    assert o.max_modes == 16 and o.rotations == 1 and o.tau_scale == 2.0 and o.energy_tol < 0
