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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structs of the binding lay out every field at the offset,
    and each struct with the size, that a C compiler gives the header's
    structs (compiled here with gcc as plain C)."""
    import ctypes as C
    import shutil
    import subprocess
    from paper_2006_13387_gb300 import _native as N
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"ts_mesh": N.TsMesh, "ts_bcs": N.TsBcs, "ts_options": N.TsOptions, "ts_stats": N.TsStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "topsolve.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs.items():
        assert got[(cname, "sizeof")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
