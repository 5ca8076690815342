"""The C-ABI library builds, loads and exports every function include/wcsim.h declares
(CPU only: no compute calls without a GPU)."""
import ast
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2104_08265_gb300 import _build
    return _build.build()


def test_library_exports_every_header_function(libpath):
    from paper_2104_08265_gb300 import wcsim
    declared = wcsim.header_functions()
    assert "wcsim_run" in declared and "wcsim_plane_create" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    L = wcsim.lib()
    for f in declared:
        assert hasattr(L, f)
    assert L.wcsim_version().startswith(b"wcsim")


def test_argument_checks_need_no_gpu(libpath):
    """Host-side validation answers before any CUDA call is made."""
    import ctypes
    from paper_2104_08265_gb300 import synth, wcsim
    L = wcsim.lib()
    g = synth.Geometry(n_wires=8, n_imp=10, n_ticks=64, pitch_mm=3.0)
    p = synth.DriftParams()
    h = ctypes.c_void_p(1)
    bad = wcsim.c_geometry(g); bad.n_wires = 0
    assert L.wcsim_plane_create(ctypes.byref(bad), ctypes.c_void_p(16), 0, 0,
                                ctypes.byref(wcsim.c_params(p)), None, ctypes.byref(h)) == wcsim.ESHAPE
    assert h.value is None
    assert b"n_wires" in L.wcsim_last_error()
    assert L.wcsim_plane_create(ctypes.byref(wcsim.c_geometry(g)), None, 0, 0,
                                ctypes.byref(wcsim.c_params(p)), None, ctypes.byref(h)) == wcsim.EINVAL
    bp = wcsim.c_params(p); bp.lifetime_us = -1.0
    assert L.wcsim_plane_create(ctypes.byref(wcsim.c_geometry(g)), ctypes.c_void_p(16), 0, 0,
                                ctypes.byref(bp), None, ctypes.byref(h)) == wcsim.EINVAL
    # 1021 is prime: no supported factorisation
    assert L.wcsim_plane_create(ctypes.byref(wcsim.c_geometry(g)), ctypes.c_void_p(16), 0, 1021,
                                ctypes.byref(wcsim.c_params(p)), None, ctypes.byref(h)) == wcsim.ESHAPE
    assert L.wcsim_plane_create(ctypes.byref(wcsim.c_geometry(g)), ctypes.c_void_p(16), 4, 0,
                                ctypes.byref(wcsim.c_params(p)), None, ctypes.byref(h)) == wcsim.ESHAPE
    for field, val in (("renormalize", 2), ("reserved", 1), ("fluctuate", 3), ("fluctuate", -1)):
        bp = wcsim.c_params(p); setattr(bp, field, val)
        assert L.wcsim_plane_create(ctypes.byref(wcsim.c_geometry(g)), ctypes.c_void_p(16), 0, 0,
                                    ctypes.byref(bp), None, ctypes.byref(h)) == wcsim.EINVAL
        assert field.encode() in L.wcsim_last_error()
    assert L.wcsim_plane_set_reuse_forward(None, 1) == wcsim.EINVAL
    assert L.wcsim_run(None, None, None, None) == wcsim.EINVAL
    assert L.wcsim_plane_destroy(None) == wcsim.OK


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (a C program
    compiled against include/wcsim.h prints them)."""
    import ctypes
    from paper_2104_08265_gb300 import wcsim
    mirrors = {"wcsim_geometry": wcsim.CGeometry, "wcsim_drift_params": wcsim.CParams,
               "wcsim_depos": wcsim.CDepos, "wcsim_depo_grads": wcsim.CDepoGrads,
               "wcsim_tune_report": wcsim.CTuneReport}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "wcsim.h"', 'int main(void) {']
    for name, cls in mirrors.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for name, cls in mirrors.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_product_path_never_touches_the_oracle():
    """Nothing in the package imports, loads or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_2104_08265_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", path
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                assert "liboracle" not in open(path).read(), path
