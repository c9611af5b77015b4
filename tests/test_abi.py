"""The C-ABI library builds, loads and exports every symbol include/*.h declares, and
its argument checks reject bad descriptors before touching a GPU (no compute here)."""
import ctypes
import glob
import os
import re

import pytest

import paper_1810_04033_gb300 as st

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(stencil_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = st.lib()
    names = declared_symbols()
    assert "stencil_apply" in names and "stencil_residual" in names
    for name in names:
        assert hasattr(L, name), name


def test_version_and_error_string():
    assert st.stencil_version() >= 10000
    assert isinstance(st.lib().stencil_last_error(), bytes)


def _grid(**kw):
    g = st.Grid()
    g.dim = kw.get("dim", 3)
    g.dtype = kw.get("dtype", st.F64)
    n = kw.get("n", (4, 4, 4))
    g.n[0], g.n[1], g.n[2] = n
    g.pitch = kw.get("pitch", 0)
    g.h = kw.get("h", 0.25)
    return g


@pytest.mark.parametrize("kw,msg", [
    (dict(dim=4), "dim"),
    (dict(dtype=7), "dtype"),
    (dict(n=(0, 4, 4)), "cells"),
    (dict(pitch=3), "pitch"),
    (dict(h=0.0), "h must"),
    (dict(h=float("nan")), "h must"),
])
def test_bad_descriptors_are_rejected_without_gpu(kw, msg):
    L = st.lib()
    g = _grid(**kw)
    fake = ctypes.c_void_p(4096)  # never dereferenced: checks fail first
    rc = L.stencil_apply(ctypes.byref(g), fake, ctypes.c_void_p(8192), 1, None)
    assert rc == -1
    assert msg in L.stencil_last_error().decode()


def test_null_and_misaligned_pointers_rejected():
    L = st.lib()
    g = _grid()
    assert L.stencil_apply(ctypes.byref(g), None, ctypes.c_void_p(8192), 1, None) == -1
    assert L.stencil_apply(ctypes.byref(g), ctypes.c_void_p(4100), ctypes.c_void_p(8192), 1, None) == -1
    assert "aligned" in L.stencil_last_error().decode()
    assert L.stencil_apply(None, ctypes.c_void_p(4096), ctypes.c_void_p(8192), 1, None) == -1
    assert L.stencil_apply(ctypes.byref(g), ctypes.c_void_p(4096), ctypes.c_void_p(8192), 9, None) == -1
    # overlapping input/output
    assert L.stencil_apply(ctypes.byref(g), ctypes.c_void_p(4096), ctypes.c_void_p(4096 + 64), 1, None) == -1
    assert "overlap" in L.stencil_last_error().decode()
    assert L.stencil_smooth_coloured(ctypes.byref(g), ctypes.c_void_p(4096), ctypes.c_void_p(1 << 20), -1, None) == -1
