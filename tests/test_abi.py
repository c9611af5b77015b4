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
    g.op = kw.get("op", st.OP_Q1)
    return g


@pytest.mark.parametrize("kw,msg", [
    (dict(dim=4), "dim"),
    (dict(dtype=7), "dtype"),
    (dict(n=(0, 4, 4)), "cells"),
    (dict(pitch=3), "pitch"),
    (dict(h=0.0), "h must"),
    (dict(h=float("nan")), "h must"),
    (dict(op=7), "operator"),
    (dict(op=st.OP_FD, dtype=st.F32), "F64 only"),
])
def test_bad_descriptors_are_rejected_without_gpu(kw, msg):
    L = st.lib()
    g = _grid(**kw)
    fake = ctypes.c_void_p(4096)  # never dereferenced: checks fail first
    rc = L.stencil_apply(ctypes.byref(g), fake, ctypes.c_void_p(8192), 1, None)
    assert rc == -1
    assert msg in L.stencil_last_error().decode()


def test_fd_operator_rejected_where_unsupported_without_gpu():
    """Entry points that implement the Q1 operator only refuse op = FD before any
    device work; the FD apply has no element-wise form."""
    L = st.lib()
    g = _grid(op=st.OP_FD)
    fake, fake2 = ctypes.c_void_p(4096), ctypes.c_void_p(1 << 20)
    assert L.stencil_apply(ctypes.byref(g), fake, fake2, st.FORM_ELEMENTWISE, None) == -1
    assert "stencil form" in L.stencil_last_error().decode()
    opts = st.SolveOpts(1e-8, 10, 8, st.F32)
    assert L.stencil_solve(ctypes.byref(g), fake, fake2, ctypes.byref(opts), None, None) == -1
    assert "Q1" in L.stencil_last_error().decode()
    mo = st.MgOpts(1e-8, 10, 2, 2, 20, 0, 0)
    assert L.stencil_mg_solve(ctypes.byref(g), fake, fake2, ctypes.byref(mo), None, None) == -1
    assert "Q1" in L.stencil_last_error().decode()
    assert L.stencil_residual_noalloc(ctypes.byref(g), fake, fake2, None, ctypes.c_void_p(1 << 21), None) == -1
    assert "Q1" in L.stencil_last_error().decode()


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
