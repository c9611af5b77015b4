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
    assert L.stencil_smooth_coloured(ctypes.byref(g), ctypes.c_void_p(4096), ctypes.c_void_p(1 << 20), -1,
                                     None, 0, None) == -1


def _ws_size(g, call, sweeps):
    n = ctypes.c_size_t(0)
    rc = st.lib().stencil_workspace_size(ctypes.byref(g), call, sweeps, ctypes.byref(n))
    return rc, n.value


def test_workspace_size_without_gpu():
    """Sizes follow from the descriptor: F64 GS needs three int64 copies of the grid
    plus the per-sweep bounds, multi-sweep Jacobi two copies, FD red-black none."""
    g = _grid(n=(7, 5, 3), pitch=10)
    span = 10 * 6 * 4
    rc, gs = _ws_size(g, st.CALL_SMOOTH_COLOURED, 4)
    assert rc == 0 and 3 * span * 8 < gs <= 3 * span * 8 + 256 + 1024
    assert gs > 3 * span * 8 + 255 - (3 * span * 8) % 256  # bounds part starts on 256 bytes
    rc, jac = _ws_size(g, st.CALL_SMOOTH_JACOBI, 4)
    assert rc == 0 and 2 * span * 8 < jac <= 2 * span * 8 + 256 + 1024
    assert _ws_size(g, st.CALL_SMOOTH_JACOBI, 1) == (0, 0)
    assert _ws_size(g, st.CALL_SMOOTH_COLOURED, 0) == (0, 0)
    rc, red = _ws_size(g, st.CALL_RESIDUAL, 0)
    assert rc == 0 and red >= 16 + 16
    g32 = _grid(n=(7, 5, 3), pitch=12, dtype=st.F32)
    assert _ws_size(g32, st.CALL_SMOOTH_COLOURED, 3) == (0, 12 * 6 * 4 * 4)
    gfd = _grid(op=st.OP_FD)
    assert _ws_size(gfd, st.CALL_SMOOTH_COLOURED, 3) == (0, 0)
    assert _ws_size(g, 99, 1)[0] == -1
    assert "unknown call" in st.lib().stencil_last_error().decode()
    assert _ws_size(g, st.CALL_SMOOTH_COLOURED, -1)[0] == -1
    assert _ws_size(_grid(dim=5), st.CALL_RESIDUAL, 0)[0] == -1


def test_short_or_misaligned_workspace_rejected_without_gpu():
    """A caller workspace smaller than stencil_workspace_size, or not 256-byte aligned,
    or overlapping an argument, is refused before any device work."""
    L = st.lib()
    g = _grid(n=(7, 5, 3))
    u, f, w = ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20)
    _, need = _ws_size(g, st.CALL_SMOOTH_COLOURED, 4)
    ws = ctypes.c_void_p(8 << 20)
    assert L.stencil_smooth_coloured(ctypes.byref(g), u, f, 4, ws, need - 1, None) == -1
    assert "too small" in L.stencil_last_error().decode()
    assert L.stencil_smooth_coloured(ctypes.byref(g), u, f, 4, ctypes.c_void_p((8 << 20) + 128), need,
                                     None) == -1
    assert "256-byte" in L.stencil_last_error().decode()
    assert L.stencil_smooth_coloured(ctypes.byref(g), u, f, 4, ctypes.c_void_p(1 << 20), need, None) == -1
    assert "overlaps" in L.stencil_last_error().decode()
    _, jneed = _ws_size(g, st.CALL_SMOOTH_JACOBI, 4)
    assert L.stencil_smooth_jacobi(ctypes.byref(g), u, f, w, 4, 0.5, ws, jneed - 8, None) == -1
    assert "too small" in L.stencil_last_error().decode()
    _, rneed = _ws_size(g, st.CALL_RESIDUAL, 0)
    assert L.stencil_residual(ctypes.byref(g), u, f, None, ctypes.c_void_p(4 << 20), ws, rneed - 1,
                              None) == -1
    assert "too small" in L.stencil_last_error().decode()


def test_tuning_table_save_load_roundtrip_without_gpu(tmp_path):
    """The launch-shape table: set, get, save as JSON, clear, load back; malformed
    files and out-of-range shapes are refused (host-only calls)."""
    import json
    import torch
    u3 = torch.zeros(9, 7, 12, dtype=torch.float64)[..., :10]  # n = (9, 6, 8), pitch 12
    u2 = torch.zeros(33, 40, dtype=torch.float64)
    st.stencil_tuning_clear()
    assert st.stencil_tuning_get(u3, 0.1, st.CALL_SMOOTH_COLOURED) is None
    st.stencil_tuning_set(u3, 0.1, st.CALL_SMOOTH_COLOURED, chunk=4)
    st.stencil_tuning_set(u2, 0.1, st.CALL_SMOOTH_JACOBI, chunk=128, depth=1, ms=1.5)
    st.stencil_tuning_set(u2, 0.1, st.CALL_APPLY_ELEMENTWISE, chunk=32)
    assert st.stencil_tuning_get(u3, 0.1, st.CALL_SMOOTH_COLOURED) == (4, 0, 0.0)
    path = str(tmp_path / "tuning.json")
    st.stencil_tuning_save(path)
    doc = json.load(open(path))
    assert doc["format"] == "stencil_gb300_tuning" and len(doc["entries"]) == 3
    e = [x for x in doc["entries"] if x["call"] == st.CALL_SMOOTH_JACOBI][0]
    assert e["dim"] == 2 and e["n"] == [39, 32, 0] and e["pitch"] == 40 and e["depth"] == 1 and e["ms"] == 1.5
    st.stencil_tuning_clear()
    assert st.stencil_tuning_get(u2, 0.1, st.CALL_SMOOTH_JACOBI) is None
    st.stencil_tuning_load(path)
    assert st.stencil_tuning_get(u2, 0.1, st.CALL_SMOOTH_JACOBI) == (128, 1, 1.5)
    assert st.stencil_tuning_get(u2, 0.1, st.CALL_APPLY_ELEMENTWISE) == (32, 0, 0.0)
    st.stencil_tuning_set(u2, 0.1, st.CALL_APPLY_ELEMENTWISE, chunk=None)  # remove
    assert st.stencil_tuning_get(u2, 0.1, st.CALL_APPLY_ELEMENTWISE) is None
    bad = tmp_path / "bad.json"
    bad.write_text('{"format": "stencil_gb300_tuning", "entries": [{"call": 9}]}')
    with pytest.raises(st.StencilError):
        st.stencil_tuning_load(str(bad))
    bad.write_text('{"format": "something else", "entries": []}')
    with pytest.raises(st.StencilError):
        st.stencil_tuning_load(str(bad))
    bad.write_text('{"format": "stencil_gb300_tuning", "entries": [')
    with pytest.raises(st.StencilError):
        st.stencil_tuning_load(str(bad))
    with pytest.raises(st.StencilError):
        st.stencil_tuning_set(u2, 0.1, st.CALL_SMOOTH_JACOBI, chunk=64, depth=3)
    with pytest.raises(st.StencilError):
        st.stencil_tuning_set(u2, 0.1, st.CALL_RESIDUAL, chunk=64)
    st.stencil_tuning_clear()
