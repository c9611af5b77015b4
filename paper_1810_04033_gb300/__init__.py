"""Python binding of libstencil_gb300 (the C ABI in include/stencil.h).

Argument marshalling only: every step runs in the library's CUDA kernels.  Functions
carry the C names and take torch CUDA tensors laid out x fastest, shape
(nz+1, ny+1, nx+1) in 3D or (ny+1, nx+1) in 2D, unit stride in x and a row stride
(pitch) >= nx+1; the z stride must equal pitch * (ny+1).  Work is queued on the current
torch stream unless `stream` is given.  There is no CPU fallback: if the library
cannot be built or loaded, every call raises.
"""
import ctypes
import os

import torch

from . import build as _build

F64, F32, BF16 = 0, 1, 2
FORM_ELEMENTWISE, FORM_STENCIL = 0, 1
OP_Q1, OP_FD = 0, 1

STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "EADMIT", -4: "ETIMEDOUT", -5: "ECUDA",
          -6: "ENOTCONV", -7: "ENOTFOUND", -8: "EBUSY"}

_DTYPES = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}


SOLVER_REFINE, SOLVER_MG = 0, 1
OK, EINVAL, ENOMEM, EADMIT, ETIMEDOUT, ECUDA, ENOTCONV, ENOTFOUND, EBUSY = 0, -1, -2, -3, -4, -5, -6, -7, -8


class StencilError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3), ("pitch", ctypes.c_int64), ("h", ctypes.c_double),
                ("op", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class PatchDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("reserved", ctypes.c_int32), ("offset", ctypes.c_int64),
                ("h", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("inner_sweeps", ctypes.c_int32), ("inner_dtype", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("solver", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rel_tol", ctypes.c_double),
                ("f", ctypes.POINTER(ctypes.c_double)), ("f_seed", ctypes.c_uint64),
                ("u0", ctypes.POINTER(ctypes.c_double))]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("relres", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("inflight", ctypes.c_int64), ("hbm_used", ctypes.c_uint64), ("hbm_budget", ctypes.c_uint64)]


REQ_SMOOTH, REQ_SOLVE = 0, 1


class SolveOpts(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("inner_sweeps", ctypes.c_int), ("inner_dtype", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("relres", ctypes.c_double), ("relres_history", ctypes.POINTER(ctypes.c_double))]


class DependOpts(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("test_stall", ctypes.c_int32), ("max_wait_ns", ctypes.c_int64), ("stalled_at", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class MgOpts(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("max_cycles", ctypes.c_int32), ("pre", ctypes.c_int32),
                ("post", ctypes.c_int32), ("coarse_sweeps", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class MgInfo(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int32), ("converged", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("relres", ctypes.c_double),
                ("relres_history", ctypes.POINTER(ctypes.c_double))]


class Tuning(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("depth", ctypes.c_int32), ("ms", ctypes.c_double)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Loads (building first if needed) the shared library; raises if impossible."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        gp = ctypes.POINTER(Grid)
        sigs = {
            "stencil_version": (ci, []),
            "stencil_last_error": (ctypes.c_char_p, []),
            "stencil_release_workspace": (ci, []),
            "stencil_apply": (ci, [gp, vp, vp, ci, vp]),
            "stencil_workspace_size": (ci, [gp, ci, ci, ctypes.POINTER(ctypes.c_size_t)]),
            "stencil_device_status": (ci, [ctypes.POINTER(ctypes.c_uint32), ci]),
            "stencil_autotune": (ci, [gp, ci, ci, ctypes.POINTER(Tuning), vp]),
            "stencil_tuning_set": (ci, [gp, ci, ctypes.POINTER(Tuning)]),
            "stencil_tuning_get": (ci, [gp, ci, ctypes.POINTER(Tuning)]),
            "stencil_tuning_clear": (ci, []),
            "stencil_tuning_save": (ci, [ctypes.c_char_p]),
            "stencil_tuning_load": (ci, [ctypes.c_char_p]),
            "stencil_smooth_coloured": (ci, [gp, vp, vp, ci, vp, ctypes.c_size_t, vp]),
            "stencil_smooth_jacobi": (ci, [gp, vp, vp, vp, ci, cd, vp, ctypes.c_size_t, vp]),
            "stencil_residual": (ci, [gp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]),
            "stencil_jacobi_step": (ci, [gp, vp, vp, vp, cd, vp]),
            "stencil_residual_noalloc": (ci, [gp, vp, vp, vp, vp, vp]),
            "stencil_solve": (ci, [gp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]),
            "stencil_smooth_depend": (ci, [gp, vp, vp, ci, ctypes.POINTER(DependOpts), vp]),
            "stencil_smooth_expensive": (ci, [gp, vp, vp, ci, ci, ci, ctypes.POINTER(DependOpts), vp]),
            "stencil_mg_solve": (ci, [gp, vp, vp, ctypes.POINTER(MgOpts), ctypes.POINTER(MgInfo), vp]),
            "stencil_mg_vcycle": (ci, [gp, vp, vp, ctypes.POINTER(MgOpts), vp]),
            "stencil_mg_restrict": (ci, [gp, vp, gp, vp, vp]),
            "stencil_mg_prolong_add": (ci, [gp, vp, gp, vp, vp]),
            "stencil_patch_batch_create": (ci, [ctypes.POINTER(PatchDesc), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(vp)]),
            "stencil_patch_batch_smooth": (ci, [vp, vp, vp, ci, vp]),
            "stencil_patch_batch_autotune": (ci, [vp, vp, vp, vp]),
            "stencil_patch_batch_config": (ci, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
            "stencil_patch_batch_destroy": (ci, [vp]),
            "stencil_server_create": (ci, [ctypes.c_size_t, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]),
            "stencil_server_submit": (ci, [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
            "stencil_server_poll": (ci, [vp, ctypes.c_uint64, ctypes.POINTER(Result)]),
            "stencil_server_wait": (ci, [vp, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(Result)]),
            "stencil_server_fetch": (ci, [vp, ctypes.c_uint64, vp]),
            "stencil_server_release": (ci, [vp, ctypes.c_uint64]),
            "stencil_server_stats": (ci, [vp, ctypes.POINTER(ServerStats)]),
            "stencil_server_destroy": (ci, [vp]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise StencilError(rc, lib().stencil_last_error().decode())


def grid_for(t: torch.Tensor, h: float, op: int = 0) -> Grid:
    """Grid descriptor for a vertex tensor (validates layout, not device residency)."""
    if t.dim() not in (2, 3):
        raise ValueError("expected a 2D or 3D vertex tensor")
    if t.dtype not in _DTYPES:
        raise ValueError("unsupported dtype %s" % t.dtype)
    if t.stride(-1) != 1:
        raise ValueError("x must have unit stride")
    g = Grid()
    g.dim = t.dim()
    g.dtype = _DTYPES[t.dtype]
    if t.dim() == 3:
        nz, ny, nx = (s - 1 for s in t.shape)
        pitch = t.stride(1)
        if t.shape[0] > 1 and t.stride(0) != pitch * t.shape[1]:
            raise ValueError("z stride must be pitch * (ny+1)")
        g.n[0], g.n[1], g.n[2] = nx, ny, nz
    else:
        ny, nx = (s - 1 for s in t.shape)
        pitch = t.stride(0)
        g.n[0], g.n[1], g.n[2] = nx, ny, 0
    g.pitch = pitch
    g.h = float(h)
    g.op = int(op)
    return g


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _same_layout(a, b):
    if a.shape != b.shape or a.stride() != b.stride() or a.dtype != b.dtype:
        raise ValueError("arrays must share shape, strides and dtype")
    if a.device != b.device or a.device.type != "cuda":
        raise ValueError("arrays must be CUDA tensors on the same device")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _device_buffer(t, what, device, min_numel=0, contiguous=True):
    """Checks a float64 buffer the library reads or writes by raw pointer: a CUDA tensor
    (on `device` unless None), contiguous when the library takes it as a flat array, and
    at least `min_numel` elements long, so that a wrong argument raises here instead of
    letting a kernel touch memory outside it."""
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise ValueError("%s must be a CUDA tensor" % what)
    if device is not None and t.device != device:
        raise ValueError("%s must be on %s" % (what, device))
    if t.dtype != torch.float64:
        raise ValueError("%s must be float64" % what)
    if contiguous and not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if t.numel() < min_numel:
        raise ValueError("%s needs at least %d elements" % (what, min_numel))


def stencil_version() -> int:
    return lib().stencil_version()


def stencil_apply(u, y, h, form=FORM_STENCIL, stream=None, op=OP_Q1):
    """y = A u (boundary rows of y set to 0); op OP_Q1 or OP_FD (stencil form only)."""
    _same_layout(u, y)
    g = grid_for(u, h, op)
    _check(lib().stencil_apply(ctypes.byref(g), _ptr(u), _ptr(y), int(form), _stream(stream)))
    return y


CALL_SMOOTH_COLOURED, CALL_SMOOTH_JACOBI, CALL_RESIDUAL = 1, 2, 3
CALL_APPLY_ELEMENTWISE, CALL_APPLY_STENCIL = 4, 5


def stencil_workspace_size(u, h, call, sweeps=0, op=OP_Q1):
    """Bytes of device workspace (`ws`) that `call` needs on u's grid for `sweeps` sweeps."""
    g = grid_for(u, h, op)
    n = ctypes.c_size_t(0)
    _check(lib().stencil_workspace_size(ctypes.byref(g), int(call), int(sweeps), ctypes.byref(n)))
    return int(n.value)


def _ws(ws, device):
    """(pointer, bytes) of a caller workspace tensor, or (NULL, 0) for the library's own."""
    if ws is None:
        return ctypes.c_void_p(0), 0
    if not isinstance(ws, torch.Tensor) or ws.device != device or not ws.is_contiguous():
        raise ValueError("ws must be a contiguous tensor on the grid's device")
    return ctypes.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size()


def stencil_smooth_coloured(u, f, h, sweeps, stream=None, op=OP_Q1, ws=None):
    """`sweeps` coloured Gauss-Seidel sweeps on A u = f, in place on u (OP_FD: red-black).
    ws: optional caller workspace (stencil_workspace_size bytes, e.g. a uint8 tensor)."""
    _same_layout(u, f)
    g = grid_for(u, h, op)
    wp, wb = _ws(ws, u.device)
    _check(lib().stencil_smooth_coloured(ctypes.byref(g), _ptr(u), _ptr(f), int(sweeps), wp, wb,
                                         _stream(stream)))
    return u


def stencil_smooth_jacobi(u, f, work, h, sweeps, omega=2.0 / 3.0, stream=None, op=OP_Q1, ws=None):
    """`sweeps` damped Jacobi sweeps; result in u, work is scratch of u's layout;
    ws: optional caller workspace as for stencil_smooth_coloured."""
    _same_layout(u, f)
    _same_layout(u, work)
    g = grid_for(u, h, op)
    wp, wb = _ws(ws, u.device)
    _check(lib().stencil_smooth_jacobi(ctypes.byref(g), _ptr(u), _ptr(f), _ptr(work),
                                       int(sweeps), float(omega), wp, wb, _stream(stream)))
    return u


def stencil_jacobi_step(u_in, f, u_out, h, omega=2.0 / 3.0, stream=None, op=OP_Q1):
    """One damped Jacobi sweep from u_in into u_out (boundary copied)."""
    _same_layout(u_in, f)
    _same_layout(u_in, u_out)
    g = grid_for(u_in, h, op)
    _check(lib().stencil_jacobi_step(ctypes.byref(g), _ptr(u_in), _ptr(f), _ptr(u_out),
                                     float(omega), _stream(stream)))
    return u_out


def stencil_residual(u, f, h, r=None, norms2=None, stream=None, op=OP_Q1, ws=None):
    """r = f - A u (if r given) and norms2 = [sum r^2, sum f^2] (device float64[2]);
    ws: optional caller workspace as for stencil_smooth_coloured."""
    _same_layout(u, f)
    if r is not None:
        _same_layout(u, r)
    if norms2 is None:
        norms2 = torch.empty(2, dtype=torch.float64, device=u.device)
    _device_buffer(norms2, "norms2", u.device, 2)
    g = grid_for(u, h, op)
    wp, wb = _ws(ws, u.device)
    _check(lib().stencil_residual(ctypes.byref(g), _ptr(u), _ptr(f),
                                  _ptr(r) if r is not None else ctypes.c_void_p(0),
                                  _ptr(norms2), wp, wb, _stream(stream)))
    return norms2


def stencil_residual_noalloc(u, f, h, norms2, r=None, stream=None):
    """stencil_residual without any device allocation: the caller supplies norms2
    (device float64[2]) and optionally r; the library's fixed scratch array is used."""
    _same_layout(u, f)
    if r is not None:
        _same_layout(u, r)
    _device_buffer(norms2, "norms2", u.device, 2)
    g = grid_for(u, h)
    _check(lib().stencil_residual_noalloc(ctypes.byref(g), _ptr(u), _ptr(f),
                                          _ptr(r) if r is not None else ctypes.c_void_p(0),
                                          _ptr(norms2), _stream(stream)))
    return norms2


def stencil_solve(u, f, h, rel_tol=1e-10, max_outer=100000, inner_sweeps=8, inner_dtype=F32,
                  stream=None, history=True):
    """Iterative refinement on A u = f (u, f float64; u updated in place).  Returns a
    dict with iterations, converged, relres and (optionally) the relative-residual
    history.  Raises StencilError except for the not-converged status (-6)."""
    _same_layout(u, f)
    if u.dtype != torch.float64:
        raise ValueError("solve needs float64 u and f")
    g = grid_for(u, h)
    opts = SolveOpts(float(rel_tol), int(max_outer), int(inner_sweeps), int(inner_dtype))
    info = SolveInfo()
    hist = None
    if history:
        hist = (ctypes.c_double * (int(max_outer) + 1))()
        info.relres_history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    rc = lib().stencil_solve(ctypes.byref(g), _ptr(u), _ptr(f), ctypes.byref(opts), ctypes.byref(info),
                             _stream(stream))
    if rc not in (0, -6):
        _check(rc)
    out = {"iterations": info.iterations, "converged": bool(info.converged), "relres": info.relres}
    if history:
        out["history"] = list(hist[:info.iterations + 1])
    return out


def stencil_smooth_depend(u, f, h, sweeps, rows=0, ctas=0, max_wait_ns=0, test_stall=0, stream=None, cols=0):
    """Dependency-driven red-black sweeps (op FD) in place on u.  Returns
    {"status": 0 or the timeout code, "stalled_at": block}; raises on other errors."""
    _same_layout(u, f)
    g = grid_for(u, h, OP_FD)
    o = DependOpts(int(rows), int(cols), int(ctas), int(test_stall), int(max_wait_ns), -1, 0)
    rc = lib().stencil_smooth_depend(ctypes.byref(g), _ptr(u), _ptr(f), int(sweeps), ctypes.byref(o),
                                     _stream(stream))
    if rc not in (0, ETIMEDOUT):
        _check(rc)
    return {"status": rc, "stalled_at": o.stalled_at}


COST_NONE, COST_UNIFORM, COST_LINEAR = 0, 1, 2


def stencil_smooth_expensive(u, f, h, sweeps, cost_mode, kmax, depend=None, stream=None):
    """Red-black sweeps of the expensive stencil S(k) (op FD) in place on u.  depend:
    None (colour passes with barriers) or a dict of stencil_smooth_depend options.
    Returns the status (0 or the timeout code)."""
    _same_layout(u, f)
    g = grid_for(u, h, OP_FD)
    o = None
    if depend is not None:
        o = DependOpts(int(depend.get("rows", 0)), int(depend.get("cols", 0)), int(depend.get("ctas", 0)),
                       int(depend.get("test_stall", 0)), int(depend.get("max_wait_ns", 0)), -1, 0)
    rc = lib().stencil_smooth_expensive(ctypes.byref(g), _ptr(u), _ptr(f), int(sweeps), int(cost_mode), int(kmax),
                                        ctypes.byref(o) if o is not None else None, _stream(stream))
    if rc not in (0, ETIMEDOUT):
        _check(rc)
    return rc


def _mg_opts(rel_tol, max_cycles, pre, post, coarse_sweeps, max_levels):
    return MgOpts(float(rel_tol), int(max_cycles), int(pre), int(post), int(coarse_sweeps), int(max_levels), 0)


def stencil_mg_solve(u, f, h, rel_tol=1e-10, max_cycles=100, pre=2, post=2, coarse_sweeps=20, max_levels=0,
                     stream=None, history=True):
    """Multigrid V-cycles on A u = f (u, f float64; u updated in place).  Returns a dict
    with cycles, converged, levels, relres and (optionally) the relative-residual
    history.  Raises StencilError except for the not-converged status (-6)."""
    _same_layout(u, f)
    if u.dtype != torch.float64:
        raise ValueError("multigrid needs float64 u and f")
    g = grid_for(u, h)
    opts = _mg_opts(rel_tol, max_cycles, pre, post, coarse_sweeps, max_levels)
    info = MgInfo()
    hist = None
    if history:
        hist = (ctypes.c_double * (int(max_cycles) + 1))()
        info.relres_history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    rc = lib().stencil_mg_solve(ctypes.byref(g), _ptr(u), _ptr(f), ctypes.byref(opts), ctypes.byref(info),
                                _stream(stream))
    if rc not in (0, -6):
        _check(rc)
    out = {"cycles": info.cycles, "converged": bool(info.converged), "levels": info.levels,
           "relres": info.relres}
    if history:
        out["history"] = list(hist[:info.cycles + 1])
    return out


def stencil_mg_vcycle(u, f, h, pre=2, post=2, coarse_sweeps=20, max_levels=0, stream=None):
    """One V-cycle on u (in place), stream-ordered."""
    _same_layout(u, f)
    g = grid_for(u, h)
    opts = _mg_opts(0.0, 0, pre, post, coarse_sweeps, max_levels)
    _check(lib().stencil_mg_vcycle(ctypes.byref(g), _ptr(u), _ptr(f), ctypes.byref(opts), _stream(stream)))
    return u


def stencil_mg_restrict(rf, rc, h, stream=None):
    """rc = R rf (full weighting); rc is a vertex array of the coarse grid."""
    _device_buffer(rf, "rf", None, contiguous=False)
    _device_buffer(rc, "rc", rf.device, contiguous=False)
    gf, gc = grid_for(rf, h), grid_for(rc, 2.0 * h)
    _check(lib().stencil_mg_restrict(ctypes.byref(gf), _ptr(rf), ctypes.byref(gc), _ptr(rc), _stream(stream)))
    return rc


def stencil_mg_prolong_add(ec, uf, h, stream=None):
    """uf += P ec on the fine interior; h is the fine mesh width."""
    _device_buffer(uf, "uf", None, contiguous=False)
    _device_buffer(ec, "ec", uf.device, contiguous=False)
    gf, gc = grid_for(uf, h), grid_for(ec, 2.0 * h)
    _check(lib().stencil_mg_prolong_add(ctypes.byref(gf), _ptr(uf), ctypes.byref(gc), _ptr(ec), _stream(stream)))
    return uf


def packed_numel(sizes, offsets) -> int:
    """Elements a packed patch array must hold: the end of the patch that ends last
    (patch p spans offsets[p] .. offsets[p] + (sizes[p]+1)^3)."""
    import numpy as np
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.asarray(offsets, dtype=np.int64)
    if sizes.size == 0:
        return 0
    return int((offsets + (sizes + 1) ** 3).max())


class PatchBatch:
    """Handle of a patch batch (stencil_patch_batch_*).  sizes: cells per edge per
    patch; offsets: element offsets in the packed arrays; neighbours: (npatch, 27) int32."""

    def __init__(self, sizes, offsets, neighbours):
        import numpy as np
        sizes = np.asarray(sizes, dtype=np.int32)
        offsets = np.asarray(offsets, dtype=np.int64)
        nb = np.ascontiguousarray(neighbours, dtype=np.int32)
        n = len(sizes)
        descs = (PatchDesc * n)()
        for i in range(n):
            descs[i].n = int(sizes[i])
            descs[i].reserved = 0
            descs[i].offset = int(offsets[i])
            descs[i].h = 0.0
        self._h = ctypes.c_void_p()
        _check(lib().stencil_patch_batch_create(descs, n, nb.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                ctypes.byref(self._h)))
        self.npatch = n
        self.numel = packed_numel(sizes, offsets)

    def _arrays(self, u_all, f_all):
        _device_buffer(u_all, "u_all", None, self.numel)
        _device_buffer(f_all, "f_all", u_all.device, self.numel)

    def smooth(self, u_all, f_all, sweeps, stream=None):
        self._arrays(u_all, f_all)
        _check(lib().stencil_patch_batch_smooth(self._h, _ptr(u_all), _ptr(f_all), int(sweeps), _stream(stream)))
        return u_all

    def autotune(self, u_all, f_all, stream=None):
        self._arrays(u_all, f_all)
        _check(lib().stencil_patch_batch_autotune(self._h, _ptr(u_all), _ptr(f_all), _stream(stream)))
        return self.config()

    def config(self):
        t, c = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().stencil_patch_batch_config(self._h, ctypes.byref(t), ctypes.byref(c)))
        return t.value, c.value

    def close(self):
        if self._h:
            lib().stencil_patch_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Handle of a request server (stencil_server_*), host-array interface."""

    def __init__(self, hbm_budget_bytes, streams=0, max_inflight=0, inner_sweeps=0, inner_dtype=F32,
                 max_outer=0, solver=0):
        """solver: SOLVER_REFINE (0) or SOLVER_MG (1) for SOLVE requests."""
        o = ServerOpts(int(streams), int(max_inflight), int(inner_sweeps), int(inner_dtype), int(max_outer),
                       int(solver))
        self._h = ctypes.c_void_p()
        _check(lib().stencil_server_create(int(hbm_budget_bytes), ctypes.byref(o), ctypes.byref(self._h)))
        self._n = {}  # ticket -> cells per edge, for the size of fetched results

    def submit(self, kind, n, sweeps=20, rel_tol=1e-8, f=None, f_seed=0, u0=None):
        """f / u0: host float64 arrays of (n+1)^3 or None (f: drawn from f_seed).  The
        library copies them during the call (it reads exactly (n+1)^3 values each)."""
        import numpy as np
        r = Request()
        r.kind, r.n, r.sweeps, r.reserved, r.rel_tol = int(kind), int(n), int(sweeps), 0, float(rel_tol)
        span = (int(n) + 1) ** 3 if int(n) > 0 else 0
        keep = []  # alive until the call returns
        if f is not None:
            fa = np.ascontiguousarray(f, dtype=np.float64)
            if fa.size != span:
                raise ValueError("f must hold (n+1)^3 = %d values, got %d" % (span, fa.size))
            keep.append(fa)
            r.f = fa.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.f_seed = int(f_seed) & 0xFFFFFFFFFFFFFFFF
        if u0 is not None:
            ua = np.ascontiguousarray(u0, dtype=np.float64)
            if ua.size != span:
                raise ValueError("u0 must hold (n+1)^3 = %d values, got %d" % (span, ua.size))
            keep.append(ua)
            r.u0 = ua.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        t = ctypes.c_uint64()
        _check(lib().stencil_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._n[t.value] = int(n)
        return t.value

    @staticmethod
    def _res(r):
        return {"status": r.status, "iterations": r.iterations, "relres": r.relres, "t_submit": r.t_submit,
                "t_admit": r.t_admit, "t_done": r.t_done}

    def poll(self, ticket):
        r = Result()
        rc = lib().stencil_server_poll(self._h, ticket, ctypes.byref(r))
        if rc == -8:
            return None
        _check(rc)
        return self._res(r)

    def wait(self, ticket, timeout_us=-1):
        r = Result()
        _check(lib().stencil_server_wait(self._h, ticket, int(timeout_us), ctypes.byref(r)))
        return self._res(r)

    def fetch(self, ticket, n=None):
        """The request's solution as a host array of (n+1)^3 values; n is the request's
        own edge (an `n` given here must match it)."""
        import numpy as np
        if ticket not in self._n:
            raise StencilError(ENOTFOUND, "server_fetch: unknown ticket")
        m = self._n[ticket]
        if n is not None and int(n) != m:
            raise ValueError("ticket %d has n = %d, not %d" % (ticket, m, int(n)))
        out = np.empty((m + 1,) * 3, dtype=np.float64)
        _check(lib().stencil_server_fetch(self._h, ticket, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def release(self, ticket):
        _check(lib().stencil_server_release(self._h, ticket))
        self._n.pop(ticket, None)

    def stats(self):
        st = ServerStats()
        _check(lib().stencil_server_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            lib().stencil_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stencil_release_workspace():
    _check(lib().stencil_release_workspace())


# ------------------------------------------------------------------ launch-shape tuning
def stencil_autotune(u, h, call, sweeps=0, stream=None):
    """Times the candidate launch shapes of `call` on u's grid shape (scratch arrays of
    the library's own) and records the fastest; returns (chunk, depth, ms)."""
    g = grid_for(u, h)
    t = Tuning()
    _check(lib().stencil_autotune(ctypes.byref(g), int(call), int(sweeps), ctypes.byref(t), _stream(stream)))
    return t.chunk, t.depth, t.ms


def stencil_tuning_set(u, h, call, chunk=0, depth=0, ms=0.0):
    """Records a launch shape for (device, call, u's grid); chunk=None removes it."""
    g = grid_for(u, h)
    if chunk is None:
        _check(lib().stencil_tuning_set(ctypes.byref(g), int(call), None))
    else:
        t = Tuning(int(chunk), int(depth), float(ms))
        _check(lib().stencil_tuning_set(ctypes.byref(g), int(call), ctypes.byref(t)))


def stencil_tuning_get(u, h, call):
    """(chunk, depth, ms) recorded for (device, call, u's grid), or None."""
    g = grid_for(u, h)
    t = Tuning()
    rc = lib().stencil_tuning_get(ctypes.byref(g), int(call), ctypes.byref(t))
    if rc == -7:
        return None
    _check(rc)
    return t.chunk, t.depth, t.ms


def stencil_tuning_clear():
    _check(lib().stencil_tuning_clear())


def stencil_tuning_save(path):
    _check(lib().stencil_tuning_save(os.fsencode(path)))


def stencil_tuning_load(path):
    _check(lib().stencil_tuning_load(os.fsencode(path)))


def stencil_device_status(clear=False):
    """Bits of the bounded device waits that ran out on the current device (0: none);
    synchronises the device."""
    v = ctypes.c_uint32(0)
    _check(lib().stencil_device_status(ctypes.byref(v), 1 if clear else 0))
    return int(v.value)
