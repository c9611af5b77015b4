"""CPU oracle for the coloured stencil codes (test infrastructure only).

Plain FP64 C (oracle.c) behind ctypes.  Only the tests, the smoke check and the
CPU-baseline leg of bench.py use this package; the GPU library never imports it.
Arrays are numpy, C-contiguous, x fastest: shape (nz+1, ny+1, nx+1) in 3D and
(ny+1, nx+1) in 2D.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        u16p = ctypes.POINTER(ctypes.c_uint16)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        ci, cd = ctypes.c_int, ctypes.c_double
        sig = {
            "oracle_q1_element_matrix": (None, [ci, cd, dp]),
            "oracle_stencil_weight": (cd, [ci, ci, ci, ci]),
            "oracle_apply_elementwise": (None, [ci, i64p, cd, dp, dp, ci]),
            "oracle_apply_stencil": (None, [ci, i64p, cd, dp, dp, ci]),
            "oracle_gs_coloured": (None, [ci, i64p, cd, dp, dp, ci, ci]),
            "oracle_gs_coloured_f32": (None, [ci, i64p, cd, fp, fp, ci]),
            "oracle_gs_coloured_bf16": (None, [ci, i64p, cd, u16p, u16p, ci]),
            "oracle_jacobi": (None, [ci, i64p, cd, dp, dp, dp, cd, ci, ci]),
            "oracle_residual": (None, [ci, i64p, cd, dp, dp, dp, dp, ci]),
            "oracle_residual_ld": (None, [ci, i64p, cd, dp, dp, dp]),
            "oracle_ir_solve": (ci, [ci, i64p, cd, dp, dp, cd, ci, ci, ci, dp, dp,
                                     ctypes.POINTER(ctypes.c_int)]),
            "oracle_patch_halo_fill": (None, [i32p, i32p, i64p, dp]),
            "oracle_patch_smooth": (None, [i32p, i32p, i64p, dp, dp, ci, ci]),
            "oracle_mg_levels": (ci, [ci, i64p, ci]),
            "oracle_mg_restrict": (None, [ci, i64p, i64p, dp, dp]),
            "oracle_mg_prolong_add": (None, [ci, i64p, i64p, dp, dp]),
            "oracle_mg_vcycle": (None, [ci, i64p, cd, dp, dp, ci, ci, ci, ci]),
            "oracle_mg_solve": (ci, [ci, i64p, cd, dp, dp, cd, ci, ci, ci, ci, ci, dp,
                                     ctypes.POINTER(ctypes.c_int)]),
            "oracle_fd_weight": (cd, [ci, ci, ci, ci]),
            "oracle_fd_apply": (None, [ci, i64p, cd, dp, dp]),
            "oracle_fd_gs_redblack": (None, [ci, i64p, cd, dp, dp, ci]),
            "oracle_fd_jacobi": (None, [ci, i64p, cd, dp, dp, dp, cd, ci]),
            "oracle_fd_residual": (None, [ci, i64p, cd, dp, dp, dp, dp]),
            "oracle_cost_diagonal": (cd, [ci, i64p, ci, ci, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]),
            "oracle_fd_gs_redblack_cost": (None, [ci, i64p, cd, dp, dp, ci, ci, ci]),
            "oracle_f32_to_bf16": (ctypes.c_uint16, [ctypes.c_float]),
            "oracle_bf16_to_f32": (ctypes.c_float, [ctypes.c_uint16]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _grid(shape):
    """(dim, int64[3] cells per axis) from an array shape (z,y,x) or (y,x)."""
    if len(shape) == 3:
        n = np.array([shape[2] - 1, shape[1] - 1, shape[0] - 1], dtype=np.int64)
        return 3, n
    n = np.array([shape[1] - 1, shape[0] - 1, 0], dtype=np.int64)
    return 2, n


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def element_matrix(dim, h):
    nv = 1 << dim
    K = np.zeros((nv, nv))
    lib().oracle_q1_element_matrix(dim, h, _ptr(K, ctypes.c_double))
    return K


def stencil_weight(dim, dx, dy, dz=0):
    return lib().oracle_stencil_weight(dim, dx, dy, dz)


def apply_elementwise(u, h, nthreads=1):
    u = _f64(u)
    dim, n = _grid(u.shape)
    y = np.empty_like(u)
    lib().oracle_apply_elementwise(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                                   _ptr(y, ctypes.c_double), nthreads)
    return y


def apply_stencil(u, h, nthreads=1):
    u = _f64(u)
    dim, n = _grid(u.shape)
    y = np.empty_like(u)
    lib().oracle_apply_stencil(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                               _ptr(y, ctypes.c_double), nthreads)
    return y


def gs_coloured(u, f, h, sweeps, nthreads=1):
    """Returns a new array: `sweeps` coloured GS sweeps applied to a copy of u."""
    u = _f64(u).copy()
    f = _f64(f)
    dim, n = _grid(u.shape)
    lib().oracle_gs_coloured(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                             _ptr(f, ctypes.c_double), sweeps, nthreads)
    return u


def gs_coloured_f32(u, f, h, sweeps):
    u = np.ascontiguousarray(u, dtype=np.float32).copy()
    f = np.ascontiguousarray(f, dtype=np.float32)
    dim, n = _grid(u.shape)
    lib().oracle_gs_coloured_f32(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_float),
                                 _ptr(f, ctypes.c_float), sweeps)
    return u


def gs_coloured_bf16(u_bits, f_bits, h, sweeps):
    """u_bits, f_bits: uint16 arrays of bf16 bit patterns."""
    u = np.ascontiguousarray(u_bits, dtype=np.uint16).copy()
    f = np.ascontiguousarray(f_bits, dtype=np.uint16)
    dim, n = _grid(u.shape)
    lib().oracle_gs_coloured_bf16(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_uint16),
                                  _ptr(f, ctypes.c_uint16), sweeps)
    return u


def jacobi(u, f, h, omega, sweeps, nthreads=1):
    u = _f64(u).copy()
    f = _f64(f)
    work = np.empty_like(u)
    dim, n = _grid(u.shape)
    lib().oracle_jacobi(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                        _ptr(f, ctypes.c_double), _ptr(work, ctypes.c_double), omega, sweeps,
                        nthreads)
    return u


def residual(u, f, h, nthreads=1):
    """Returns (r, [sum r^2, sum f^2])."""
    u = _f64(u)
    f = _f64(f)
    r = np.empty_like(u)
    nrm = np.zeros(2)
    dim, n = _grid(u.shape)
    lib().oracle_residual(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                          _ptr(f, ctypes.c_double), _ptr(r, ctypes.c_double),
                          _ptr(nrm, ctypes.c_double), nthreads)
    return r, nrm


def residual_norms_ld(u, f, h):
    """[sum r^2, sum f^2] computed in long double (returned as doubles)."""
    u = _f64(u)
    f = _f64(f)
    nrm = np.zeros(2)
    dim, n = _grid(u.shape)
    lib().oracle_residual_ld(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                             _ptr(f, ctypes.c_double), _ptr(nrm, ctypes.c_double))
    return nrm


def ir_solve(x0, f, h, tol, max_outer, inner_sweeps, inner_prec, keep_history=False):
    """Returns (x, relres history, iterations, converged[, x history])."""
    x = _f64(x0).copy()
    f = _f64(f)
    dim, n = _grid(x.shape)
    relres = np.zeros(max_outer + 1)
    hist = np.zeros((max_outer,) + x.shape) if keep_history else None
    conv = ctypes.c_int(0)
    k = lib().oracle_ir_solve(dim, _ptr(n, ctypes.c_int64), h, _ptr(x, ctypes.c_double),
                              _ptr(f, ctypes.c_double), tol, max_outer, inner_sweeps,
                              inner_prec, _ptr(relres, ctypes.c_double),
                              _ptr(hist, ctypes.c_double) if keep_history else None,
                              ctypes.byref(conv))
    out = (x, relres[:k + 1], k, bool(conv.value))
    if keep_history:
        out = out + (hist[:k],)
    return out


def coarse_shape(shape):
    """Vertex-array shape of the coarse grid of the multigrid hierarchy (None if the
    grid is the coarsest): n/2 when all n are even, ceil(n/2) when all n are equal."""
    dim, n = _grid(shape)
    n = [int(v) for v in n[:dim]]
    if min(n) < 4 or (any(v % 2 for v in n) and len(set(n)) > 1):
        return None
    nc = [(v + 1) // 2 for v in n]
    return tuple(v + 1 for v in reversed(nc))


def mg_levels(shape, max_levels=64):
    """Grids in the multigrid hierarchy of a vertex array of this shape."""
    dim, n = _grid(shape)
    return lib().oracle_mg_levels(dim, _ptr(n, ctypes.c_int64), max_levels)


def mg_restrict(rf, coarse=None):
    """Restriction R rf onto the coarse grid of rf's grid (or onto `coarse`, a shape)."""
    rf = _f64(rf)
    dim, nf = _grid(rf.shape)
    cs = coarse if coarse is not None else coarse_shape(rf.shape)
    _, nc = _grid(cs)
    rc = np.zeros(cs)
    lib().oracle_mg_restrict(dim, _ptr(nf, ctypes.c_int64), _ptr(nc, ctypes.c_int64),
                             _ptr(rf, ctypes.c_double), _ptr(rc, ctypes.c_double))
    return rc


def mg_prolong_add(ec, uf):
    """uf + P ec on the fine interior (uf's boundary unchanged)."""
    ec = _f64(ec)
    u = _f64(uf).copy()
    dim, nf = _grid(u.shape)
    _, nc = _grid(ec.shape)
    lib().oracle_mg_prolong_add(dim, _ptr(nf, ctypes.c_int64), _ptr(nc, ctypes.c_int64),
                                _ptr(ec, ctypes.c_double), _ptr(u, ctypes.c_double))
    return u


def mg_vcycle(u0, f, h, levels, pre=2, post=2, coarse_sweeps=20):
    u = _f64(u0).copy()
    f = _f64(f)
    dim, n = _grid(u.shape)
    lib().oracle_mg_vcycle(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                           _ptr(f, ctypes.c_double), levels, pre, post, coarse_sweeps)
    return u


def mg_solve(u0, f, h, tol, max_cycles, levels=64, pre=2, post=2, coarse_sweeps=20):
    """Returns (u, relres history, cycles, converged)."""
    u = _f64(u0).copy()
    f = _f64(f)
    dim, n = _grid(u.shape)
    levels = min(levels, mg_levels(u.shape))
    relres = np.zeros(max_cycles + 1)
    conv = ctypes.c_int(0)
    k = lib().oracle_mg_solve(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                              _ptr(f, ctypes.c_double), tol, max_cycles, levels, pre, post,
                              coarse_sweeps, _ptr(relres, ctypes.c_double), ctypes.byref(conv))
    return u, relres[:k + 1], k, bool(conv.value)


def fd_weight(dim, dx, dy, dz=0):
    return lib().oracle_fd_weight(dim, dx, dy, dz)


def fd_apply(u, h):
    u = _f64(u)
    dim, n = _grid(u.shape)
    y = np.empty_like(u)
    lib().oracle_fd_apply(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double), _ptr(y, ctypes.c_double))
    return y


def fd_gs_redblack(u0, f, h, sweeps):
    u = _f64(u0).copy()
    f = _f64(f)
    dim, n = _grid(u.shape)
    lib().oracle_fd_gs_redblack(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                                _ptr(f, ctypes.c_double), sweeps)
    return u


def fd_jacobi(u0, f, h, omega, sweeps):
    u = _f64(u0).copy()
    f = _f64(f)
    w = np.empty_like(u)
    dim, n = _grid(u.shape)
    lib().oracle_fd_jacobi(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double), _ptr(f, ctypes.c_double),
                           _ptr(w, ctypes.c_double), omega, sweeps)
    return u


def fd_residual(u, f, h):
    u = _f64(u)
    f = _f64(f)
    dim, n = _grid(u.shape)
    r = np.empty_like(u)
    nrm = np.zeros(2)
    lib().oracle_fd_residual(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double), _ptr(f, ctypes.c_double),
                             _ptr(r, ctypes.c_double), _ptr(nrm, ctypes.c_double))
    return r, nrm


def cost_diagonal(shape, mode, kmax, i, j, k=0):
    dim, n = _grid(shape)
    return lib().oracle_cost_diagonal(dim, _ptr(n, ctypes.c_int64), mode, kmax, i, j, k)


def fd_gs_redblack_cost(u0, f, h, sweeps, mode, kmax):
    u = _f64(u0).copy()
    f = _f64(f)
    dim, n = _grid(u.shape)
    lib().oracle_fd_gs_redblack_cost(dim, _ptr(n, ctypes.c_int64), h, _ptr(u, ctypes.c_double),
                                     _ptr(f, ctypes.c_double), sweeps, mode, kmax)
    return u


def patch_halo_fill(lat, np_sizes, offsets, u_all):
    lat = np.ascontiguousarray(lat, dtype=np.int32)
    nps = np.ascontiguousarray(np_sizes, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    u = _f64(u_all).copy()
    lib().oracle_patch_halo_fill(_ptr(lat, ctypes.c_int32), _ptr(nps, ctypes.c_int32),
                                 _ptr(off, ctypes.c_int64), _ptr(u, ctypes.c_double))
    return u


def patch_smooth(lat, np_sizes, offsets, u_all, f_all, sweeps, nthreads=1):
    lat = np.ascontiguousarray(lat, dtype=np.int32)
    nps = np.ascontiguousarray(np_sizes, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    u = _f64(u_all).copy()
    f = _f64(f_all)
    lib().oracle_patch_smooth(_ptr(lat, ctypes.c_int32), _ptr(nps, ctypes.c_int32),
                              _ptr(off, ctypes.c_int64), _ptr(u, ctypes.c_double),
                              _ptr(f, ctypes.c_double), sweeps, nthreads)
    return u


def f32_to_bf16(x):
    return lib().oracle_f32_to_bf16(float(x))


def bf16_to_f32(b):
    return lib().oracle_bf16_to_f32(int(b))
