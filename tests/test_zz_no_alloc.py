"""The allocation-free residual entry point (stencil_residual_noalloc).

It exists for callers that cannot let the library call cudaMalloc (a device-wide
synchronisation they cannot afford, device memory already owned by another allocator,
or a no-allocation-after-start-up rule).  The test calls it through the C ABI twice in
a row, on different grids, and checks each result against the allocating
stencil_residual and against the CPU oracle within the FP64 parity tolerance; it also
checks that the second call leaves the device's free memory unchanged and that an
oversize grid is refused.
This file is collected last so that a run stopping at the first failure has already
run every other test; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1810_04033_gb300 as st
import synth
from tests.parity_util import TOL_F64, apply_err, to_dev, to_host

pytestmark = pytest.mark.gpu


def _case(dim, n, seed):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u = synth.uniform_field(shape, seed, zero_bc=False)
    f = synth.uniform_field(shape, seed + 1)
    return h, u, f


def _noalloc_call(h, ud, fd, r_new, n_new):
    g = st.grid_for(ud, h)
    rc = st.lib().stencil_residual_noalloc(ctypes.byref(g), ctypes.c_void_p(ud.data_ptr()),
                                           ctypes.c_void_p(fd.data_ptr()),
                                           ctypes.c_void_p(r_new.data_ptr()),
                                           ctypes.c_void_p(n_new.data_ptr()), None)
    assert rc == 0, st.lib().stencil_last_error()
    torch.cuda.synchronize()


def _compare(h, u, ud, fd, r_new, n_new):
    r_ref = torch.full_like(ud, float("nan"))
    n_ref = st.stencil_residual(ud, fd, h, r=r_ref)
    torch.cuda.synchronize()
    assert apply_err(to_host(r_new), to_host(r_ref), u, h) <= TOL_F64
    a, b = n_new.cpu().numpy(), n_ref.cpu().numpy()
    assert abs(a[1] - b[1]) <= TOL_F64 * b[1]
    assert abs(a[0] - b[0]) <= TOL_F64 * max(b[0], 1e-300) * 10
    # and against the oracle: r everywhere, the norm sums as in the parity tests
    rref, nref = oracle.residual(u, to_host(fd), h)
    assert apply_err(to_host(r_new), rref, u, h) <= TOL_F64
    assert abs(a[1] - nref[1]) <= 1e-12 * nref[1]
    assert abs(a[0] - nref[0]) <= 1e-11 * nref[0]


def test_noalloc_residual_matches_allocating_entry_point_twice_in_a_row():
    torch.cuda.init()
    h1, u1, f1 = _case(3, (40, 17, 12), 901)
    h2, u2, f2 = _case(2, (130, 67), 903)
    u1d, f1d = to_dev(u1), to_dev(f1)
    u2d, f2d = to_dev(u2), to_dev(f2)
    r1 = torch.full_like(u1d, float("nan"))
    n1 = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    r2 = torch.full_like(u2d, float("nan"))
    n2 = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    _noalloc_call(h1, u1d, f1d, r1, n1)          # first call on the device: set-up
    _compare(h1, u1, u1d, f1d, r1, n1)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    _noalloc_call(h2, u2d, f2d, r2, n2)          # second call in a row, another grid
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before             # the call reserved no device memory
    _compare(h2, u2, u2d, f2d, r2, n2)


def test_noalloc_residual_norms_only_and_oversize_refused():
    h, u, f = _case(3, (33, 9, 7), 905)
    ud, fd = to_dev(u), to_dev(f)
    n = torch.empty(2, dtype=torch.float64, device="cuda")
    st.stencil_residual_noalloc(ud, fd, h, n)          # r = NULL
    ref = st.stencil_residual(ud, fd, h)
    torch.cuda.synchronize()
    assert abs(n[1].item() - ref[1].item()) <= TOL_F64 * ref[1].item()
    # 1023^3 cells: 1024*1024 x-rows > 524288 -> refused before touching memory
    g = st.Grid()
    g.dim, g.dtype = 3, st.F64
    g.n[0], g.n[1], g.n[2] = 1023, 1023, 1023
    g.pitch, g.h = 0, 1.0 / 1023
    rc = st.lib().stencil_residual_noalloc(ctypes.byref(g), ctypes.c_void_p(ud.data_ptr()),
                                           ctypes.c_void_p(fd.data_ptr()), None,
                                           ctypes.c_void_p(n.data_ptr()), None)
    assert rc == -1
    assert "too large" in st.lib().stencil_last_error().decode()
