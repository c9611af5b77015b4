"""Caller-owned workspaces: the smoothers and the residual with a `ws` buffer of
stencil_workspace_size bytes give the same bits as with the library's own workspace,
match the oracle, and allocate no device memory."""
import numpy as np
import pytest
import torch

import oracle
import paper_1810_04033_gb300 as st
import synth
from tests.parity_util import TOL_F64, apply_err, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = [(3, (40, 33, 20), 7), (3, (21, 14, 9), 0), (2, (300, 130), 7), (2, (57, 40), 0)]


def _ws(u, h, call, sweeps):
    n = st.stencil_workspace_size(u, h, call, sweeps)
    # a zero-size request still gets a real buffer (a NULL pointer would select the
    # library's own workspace)
    return torch.empty(max(n, 1), dtype=torch.uint8, device=u.device)


@pytest.mark.parametrize("dim,n,pad", CASES)
def test_caller_workspace_gives_identical_bits(dim, n, pad):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 3100 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 3101 + sum(n))
    fd = to_dev(f, pad)
    for sweeps in (1, 4, 5):
        a, b = to_dev(u0, pad), to_dev(u0, pad)
        st.stencil_smooth_coloured(a, fd, h, sweeps)
        st.stencil_smooth_coloured(b, fd, h, sweeps, ws=_ws(b, h, st.CALL_SMOOTH_COLOURED, sweeps))
        torch.cuda.synchronize()
        assert torch.equal(a, b), ("gs", sweeps)
        assert rel_err(to_host(b), oracle.gs_coloured(u0, f, h, sweeps)) <= TOL_F64
        a, b = to_dev(u0, pad), to_dev(u0, pad)
        wa, wb = to_dev(np.zeros(shape), pad), to_dev(np.zeros(shape), pad)
        st.stencil_smooth_jacobi(a, fd, wa, h, sweeps, 2.0 / 3.0)
        st.stencil_smooth_jacobi(b, fd, wb, h, sweeps, 2.0 / 3.0, ws=_ws(b, h, st.CALL_SMOOTH_JACOBI, sweeps))
        torch.cuda.synchronize()
        assert torch.equal(a, b), ("jacobi", sweeps)
        assert rel_err(to_host(b), oracle.jacobi(u0, f, h, 2.0 / 3.0, sweeps)) <= TOL_F64
    ud = to_dev(u0, pad)
    ra, rb = to_dev(np.full(shape, np.nan), pad), to_dev(np.full(shape, np.nan), pad)
    na = st.stencil_residual(ud, fd, h, r=ra)
    ws = _ws(ud, h, st.CALL_RESIDUAL, 0)
    ws.fill_(0xA5)  # the call clears its counter itself
    nb = st.stencil_residual(ud, fd, h, r=rb, ws=ws)
    nc = st.stencil_residual(ud, fd, h, ws=ws)  # again on the same buffer
    torch.cuda.synchronize()
    assert torch.equal(ra, rb) and torch.equal(na, nb) and torch.equal(na, nc)
    rref, _ = oracle.residual(u0, f, h)
    assert apply_err(to_host(rb), rref, u0, h) <= TOL_F64


def test_caller_workspace_allocates_nothing():
    n = (64, 48, 40)
    h = 1.0 / 64
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 3200)
    f = synth.uniform_field(shape, 3201)
    ud, fd, wd = to_dev(u0, 7), to_dev(f, 7), to_dev(np.zeros(shape), 7)
    wgs = _ws(ud, h, st.CALL_SMOOTH_COLOURED, 6)
    wjac = _ws(ud, h, st.CALL_SMOOTH_JACOBI, 6)
    wres = _ws(ud, h, st.CALL_RESIDUAL, 0)
    nrm = torch.empty(2, dtype=torch.float64, device="cuda")

    def calls(own):
        st.stencil_smooth_coloured(ud, fd, h, 6, ws=wgs if own else None)
        st.stencil_smooth_jacobi(ud, fd, wd, h, 6, 0.8, ws=wjac if own else None)
        st.stencil_residual(ud, fd, h, norms2=nrm, ws=wres if own else None)

    calls(False)  # loads the kernels
    torch.cuda.synchronize()
    st.stencil_release_workspace()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    calls(True)
    calls(True)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
