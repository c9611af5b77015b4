"""5/7-point finite differences with red-black colouring (op = STENCIL_OP_FD) on the
GPU against the oracle: apply, red-black GS (Algorithm 1's pass order), Jacobi and the
residual with its norms, on several shapes and pitches."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1810_04033_gb300 as st
import synth
from tests import dense_reference as dr
from tests.parity_util import TOL_F64, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

SHAPES = [(3, (1, 1, 1)), (3, (2, 3, 4)), (3, (17, 9, 6)), (3, (64, 40, 33)),
          (2, (1, 1)), (2, (5, 3)), (2, (300, 41)), (2, (1000, 777))]
FD = st.OP_FD


def _apply_err(got, ref, u, h):
    denom = max(np.max(np.abs(ref)), (4 * u.ndim / h ** 2) * np.max(np.abs(u)) * 1e-3)
    return float(np.max(np.abs(got - ref)) / denom)


@pytest.mark.parametrize("dim,n", SHAPES)
@pytest.mark.parametrize("pad", [0, 3])
def test_fd_apply(dim, n, pad):
    h = 1.0 / max(n)
    u = synth.uniform_field(synth.grid_shape(dim, n), 900 + sum(n), zero_bc=False)
    yd = to_dev(np.full(u.shape, np.nan), pad=pad)
    st.stencil_apply(to_dev(u, pad=pad), yd, h, st.FORM_STENCIL, op=FD)
    torch.cuda.synchronize()
    assert _apply_err(to_host(yd), oracle.fd_apply(u, h), u, h) <= TOL_F64


@pytest.mark.parametrize("dim,n", SHAPES)
@pytest.mark.parametrize("sweeps", [1, 3])
def test_fd_gs_redblack(dim, n, sweeps):
    h = 1.0 / max(n)
    u0 = synth.uniform_field(synth.grid_shape(dim, n), 910 + sum(n), zero_bc=False)
    f = synth.uniform_field(u0.shape, 911 + sum(n))
    ud = to_dev(u0, pad=2)
    st.stencil_smooth_coloured(ud, to_dev(f, pad=2), h, sweeps, op=FD)
    torch.cuda.synchronize()
    got = to_host(ud)
    assert rel_err(got, oracle.fd_gs_redblack(u0, f, h, sweeps)) <= TOL_F64
    inner = dr.interior_mask(u0.shape)
    assert np.array_equal(got[~inner], u0[~inner])


@pytest.mark.parametrize("dim,n", SHAPES)
@pytest.mark.parametrize("sweeps,omega", [(1, 2.0 / 3.0), (4, 0.8), (3, 1.2)])
def test_fd_jacobi(dim, n, sweeps, omega):
    h = 1.0 / max(n)
    u0 = synth.uniform_field(synth.grid_shape(dim, n), 920 + sum(n), zero_bc=False)
    f = synth.uniform_field(u0.shape, 921 + sum(n))
    ud = to_dev(u0)
    st.stencil_smooth_jacobi(ud, to_dev(f), torch.empty_like(ud), h, sweeps, omega, op=FD)
    od = torch.empty_like(ud)
    st.stencil_jacobi_step(to_dev(u0), to_dev(f), od, h, omega, op=FD)
    torch.cuda.synchronize()
    assert rel_err(to_host(ud), oracle.fd_jacobi(u0, f, h, omega, sweeps)) <= TOL_F64
    assert rel_err(to_host(od), oracle.fd_jacobi(u0, f, h, omega, 1)) <= TOL_F64


@pytest.mark.parametrize("dim,n", SHAPES)
def test_fd_residual_and_norms(dim, n):
    h = 1.0 / max(n)
    u = synth.uniform_field(synth.grid_shape(dim, n), 930 + sum(n), zero_bc=False)
    f = synth.uniform_field(u.shape, 931 + sum(n))
    rref, nref = oracle.fd_residual(u, f, h)
    rd = to_dev(np.full(u.shape, np.nan), pad=1)
    nrm = st.stencil_residual(to_dev(u, pad=1), to_dev(f, pad=1), h, r=rd, op=FD)
    nrm2 = st.stencil_residual(to_dev(u, pad=1), to_dev(f, pad=1), h, op=FD)
    torch.cuda.synchronize()
    assert _apply_err(to_host(rd), rref, u, h) <= TOL_F64
    got = nrm.cpu().numpy()
    assert abs(got[1] - nref[1]) <= 1e-12 * nref[1]
    assert abs(got[0] - nref[0]) <= 1e-11 * nref[0]
    assert np.array_equal(got, nrm2.cpu().numpy())  # deterministic, with or without r


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 24)])
def test_fd_gs_converges_to_closed_form(dim, n):
    h = 1.0 / n
    modes = (2, 1, 1)
    f = synth.zero_boundary(np.ascontiguousarray(dr.sine_mode(dim, n, modes)))
    lam = sum(2 - 2 * math.cos(m * math.pi * h) for m in modes[:dim])
    uh = h * h * f / lam
    ud = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    st.stencil_smooth_coloured(ud, to_dev(f), h, 6000, op=FD)
    torch.cuda.synchronize()
    assert rel_err(to_host(ud), uh) <= 1e-9
