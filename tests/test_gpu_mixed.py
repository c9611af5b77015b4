"""GPU parity of the reduced-precision smoother and the iterative refinement.

FP32 sweeps against the FP32-arithmetic oracle (1e-5 relative max norm: rounding-order
differences only); bf16-storage sweeps against the bf16-emulating oracle (2e-2: a few
bf16 units); every refinement iterate against the oracle's iterate of the same
algorithm; the converged solution against the closed-form discrete solution.
"""
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

TOL_F32 = 1e-5
TOL_BF16 = 2e-2


def _bf16_bits(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


def _bits_to_f64(b):
    return torch.from_numpy(b.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()


def _bf16_iterate_bound(hist, k, sweeps=8):
    """Bound on |x_k(GPU) - x_k(oracle)|_inf / |x_k|_inf for bf16-storage refinement.

    Both sides run the same algorithm; their FP32 arithmetic differs in rounding order
    (FMA contraction), so a bf16 store can round to the other neighbour: one bf16 unit,
    at most 2^-7 of the stored value.  A GS update is a convex combination of its
    neighbours (3D weights (2 E + C)/32 sum to 1), so a difference does not grow in the
    max norm through later updates; each of the `sweeps` inner sweeps, and the bf16
    rounding of the residual, adds at most one unit.  Correction i thus differs by at
    most (sweeps + 1) 2^-7 |e_i|_inf, and x_k = e_1 + ... + e_k."""
    prev = np.zeros_like(hist[0])
    total = 0.0
    for i in range(k):
        total += float(np.max(np.abs(hist[i] - prev)))
        prev = hist[i]
    return (sweeps + 1) * 2.0 ** -7 * total / float(np.max(np.abs(hist[k - 1])))


@pytest.mark.parametrize("n", [(8, 8, 8), (33, 9, 7), (64, 40, 20), (3, 70, 35)])
def test_fp32_gs_matches_fp32_oracle(n):
    h = 1.0 / max(n)
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 2000 + sum(n), zero_bc=False).astype(np.float32)
    f = synth.uniform_field(shape, 2001 + sum(n)).astype(np.float32)
    for sweeps in (1, 4):
        ref = oracle.gs_coloured_f32(u0, f, h, sweeps).astype(np.float64)
        ud = torch.from_numpy(u0).cuda()
        st.stencil_smooth_coloured(ud, torch.from_numpy(f).cuda(), h, sweeps)
        torch.cuda.synchronize()
        assert rel_err(ud.double().cpu().numpy(), ref) <= TOL_F32, sweeps


@pytest.mark.parametrize("n", [(8, 8, 8), (33, 9, 7), (40, 31, 17)])
def test_bf16_gs_matches_bf16_oracle(n):
    h = 1.0 / max(n)
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 2100 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 2101 + sum(n))
    ub, fb = _bf16_bits(u0), _bf16_bits(f)
    for sweeps in (1, 3):
        ref = _bits_to_f64(oracle.gs_coloured_bf16(ub, fb, h, sweeps))
        ud = torch.from_numpy(ub.view(np.int16)).view(torch.bfloat16).cuda()
        fd = torch.from_numpy(fb.view(np.int16)).view(torch.bfloat16).cuda()
        st.stencil_smooth_coloured(ud, fd, h, sweeps)
        torch.cuda.synchronize()
        assert rel_err(ud.double().cpu().numpy(), ref) <= TOL_BF16, sweeps


@pytest.mark.parametrize("prec,tol", [(st.F64, TOL_F64), (st.F32, 1e-5), (st.BF16, None)])
def test_refinement_iterates_match_oracle(prec, tol):
    """Iterate k of the GPU refinement against iterate k of the oracle (same algorithm
    in the same precisions), k = 1..4; error relative to the iterate's max norm (bf16:
    the bound of _bf16_iterate_bound)."""
    n = 24
    h = 1.0 / n
    f = synth.sin_rhs(3, n, (2, 3, 1))
    prec_o = {st.F64: 0, st.F32: 1, st.BF16: 2}[prec]
    _, _, k, _, hist = oracle.ir_solve(np.zeros_like(f), f, h, 0.0, 4, 8, prec_o, keep_history=True)
    for it in range(1, 5):
        ud = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
        res = st.stencil_solve(ud, to_dev(f), h, rel_tol=0.0, max_outer=it, inner_sweeps=8, inner_dtype=prec)
        assert res["iterations"] == it
        bound = tol if tol is not None else _bf16_iterate_bound(hist, it)
        assert rel_err(to_host(ud), hist[it - 1]) <= bound, it


@pytest.mark.parametrize("prec", [st.F64, st.F32, st.BF16])
def test_refinement_converges_to_closed_form(prec):
    """Manufactured sin(2 pi x) sin(3 pi y) sin(pi z) problem at n = 32, solved to a
    relative residual of 1e-10: the result is the closed-form discrete solution
    h^2 f / lambda_S(theta) to within kappa * 1e-10."""
    n = 32
    h = 1.0 / n
    modes = (2, 3, 1)
    f = synth.sin_rhs(3, n, modes)
    uh = h * h * f / dr.symbol(3, [m * math.pi * h for m in modes])
    ud = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    res = st.stencil_solve(ud, to_dev(f), h, rel_tol=1e-10, max_outer=20000, inner_sweeps=8, inner_dtype=prec)
    assert res["converged"]
    assert res["relres"] <= 1e-10
    hist = res["history"]
    assert hist[0] == pytest.approx(1.0)
    assert rel_err(to_host(ud), uh) < 2e-7
    # the FP64 oracle's plain GS reaches the same solution
    if prec == st.F64:
        xo, _, ko, conv = oracle.ir_solve(np.zeros_like(f), f, h, 1e-10, 20000, 8, 0)
        assert conv and abs(ko - res["iterations"]) <= 1


def test_solve_reports_not_converged_and_keeps_iterate():
    n = 16
    h = 1.0 / n
    f = synth.uniform_field(synth.grid_shape(3, n), 7)
    ud = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    res = st.stencil_solve(ud, to_dev(f), h, rel_tol=1e-12, max_outer=3, inner_sweeps=2, inner_dtype=st.F32)
    assert not res["converged"] and res["iterations"] == 3
    assert len(res["history"]) == 4 and res["history"][-1] < res["history"][0]
    assert float(ud.abs().max()) > 0


@pytest.mark.parametrize("n", [(33, 9, 7), (64, 40, 20), (130, 61, 45)])
def test_fp32_gs_padded_matches_fp32_oracle(n):
    """FP32 sweeps on arrays whose pitch is a multiple of 4 floats (the TMA-staged
    kernel): several tiles with ragged tails, nonzero Dirichlet data."""
    h = 1.0 / max(n)
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 2200 + sum(n), zero_bc=False).astype(np.float32)
    f = synth.uniform_field(shape, 2201 + sum(n)).astype(np.float32)
    pad = (-shape[2]) % 4 or 4
    for sweeps in (1, 4):
        ref = oracle.gs_coloured_f32(u0, f, h, sweeps).astype(np.float64)
        ud = to_dev(u0, pad, torch.float32)
        fd = to_dev(f, pad, torch.float32)
        assert ud.stride(1) % 4 == 0
        st.stencil_smooth_coloured(ud, fd, h, sweeps)
        torch.cuda.synchronize()
        got = ud.double().cpu().numpy()
        assert rel_err(got, ref) <= TOL_F32, sweeps
        b = np.ones(shape, dtype=bool)
        b[1:-1, 1:-1, 1:-1] = False
        assert np.array_equal(got[b], u0.astype(np.float64)[b])


def test_refinement_iterates_match_oracle_padded_fp32():
    """FP32-inner refinement on a pitch that is a multiple of 4 (TMA-staged inner
    sweeps): iterate k against the oracle's iterate k."""
    n = 24
    h = 1.0 / n
    f = synth.sin_rhs(3, n, (2, 3, 1))
    _, _, k, _, hist = oracle.ir_solve(np.zeros_like(f), f, h, 0.0, 3, 8, 1, keep_history=True)
    for it in range(1, 4):
        ud = to_dev(np.zeros_like(f), 3)
        fd = to_dev(f, 3)
        assert ud.stride(1) % 4 == 0
        res = st.stencil_solve(ud, fd, h, rel_tol=0.0, max_outer=it, inner_sweeps=8, inner_dtype=st.F32)
        assert res["iterations"] == it
        assert rel_err(to_host(ud), hist[it - 1]) <= 1e-5, it


@pytest.mark.parametrize("n", [(33, 9, 7), (100, 40, 20), (100, 64, 12)])
def test_bf16_gs_padded_matches_bf16_oracle(n):
    """bf16-storage sweeps on arrays whose pitch is a multiple of 8 (the TMA-staged
    kernel): several tiles with ragged tails, nonzero Dirichlet data; (100, 64, 12)
    also has tiles whose computed vertices are all interior (the edge-free path)."""
    h = 1.0 / max(n)
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 2300 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 2301 + sum(n))
    ub, fb = _bf16_bits(u0), _bf16_bits(f)
    pad = (-shape[2]) % 8 or 8
    for sweeps in (1, 3):
        ref = _bits_to_f64(oracle.gs_coloured_bf16(ub, fb, h, sweeps))
        ud = to_dev(_bits_to_f64(ub), pad, torch.bfloat16)
        fd = to_dev(_bits_to_f64(fb), pad, torch.bfloat16)
        assert ud.stride(1) % 8 == 0
        st.stencil_smooth_coloured(ud, fd, h, sweeps)
        torch.cuda.synchronize()
        assert rel_err(ud.double().cpu().numpy(), ref) <= TOL_BF16, sweeps


def test_refinement_iterates_match_oracle_padded_bf16():
    """bf16-inner refinement on a pitch that is a multiple of 8 (TMA-staged inner
    sweeps): iterate k against the oracle's iterate k."""
    n = 24
    h = 1.0 / n
    f = synth.sin_rhs(3, n, (2, 3, 1))
    _, _, k, _, hist = oracle.ir_solve(np.zeros_like(f), f, h, 0.0, 3, 8, 2, keep_history=True)
    for it in range(1, 4):
        ud = to_dev(np.zeros_like(f), 7)
        fd = to_dev(f, 7)
        assert ud.stride(1) % 8 == 0
        res = st.stencil_solve(ud, fd, h, rel_tol=0.0, max_outer=it, inner_sweeps=8, inner_dtype=st.BF16)
        assert res["iterations"] == it
        assert rel_err(to_host(ud), hist[it - 1]) <= _bf16_iterate_bound(hist, it), it
