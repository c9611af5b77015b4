"""GPU parity: every CUDA entry point against the oracle on the same seeded inputs.

Small and ragged grids (several tiles plus a partial tile), padded pitches, the
degenerate one-cell grids, 2D and 3D; FP64 bar 1e-12 relative max norm.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1810_04033_gb300 as st
import synth
from tests.parity_util import TOL_F64, apply_err, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

SHAPES_3D = [(1, 1, 1), (2, 2, 2), (3, 5, 4), (8, 8, 8), (33, 9, 7), (40, 17, 12), (64, 20, 9)]
SHAPES_2D = [(1, 1), (2, 2), (5, 3), (37, 19), (130, 67)]


def _cases():
    for n in SHAPES_3D:
        yield 3, n
    for n in SHAPES_2D:
        yield 2, n


@pytest.mark.parametrize("dim,n", list(_cases()))
@pytest.mark.parametrize("form", [st.FORM_ELEMENTWISE, st.FORM_STENCIL])
@pytest.mark.parametrize("pad", [0, 3])
def test_apply(dim, n, form, pad):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u = synth.uniform_field(shape, 100 + sum(n), zero_bc=False)
    ref = oracle.apply_elementwise(u, h) if form == st.FORM_ELEMENTWISE else oracle.apply_stencil(u, h)
    ud = to_dev(u, pad)
    yd = to_dev(np.full(shape, np.nan), pad)
    st.stencil_apply(ud, yd, h, form)
    torch.cuda.synchronize()
    got = to_host(yd)
    assert apply_err(got, ref, u, h) <= TOL_F64
    assert np.all(got[~_interior(shape)] == 0.0)


def _interior(shape):
    m = np.zeros(shape, dtype=bool)
    m[tuple(slice(1, s - 1) for s in shape)] = True
    return m


@pytest.mark.parametrize("dim,n", list(_cases()))
@pytest.mark.parametrize("pad", [0, 1])
def test_gs_coloured(dim, n, pad):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 200 + sum(n), zero_bc=False)  # nonzero Dirichlet data
    f = synth.uniform_field(shape, 300 + sum(n))
    sweeps = 3
    ref = oracle.gs_coloured(u0, f, h, sweeps)
    ud = to_dev(u0, pad)
    fd = to_dev(f, pad)
    st.stencil_smooth_coloured(ud, fd, h, sweeps)
    torch.cuda.synchronize()
    got = to_host(ud)
    assert rel_err(got, ref) <= TOL_F64
    b = ~_interior(shape)
    assert np.array_equal(got[b], u0[b])


def test_gs_zero_sweeps_is_identity():
    shape = synth.grid_shape(3, 6)
    u0 = synth.uniform_field(shape, 1, zero_bc=False)
    ud = to_dev(u0)
    st.stencil_smooth_coloured(ud, to_dev(u0 * 0), 1 / 6, 0)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(ud), u0)


def _boundary(a):
    """All boundary entries (first/last index on any axis), flattened."""
    m = np.zeros(a.shape, dtype=bool)
    for ax in range(a.ndim):
        idx = [slice(None)] * a.ndim
        idx[ax] = 0
        m[tuple(idx)] = True
        idx[ax] = -1
        m[tuple(idx)] = True
    return a[m]


@pytest.mark.parametrize("dim,n", list(_cases()))
@pytest.mark.parametrize("sweeps,omega", [(1, 2.0 / 3.0), (2, 2.0 / 3.0), (5, 2.0 / 3.0), (3, 1.0), (3, 1.3)])
def test_jacobi(dim, n, sweeps, omega):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 400 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 500 + sum(n))
    ref = oracle.jacobi(u0, f, h, omega, sweeps)
    ud, fd = to_dev(u0), to_dev(f)
    wd = torch.empty_like(ud)
    st.stencil_smooth_jacobi(ud, fd, wd, h, sweeps, omega)
    torch.cuda.synchronize()
    got = to_host(ud)
    assert rel_err(got, ref) <= TOL_F64
    assert np.array_equal(_boundary(got), _boundary(u0))  # Dirichlet data untouched


@pytest.mark.parametrize("dim,n", list(_cases()))
def test_residual_and_norms(dim, n):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u = synth.uniform_field(shape, 600 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 700 + sum(n))
    rref, nref = oracle.residual(u, f, h)
    ud, fd = to_dev(u), to_dev(f)
    rd = torch.full_like(ud, float("nan"))
    norms = st.stencil_residual(ud, fd, h, r=rd)
    torch.cuda.synchronize()
    assert apply_err(to_host(rd), rref, u, h) <= TOL_F64
    got = norms.cpu().numpy()
    if nref[1] > 0:
        assert abs(got[1] - nref[1]) <= 1e-12 * nref[1]
        assert abs(got[0] - nref[0]) <= 1e-11 * max(nref[0], 1e-300) + 1e-12 * nref[1] * 1e-4
    else:
        assert got[0] == 0.0 and got[1] == 0.0
    # norms-only call and determinism: identical bits on repeat
    n2 = st.stencil_residual(ud, fd, h)
    n3 = st.stencil_residual(ud, fd, h)
    torch.cuda.synchronize()
    assert torch.equal(n2, norms) and torch.equal(n3, norms)


def test_gs_converges_to_closed_form_on_gpu():
    """Config-0 shape: 32^3 cells, f = 3 pi^2 sin sin sin, u0 = 0: the GPU iterate
    converges to the closed-form discrete solution h^2 f / lambda_S."""
    import math
    from tests import dense_reference as dr
    n = 32
    h = 1.0 / n
    f = synth.sin_rhs(3, n)
    uh = h * h * f / dr.symbol(3, [math.pi * h] * 3)
    ud = torch.zeros(synth.grid_shape(3, n), dtype=torch.float64, device="cuda")
    fd = to_dev(f)
    prev = np.inf
    for _ in range(10):
        st.stencil_smooth_coloured(ud, fd, h, 1)
        nrm = st.stencil_residual(ud, fd, h).cpu().numpy()
        assert nrm[0] < prev
        prev = nrm[0]
    ref10 = oracle.gs_coloured(np.zeros_like(f), f, h, 10)
    assert rel_err(to_host(ud), ref10) <= TOL_F64
    st.stencil_smooth_coloured(ud, fd, h, 3000)
    torch.cuda.synchronize()
    assert rel_err(to_host(ud), uh) < 1e-9


@pytest.mark.parametrize("dim,n", [(3, (9, 7, 5)), (2, (33, 20))])
def test_jacobi_step_out_of_place(dim, n):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 800, zero_bc=False)
    f = synth.uniform_field(shape, 801)
    ref = oracle.jacobi(u0, f, h, 0.7, 1)
    ud, fd = to_dev(u0), to_dev(f)
    od = torch.full_like(ud, float("nan"))
    st.stencil_jacobi_step(ud, fd, od, h, 0.7)
    torch.cuda.synchronize()
    assert rel_err(to_host(od), ref) <= TOL_F64
    assert np.array_equal(to_host(ud), u0)


@pytest.mark.parametrize("n", [(20, 70, 6), (10, 10, 70), (130, 33, 35), (59, 31, 5)])
def test_gs_multi_tile_and_chunk(n):
    """Grids spanning several (x, y) tiles and several z chunks of the fused sweep."""
    h = 1.0 / max(n)
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 1000 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 1100 + sum(n))
    for sweeps in (1, 2, 5):
        ref = oracle.gs_coloured(u0, f, h, sweeps)
        ud, fd = to_dev(u0), to_dev(f)
        st.stencil_smooth_coloured(ud, fd, h, sweeps)
        torch.cuda.synchronize()
        assert rel_err(to_host(ud), ref) <= TOL_F64, sweeps


@pytest.mark.parametrize("scale", [1e305, 1e-280, 1e-5, 1e12])
@pytest.mark.parametrize("pad", [0, 1])
def test_gs_extreme_magnitudes(scale, pad):
    """Magnitudes outside the fixed-point range take the kernel's FP64 branch; the
    others exercise the tracked bound at unusual scales (odd pitch: register-staged
    kernels; even pitch: TMA-staged)."""
    n = (12, 9, 14)
    h = 1.0 / 14
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 77, zero_bc=False) * scale
    f = synth.uniform_field(shape, 78) * scale
    ref = oracle.gs_coloured(u0, f, h, 3)
    ud, fd = to_dev(u0, pad), to_dev(f, pad)
    st.stencil_smooth_coloured(ud, fd, h, 3)
    jd = to_dev(u0, pad)
    st.stencil_smooth_jacobi(jd, fd, to_dev(np.zeros(shape), pad), h, 4, 0.8)
    torch.cuda.synchronize()
    assert rel_err(to_host(ud), ref) <= TOL_F64
    assert rel_err(to_host(jd), oracle.jacobi(u0, f, h, 0.8, 4)) <= TOL_F64


def test_gs_shrinking_iterate_keeps_relative_accuracy():
    """f = 0: the iterate decays over the sweeps; the tracked bound follows it."""
    n = (16, 16, 16)
    h = 1.0 / 16
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 91)
    f = np.zeros(shape)
    ref = oracle.gs_coloured(u0, f, h, 40)
    ud, fd = to_dev(u0), to_dev(f)
    st.stencil_smooth_coloured(ud, fd, h, 40)
    torch.cuda.synchronize()
    assert rel_err(to_host(ud), ref) <= TOL_F64


@pytest.mark.parametrize("n", [(61, 33, 33), (130, 70, 66), (5, 80, 40)])
def test_out_of_place_ops_multi_tile(n):
    """Apply, Jacobi step and residual on grids spanning several tiles and z chunks."""
    h = 1.0 / max(n)
    shape = synth.grid_shape(3, n)
    u = synth.uniform_field(shape, 1200 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 1300 + sum(n))
    ud, fd = to_dev(u), to_dev(f)
    yd = torch.full_like(ud, float("nan"))
    st.stencil_apply(ud, yd, h, st.FORM_STENCIL)
    od = torch.full_like(ud, float("nan"))
    st.stencil_jacobi_step(ud, fd, od, h, 2.0 / 3.0)
    rd = torch.full_like(ud, float("nan"))
    nrm = st.stencil_residual(ud, fd, h, r=rd)
    torch.cuda.synchronize()
    assert apply_err(to_host(yd), oracle.apply_stencil(u, h), u, h) <= TOL_F64
    assert rel_err(to_host(od), oracle.jacobi(u, f, h, 2.0 / 3.0, 1)) <= TOL_F64
    rref, nref = oracle.residual(u, f, h)
    assert apply_err(to_host(rd), rref, u, h) <= TOL_F64
    got = nrm.cpu().numpy()
    assert abs(got[1] - nref[1]) <= 1e-12 * nref[1]
    assert abs(got[0] - nref[0]) <= 1e-11 * nref[0]


@pytest.mark.parametrize("scale", [1e300, 1e-280, 1e-6])
def test_out_of_place_ops_extreme_and_mixed_magnitudes(scale):
    """Out-of-range magnitudes switch a tile to FP64; a plane-by-plane growing scale
    exercises the rescaling of staged planes."""
    n = (40, 36, 45)
    h = 1.0 / 45
    shape = synth.grid_shape(3, n)
    u = synth.uniform_field(shape, 1400, zero_bc=False) * scale
    z = np.arange(shape[0], dtype=np.float64)[:, None, None]
    u = u * (1.0 + 1e3 * (z / shape[0]) ** 4)  # magnitudes grow along z
    f = synth.uniform_field(shape, 1401) * scale
    ud, fd = to_dev(u), to_dev(f)
    yd = torch.empty_like(ud)
    st.stencil_apply(ud, yd, h, st.FORM_STENCIL)
    od = torch.empty_like(ud)
    st.stencil_jacobi_step(ud, fd, od, h, 0.8)
    torch.cuda.synchronize()
    assert apply_err(to_host(yd), oracle.apply_stencil(u, h), u, h) <= TOL_F64
    assert rel_err(to_host(od), oracle.jacobi(u, f, h, 0.8, 1)) <= TOL_F64
    # the element-wise form on both of its kernels (odd pitch, and 16-byte pairs at an
    # even pitch): warps whose planes leave the fixed-point range part-way up the z
    # column continue in FP64 from that layer, and a growing scale rescales their sums
    ref = oracle.apply_elementwise(u, h)
    for pad in (0, 7):
        ue = to_dev(u, pad)
        ye = to_dev(np.full(shape, np.nan), pad)
        st.stencil_apply(ue, ye, h, st.FORM_ELEMENTWISE)
        torch.cuda.synchronize()
        assert apply_err(to_host(ye), ref, u, h) <= TOL_F64, pad


def test_full_size_sampled_apply_and_gs():
    """512^3 cells at the benchmark's pitch (520: the TMA-staged kernels): the stencil
    apply compared with the oracle on sampled vertices (the oracle evaluates the 3x3x3
    neighbourhood of each sample), then one GS sweep compared everywhere.  The
    benchmark's own calls (both applies, 6- and 50-sweep smoothers, residual) are
    compared everywhere in test_gpu_bench_layout.py."""
    n = 512
    h = 1.0 / n
    shape = synth.grid_shape(3, n)
    u = synth.uniform_field(shape, 1)
    f = synth.sin_rhs(3, n)
    ud, fd = to_dev(u, 7), to_dev(f, 7)
    assert ud.stride(1) == 520
    yd = to_dev(np.zeros(shape), 7)
    st.stencil_apply(ud, yd, h, st.FORM_STENCIL)
    torch.cuda.synchronize()
    y = to_host(yd)
    g = synth.rng(5)
    pts = g.integers(1, n, size=(400, 3))
    pts = np.vstack([pts, [[1, 1, 1], [n - 1, n - 1, n - 1], [1, n - 1, 1], [256, 256, 256]]])
    for k, j, i in pts:
        blk = u[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2]
        ref = oracle.apply_stencil(blk, h)[1, 1, 1]
        assert abs(y[k, j, i] - ref) <= TOL_F64 * max(abs(ref), (16 / 3) / h ** 2 * 1e-3)
    assert np.all(y[0] == 0) and np.all(y[:, :, -1] == 0)
    # one full sweep: oracle on all host cores, compared everywhere
    import os
    st.stencil_smooth_coloured(ud, fd, h, 1)
    ref = oracle.gs_coloured(u, f, h, 1, nthreads=os.cpu_count() or 1)
    torch.cuda.synchronize()
    assert rel_err(to_host(ud), ref) <= TOL_F64


@pytest.mark.parametrize("n", [(200, 150), (61, 300), (29, 29), (31, 130), (45, 601), (70, 514)])
def test_2d_ops_multi_segment(n):
    """2D apply (both forms), GS, Jacobi step and residual over several warp segments
    and row chunks."""
    h = 1.0 / max(n)
    shape = synth.grid_shape(2, n)
    u = synth.uniform_field(shape, 1500 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 1600 + sum(n))
    ud, fd = to_dev(u, pad=5), to_dev(f, pad=5)
    for form, ref in ((st.FORM_ELEMENTWISE, oracle.apply_elementwise(u, h)),
                      (st.FORM_STENCIL, oracle.apply_stencil(u, h))):
        yd = to_dev(np.full(shape, np.nan), pad=5)
        st.stencil_apply(ud, yd, h, form)
        torch.cuda.synchronize()
        assert apply_err(to_host(yd), ref, u, h) <= TOL_F64, form
    od = to_dev(np.full(shape, np.nan), pad=5)
    st.stencil_jacobi_step(ud, fd, od, h, 2.0 / 3.0)
    rd = to_dev(np.full(shape, np.nan), pad=5)
    nrm = st.stencil_residual(ud, fd, h, r=rd)
    torch.cuda.synchronize()
    assert rel_err(to_host(od), oracle.jacobi(u, f, h, 2.0 / 3.0, 1)) <= TOL_F64
    rref, nref = oracle.residual(u, f, h)
    assert apply_err(to_host(rd), rref, u, h) <= TOL_F64
    got = nrm.cpu().numpy()
    assert abs(got[1] - nref[1]) <= 1e-12 * nref[1]
    assert abs(got[0] - nref[0]) <= 1e-11 * nref[0]
    for sweeps in (1, 2, 3, 4, 7):
        gd = to_dev(u, pad=5)
        st.stencil_smooth_coloured(gd, fd, h, sweeps)
        jd = to_dev(u, pad=5)
        st.stencil_smooth_jacobi(jd, fd, to_dev(np.zeros(shape), pad=5), h, sweeps, 2.0 / 3.0)
        torch.cuda.synchronize()
        assert rel_err(to_host(gd), oracle.gs_coloured(u, f, h, sweeps)) <= TOL_F64, sweeps
        assert rel_err(to_host(jd), oracle.jacobi(u, f, h, 2.0 / 3.0, sweeps)) <= TOL_F64, sweeps


@pytest.mark.parametrize("scale", [1e300, 1e-280, 1e-7])
def test_2d_extreme_and_growing_magnitudes(scale):
    n = (70, 90)
    h = 1.0 / 90
    shape = synth.grid_shape(2, n)
    yy = np.arange(shape[0], dtype=np.float64)[:, None]
    u = synth.uniform_field(shape, 1700, zero_bc=False) * scale * (1.0 + 1e3 * (yy / shape[0]) ** 4)
    f = synth.uniform_field(shape, 1701) * scale
    ud, fd = to_dev(u), to_dev(f)
    for form, ref in ((st.FORM_ELEMENTWISE, oracle.apply_elementwise(u, h)),
                      (st.FORM_STENCIL, oracle.apply_stencil(u, h))):
        yd = torch.empty_like(ud)
        st.stencil_apply(ud, yd, h, form)
        torch.cuda.synchronize()
        assert apply_err(to_host(yd), ref, u, h) <= TOL_F64
        # the same at an even pitch (16-byte pairs)
        ue, ye = to_dev(u, 7), to_dev(np.full(shape, np.nan), 7)
        st.stencil_apply(ue, ye, h, form)
        torch.cuda.synchronize()
        assert apply_err(to_host(ye), ref, u, h) <= TOL_F64
    gd = ud.clone()
    st.stencil_smooth_coloured(gd, fd, h, 2)
    od = torch.empty_like(ud)
    st.stencil_jacobi_step(ud, fd, od, h, 0.9)
    torch.cuda.synchronize()
    assert rel_err(to_host(gd), oracle.gs_coloured(u, f, h, 2)) <= TOL_F64
    assert rel_err(to_host(od), oracle.jacobi(u, f, h, 0.9, 1)) <= TOL_F64
    # several sweeps per call: fixed point between sweeps where the bound allows it,
    # FP64 buffers throughout where it does not (1e300)
    gd = ud.clone()
    st.stencil_smooth_coloured(gd, fd, h, 4)
    jd = ud.clone()
    st.stencil_smooth_jacobi(jd, fd, torch.empty_like(ud), h, 4, 0.9)
    torch.cuda.synchronize()
    assert rel_err(to_host(gd), oracle.gs_coloured(u, f, h, 4)) <= TOL_F64
    assert rel_err(to_host(jd), oracle.jacobi(u, f, h, 0.9, 4)) <= TOL_F64


@pytest.mark.parametrize("n", [(130, 300), (57, 40)])
def test_2d_sweeps_unaligned_base(n):
    """Applies, Jacobi step, residual and multi-sweep GS and Jacobi on arrays whose base
    is 8 but not 16-byte aligned (even pitch): the kernels must take their 8-byte
    column path."""
    h = 1.0 / max(n)
    shape = synth.grid_shape(2, n)
    u = synth.uniform_field(shape, 1800 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 1801 + sum(n))

    def shifted(a):
        pitch = shape[1] + 1 + (shape[1] + 1) % 2  # even, > nx + 1
        buf = torch.full((shape[0], pitch), float("nan"), dtype=torch.float64, device="cuda")
        v = buf[:, 1:1 + shape[1]]
        v.copy_(torch.from_numpy(a).cuda())
        assert v.data_ptr() % 16 == 8 and v.stride(0) % 2 == 0
        return v

    ud, fd = shifted(u), shifted(f)
    for form, ref in ((st.FORM_ELEMENTWISE, oracle.apply_elementwise(u, h)),
                      (st.FORM_STENCIL, oracle.apply_stencil(u, h))):
        yd = shifted(np.full(shape, np.nan))
        st.stencil_apply(ud, yd, h, form)
        torch.cuda.synchronize()
        assert apply_err(to_host(yd), ref, u, h) <= TOL_F64, form
    od = shifted(np.full(shape, np.nan))
    st.stencil_jacobi_step(ud, fd, od, h, 2.0 / 3.0)
    rd = shifted(np.full(shape, np.nan))
    st.stencil_residual(ud, fd, h, r=rd)
    torch.cuda.synchronize()
    assert rel_err(to_host(od), oracle.jacobi(u, f, h, 2.0 / 3.0, 1)) <= TOL_F64
    assert apply_err(to_host(rd), oracle.residual(u, f, h)[0], u, h) <= TOL_F64
    for sweeps in (2, 5):
        gd, fd = shifted(u), shifted(f)
        st.stencil_smooth_coloured(gd, fd, h, sweeps)
        jd = shifted(u)
        st.stencil_smooth_jacobi(jd, fd, shifted(np.zeros(shape)), h, sweeps, 2.0 / 3.0)
        torch.cuda.synchronize()
        assert rel_err(to_host(gd), oracle.gs_coloured(u, f, h, sweeps)) <= TOL_F64, sweeps
        assert rel_err(to_host(jd), oracle.jacobi(u, f, h, 2.0 / 3.0, sweeps)) <= TOL_F64, sweeps


@pytest.mark.parametrize("n", [(70, 40, 9), (33, 9, 7)])
def test_3d_ops_misaligned_f_and_out(n):
    """3D apply, Jacobi step and residual with u 16-byte aligned (even pitch: the staged
    TMA path) but f and the outputs 8 bytes off: pair accesses must fall back."""
    h = 1.0 / max(n)
    shape = synth.grid_shape(3, n)
    u = synth.uniform_field(shape, 1900 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 1901 + sum(n))
    pitch = shape[2] + 1 + (shape[2] + 1) % 2  # even, room for a one-element offset

    def view(a, off):
        buf = torch.full(shape[:2] + (pitch,), float("nan"), dtype=torch.float64, device="cuda")
        v = buf[:, :, off:off + shape[2]]
        v.copy_(torch.from_numpy(a).cuda())
        return v

    ud = view(u, 0)
    fd = view(f, 1)
    assert ud.data_ptr() % 16 == 0 and fd.data_ptr() % 16 == 8
    yd = view(np.full(shape, np.nan), 1)
    st.stencil_apply(ud, yd, h, st.FORM_STENCIL)
    od = view(np.full(shape, np.nan), 1)
    st.stencil_jacobi_step(ud, fd, od, h, 2.0 / 3.0)
    rd = view(np.full(shape, np.nan), 1)
    nrm = st.stencil_residual(ud, fd, h, r=rd)
    torch.cuda.synchronize()
    assert apply_err(to_host(yd), oracle.apply_stencil(u, h), u, h) <= TOL_F64
    assert rel_err(to_host(od), oracle.jacobi(u, f, h, 2.0 / 3.0, 1)) <= TOL_F64
    rref, nref = oracle.residual(u, f, h)
    assert apply_err(to_host(rd), rref, u, h) <= TOL_F64
    got = nrm.cpu().numpy()
    assert abs(got[1] - nref[1]) <= 1e-12 * nref[1]
    assert abs(got[0] - nref[0]) <= 1e-11 * nref[0]


@pytest.mark.parametrize("pad", [0, 1])
@pytest.mark.parametrize("sweeps", [2, 5])
def test_gs_3d_many_tiles_and_chunks(pad, sweeps):
    """Multi-sweep 3D GS over several (x, y) tiles with ragged tails and several plane
    chunks (odd and even pitch: the single-pass and the two-launch kernels), nonzero
    Dirichlet data."""
    n = (130, 61, 45)
    h = 1.0 / 130
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 2100 + sweeps, zero_bc=False)
    f = synth.uniform_field(shape, 2101)
    ref = oracle.gs_coloured(u0, f, h, sweeps)
    ud, fd = to_dev(u0, pad), to_dev(f, pad)
    st.stencil_smooth_coloured(ud, fd, h, sweeps)
    torch.cuda.synchronize()
    got = to_host(ud)
    assert rel_err(got, ref) <= TOL_F64
    b = ~_interior(shape)
    assert np.array_equal(got[b], u0[b])
