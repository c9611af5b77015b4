"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped stencil term, a
wrong sign, a transposed index, a wrong colour order or scaling) makes one of them
fail.  No GPU is needed.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests import dense_reference as dr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b, denom=None):
    d = np.max(np.abs(b)) if denom is None else denom
    return float(np.max(np.abs(a - b)) / d)


# ----------------------------------------------------------- paper's printed stencil

def _paper_9pt():
    rows = []
    with open(os.path.join(GOLDEN, "fig1_9point_fe_stencil.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([Fraction(t) for t in line.split()])
    return rows  # rows[0] is dy=+1


def test_2d_element_assembly_reproduces_paper_9point_stencil():
    """Fig. 1: assembling the 2D bilinear element matrix onto one vertex gives the
    printed 9-point stencil (centre 8/3, all neighbours -1/3)."""
    K = oracle.element_matrix(2, 1.0)  # h-free in 2D
    S = np.zeros((3, 3))  # S[dy+1, dx+1]
    # the vertex at the origin is local vertex v of the cell whose lower-left corner
    # is at -(v's offset); every local pair (v, w) contributes K[v, w] at w - v.
    for v in range(4):
        vx, vy = v & 1, v >> 1
        for w in range(4):
            wx, wy = w & 1, w >> 1
            S[wy - vy + 1, wx - vx + 1] += K[v, w]
    paper = _paper_9pt()
    for r, dy in enumerate((1, 0, -1)):
        for c, dx in enumerate((-1, 0, 1)):
            assert S[dy + 1, dx + 1] == pytest.approx(float(paper[r][c]), abs=1e-15)
            assert oracle.stencil_weight(2, dx, dy) == pytest.approx(float(paper[r][c]), abs=1e-15)


def test_2d_apply_on_delta_reproduces_paper_stencil():
    n, h = 6, 1.0 / 6
    u = np.zeros((n + 1, n + 1))
    u[3, 3] = 1.0
    paper = _paper_9pt()
    for y in (oracle.apply_stencil(u, h), oracle.apply_elementwise(u, h)):
        for r, dy in enumerate((1, 0, -1)):
            for c, dx in enumerate((-1, 0, 1)):
                # y_i = sum_j A_ij u_j with u = delta at the centre gives A_{i,centre},
                # the mirrored stencil; the 9-point stencil is symmetric.
                assert y[3 - dy, 3 - dx] * h * h == pytest.approx(float(paper[r][c]), rel=1e-13)


def test_3d_element_matrix_structure():
    K = oracle.element_matrix(3, 1.0)
    assert np.allclose(K, K.T, atol=0)
    assert np.allclose(K.sum(axis=1), 0.0, atol=1e-15)
    for v in range(8):
        for w in range(8):
            m = bin(v ^ w).count("1")
            expect = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[m]
            assert K[v, w] == pytest.approx(expect, abs=1e-15)
    # assembled weights: shared by 2^(3-m) cells
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                m = abs(dx) + abs(dy) + abs(dz)
                expect = {0: 8 / 3, 1: 0.0, 2: -1 / 6, 3: -1 / 12}[m]
                assert oracle.stencil_weight(3, dx, dy, dz) == pytest.approx(expect, abs=1e-15)


# ------------------------------------------------------- brute-force global assembly

@pytest.mark.parametrize("dim,n", [(2, (4, 4)), (2, (3, 5)), (3, (3, 3, 3)), (3, (2, 3, 4)),
                                   (3, (4, 4, 4))])
def test_applies_equal_kronecker_assembly(dim, n):
    h = 0.25
    shape = synth.grid_shape(dim, n)
    u = synth.uniform_field(shape, 11, zero_bc=False)  # nonzero Dirichlet data too
    y_ref = dr.dense_apply(u, h)
    denom = (16.0 / 3.0) / h ** 2 * np.max(np.abs(u))
    assert _rel(oracle.apply_elementwise(u, h), y_ref, denom) < 1e-14
    assert _rel(oracle.apply_stencil(u, h), y_ref, denom) < 1e-14


def test_apply_forms_agree_and_threads_do_not_change_bits():
    n, h = 12, 1.0 / 12
    u = synth.uniform_field(synth.grid_shape(3, n), 5, zero_bc=False)
    y1 = oracle.apply_elementwise(u, h, nthreads=1)
    y4 = oracle.apply_elementwise(u, h, nthreads=4)
    assert np.array_equal(y1, y4)
    ys = oracle.apply_stencil(u, h, nthreads=3)
    assert _rel(y1, ys, (16 / 3) / h ** 2) < 1e-14


# ------------------------------------------------------- closed forms (polynomials)

@pytest.mark.parametrize("form", ["elementwise", "stencil"])
def test_polynomials_up_to_cubic_exact_3d(form):
    """A = S/h^2 reproduces -Laplace exactly on every polynomial of total degree <= 3
    (1D mass averages are exact on linears, second differences on cubics)."""
    n = 8
    h = 1.0 / n
    x = np.arange(n + 1) * h
    X = x[None, None, :]
    Y = x[None, :, None]
    Z = x[:, None, None]
    ones = np.ones((n + 1,) * 3)
    app = oracle.apply_elementwise if form == "elementwise" else oracle.apply_stencil
    # (u, -Laplace u): A u must reproduce the second entry at interior vertices
    cases = [
        (ones * 1.0, 0.0 * ones),
        (X * ones, 0.0 * ones),
        (X * Y * Z * ones, 0.0 * ones),
        ((X ** 2 + Y ** 2 + Z ** 2) * ones, -6.0 * ones),
        ((X ** 3) * ones, -6.0 * X * ones),
        ((X ** 2 * Y) * ones, -2.0 * Y * ones),
        ((Y ** 2 * Z - Z ** 3) * ones, (-2.0 * Z + 6.0 * Z) * ones),
    ]
    inner = dr.interior_mask(ones.shape)
    for u, expect in cases:
        y = app(np.ascontiguousarray(u), h)
        # rounding of O(1/h^2) terms: bound by a few ulps of |A| |u|
        tol = 64 * np.finfo(float).eps * (16 / 3) / h ** 2 * max(1.0, np.max(np.abs(u)))
        assert np.max(np.abs(y[inner] - expect[inner])) < tol
        assert np.all(y[~inner] == 0.0)


def test_polynomials_2d():
    n = 10
    h = 1.0 / n
    x = np.arange(n + 1) * h
    X = x[None, :]
    Y = x[:, None]
    ones = np.ones((n + 1, n + 1))
    inner = dr.interior_mask(ones.shape)
    # (u, -Laplace u)
    for u, expect in [((X ** 2 + Y ** 2) * ones, -4.0), ((X * Y) * ones, 0.0)]:
        for app in (oracle.apply_elementwise, oracle.apply_stencil):
            y = app(np.ascontiguousarray(u), h)
            tol = 64 * np.finfo(float).eps * (16 / 3) / h ** 2
            assert np.max(np.abs(y[inner] - expect)) < tol
    u = np.ascontiguousarray((X ** 3 - 3 * X * Y ** 2) * ones)  # harmonic cubic
    y = oracle.apply_stencil(u, h)
    assert np.max(np.abs(y[inner])) < 64 * np.finfo(float).eps * (16 / 3) / h ** 2


@pytest.mark.parametrize("dim,modes", [(3, (1, 1, 1)), (3, (2, 3, 1)), (3, (5, 1, 2)),
                                       (2, (1, 1)), (2, (3, 2))])
def test_sine_modes_are_eigenvectors_with_closed_form_symbol(dim, modes):
    n = 16
    h = 1.0 / n
    u = dr.sine_mode(dim, n, modes)
    lam = dr.symbol(dim, [m * math.pi * h for m in modes])
    inner = dr.interior_mask(u.shape)
    for app in (oracle.apply_elementwise, oracle.apply_stencil):
        y = app(np.ascontiguousarray(u), h)
        assert np.max(np.abs(y[inner] - lam / h ** 2 * u[inner])) < 1e-12 * (16 / 3) / h ** 2


def test_symbol_spot_values():
    assert dr.symbol(3, [0, 0, 0]) == 0.0
    assert dr.symbol(3, [math.pi, 0, 0]) == pytest.approx(4.0)
    assert dr.symbol(2, [math.pi, math.pi]) == pytest.approx(2 * 4 * (1 / 3))


def test_symmetry():
    n, h = 7, 1.0 / 7
    shape = synth.grid_shape(3, n)
    u = synth.uniform_field(shape, 1)
    v = synth.uniform_field(shape, 2)
    for app in (oracle.apply_elementwise, oracle.apply_stencil):
        a = float(np.sum(app(u, h) * v))
        b = float(np.sum(u * app(v, h)))
        assert a == pytest.approx(b, rel=1e-13)


# ------------------------------------------------------------------ Gauss-Seidel

@pytest.mark.parametrize("dim,n", [(2, (2, 2)), (2, (5, 4)), (2, (6, 6)), (3, (2, 2, 2)),
                                   (3, (3, 4, 5)), (3, (5, 5, 5)), (3, (6, 3, 4))])
def test_coloured_gs_equals_dense_bruteforce(dim, n):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 21, zero_bc=False)
    f = synth.uniform_field(shape, 22)
    ref = dr.dense_gs(u0, f, h, sweeps=3)
    got = oracle.gs_coloured(u0, f, h, sweeps=3)
    assert _rel(got, ref) < 1e-13
    # boundary never written
    bmask = ~dr.interior_mask(shape)
    assert np.array_equal(got[bmask], u0[bmask])


def test_gs_colour_order_matters_and_inside_colour_order_does_not():
    n, h = 5, 0.2
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 31)
    f = synth.uniform_field(shape, 32)
    a = dr.dense_gs(u0, f, h, 2)
    b = dr.dense_gs(u0, f, h, 2, order_seed=7)
    assert np.array_equal(a, b)  # updates inside a colour are independent
    # same-colour vertices are never coupled
    A = dr.global_matrix(3, (n, n, n), h)
    col = dr.colour_array(shape).ravel()
    same = col[:, None] == col[None, :]
    np.fill_diagonal(same, False)
    assert np.all(A[same] == 0.0)


def test_gs_threads_do_not_change_bits():
    n, h = 10, 0.1
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 41)
    f = synth.uniform_field(shape, 42)
    assert np.array_equal(oracle.gs_coloured(u0, f, h, 3, nthreads=1),
                          oracle.gs_coloured(u0, f, h, 3, nthreads=4))


def test_gs_converges_to_closed_form_discrete_solution():
    """f = 3 pi^2 sin sin sin is an eigenvector, so the discrete solution is
    u_h = h^2 f / lambda_S(pi h, pi h, pi h); GS from 0 converges to it with the
    residual decreasing every sweep."""
    n = 8
    h = 1.0 / n
    f = synth.sin_rhs(3, n)
    lam = dr.symbol(3, [math.pi * h] * 3)
    uh = h * h * f / lam
    u = np.zeros_like(f)
    prev = np.inf
    for _ in range(80):
        u = oracle.gs_coloured(u, f, h, 1)
        _, nrm = oracle.residual(u, f, h)
        assert nrm[0] < prev
        prev = nrm[0]
    assert _rel(u, uh) < 1e-12


def test_gs_energy_norm_of_error_decreases():
    n = 6
    h = 1.0 / n
    shape = synth.grid_shape(3, n)
    f = synth.uniform_field(shape, 51)
    A = dr.global_matrix(3, (n, n, n), h)
    inner = dr.interior_mask(shape).ravel()
    AII = A[np.ix_(inner, inner)]
    xs = np.linalg.solve(AII, f.ravel()[inner])
    u = synth.uniform_field(shape, 52)
    prev = np.inf
    for _ in range(10):
        u = oracle.gs_coloured(u, f, h, 1)
        e = u.ravel()[inner] - xs
        en = float(e @ AII @ e)
        assert en < prev
        prev = en


def test_fp32_and_bf16_sweeps_track_fp64():
    n = 8
    h = 1.0 / n
    shape = synth.grid_shape(3, n)
    u0 = synth.uniform_field(shape, 61)
    f = synth.uniform_field(shape, 62)
    r64 = oracle.gs_coloured(u0, f, h, 4)
    r32 = oracle.gs_coloured_f32(u0.astype(np.float32), f.astype(np.float32), h, 4)
    assert _rel(r32.astype(np.float64), r64) < 1e-5
    import torch
    ub = torch.from_numpy(u0.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    fb = torch.from_numpy(f.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    rb = oracle.gs_coloured_bf16(ub, fb, h, 4)
    rbf = torch.from_numpy(rb.view(np.int16)).view(torch.bfloat16).to(torch.float32).numpy()
    assert _rel(rbf.astype(np.float64), r64) < 3e-2


def test_bf16_rounding_matches_torch():
    import torch
    g = synth.rng(5)
    # random values, ties to even both ways and signs, zeros, overflow to infinity (the
    # largest finite FP32 values), infinities, subnormals down to the smallest, and the
    # just-below-a-tie / just-above-a-tie neighbours of a tie
    edges = [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, -1.0 - 3 * 2 ** -8, 0.0, -0.0, 3.0e38, 1e-40,
             np.finfo(np.float32).max, -np.finfo(np.float32).max, np.inf, -np.inf, 1.4e-45, -1.4e-45,
             np.finfo(np.float32).tiny, 2 ** -126 * (1 + 2 ** -8), 3.3961776e38, 3.3895314e38,
             1.0 + 2 ** -8 + 2 ** -20, 1.0 + 2 ** -8 - 2 ** -20]
    xs = np.concatenate([g.standard_normal(2000).astype(np.float32) * 1e3, np.array(edges, dtype=np.float32)])
    tb = torch.from_numpy(xs).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    for x, t in zip(xs, tb):
        assert oracle.f32_to_bf16(x) == int(t)
        back = torch.from_numpy(np.array([t], dtype=np.uint16).view(np.int16)).view(torch.bfloat16)
        assert oracle.bf16_to_f32(int(t)) == float(back.float().item())


# ------------------------------------------------------------ Jacobi and residual

def test_jacobi_damps_eigenmode_by_closed_form_factor():
    n = 12
    h = 1.0 / n
    for modes in [(1, 1, 1), (3, 2, 5), (11, 11, 11)]:
        u0 = dr.sine_mode(3, n, modes)
        lam = dr.symbol(3, [m * math.pi * h for m in modes])
        omega = 2.0 / 3.0
        fac = 1.0 - omega * (3.0 / 8.0) * lam
        u1 = oracle.jacobi(u0, np.zeros_like(u0), h, omega, 1)
        assert np.max(np.abs(u1 - fac * u0)) < 1e-14
        u3 = oracle.jacobi(u0, np.zeros_like(u0), h, omega, 3)
        assert np.max(np.abs(u3 - fac ** 3 * u0)) < 1e-13


@pytest.mark.parametrize("dim,n", [(2, (5, 6)), (3, (4, 5, 3))])
def test_jacobi_equals_dense_and_is_order_free(dim, n):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 71, zero_bc=False)
    f = synth.uniform_field(shape, 72)
    ref = dr.dense_jacobi(u0, f, h, 2 / 3, 2)
    got1 = oracle.jacobi(u0, f, h, 2 / 3, 2, nthreads=1)
    got3 = oracle.jacobi(u0, f, h, 2 / 3, 2, nthreads=3)
    assert np.array_equal(got1, got3)
    assert _rel(got1, ref) < 1e-13


def test_residual_equals_dense_and_vanishes_at_discrete_solution():
    n = 6
    h = 1.0 / n
    shape = synth.grid_shape(3, n)
    u = synth.uniform_field(shape, 81)
    f = synth.uniform_field(shape, 82)
    r, nrm = oracle.residual(u, f, h)
    rref = f - dr.dense_apply(u, h)
    rref[~dr.interior_mask(shape)] = 0.0
    assert _rel(r, rref) < 1e-13
    inner = dr.interior_mask(shape)
    assert nrm[0] == pytest.approx(float(np.sum(rref[inner] ** 2)), rel=1e-13)
    assert nrm[1] == pytest.approx(float(np.sum(f[inner] ** 2)), rel=1e-13)
    fs = synth.sin_rhs(3, n)
    uh = h * h * fs / dr.symbol(3, [math.pi * h] * 3)
    r2, nrm2 = oracle.residual(uh, fs, h)
    assert math.sqrt(nrm2[0] / nrm2[1]) < 1e-14


def _exact_weight(dim, m):
    """Assembled Q1 stencil weight as an exact rational (m = coordinates that differ)."""
    if m == 0:
        return Fraction(8, 3)
    if dim == 2:
        return Fraction(-1, 3)
    return [None, Fraction(0), Fraction(-1, 6), Fraction(-1, 12)][m]


@pytest.mark.parametrize("dim,n", [(2, 7), (3, 5)])
def test_residual_norms_against_exact_rational_arithmetic(dim, n):
    """The norms of r = f - S u / h^2 over the interior, evaluated exactly in rational
    arithmetic on the FP64 inputs.  The long double oracle must agree to far below
    FP64 rounding; the FP64 oracle within a forward error bound: each r_i carries at
    most (K + 8) eps (|f_i| + sum |w||u| / h^2) (K stencil products, the rounded
    weights, h^2 and the division), and the sum of N squares a further (N + 2) eps."""
    h = 1.0 / n
    shape = synth.grid_shape(dim, n)
    u = synth.uniform_field(shape, 91 + dim)
    f = synth.uniform_field(shape, 93 + dim)
    hq = Fraction(h)
    offs = [(dz, dy, dx) for dz in ((-1, 0, 1) if dim == 3 else (0,)) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    u3 = u.reshape((1,) + u.shape) if dim == 2 else u
    f3 = f.reshape((1,) + f.shape) if dim == 2 else f
    ks = range(1, n) if dim == 3 else range(0, 1)
    rr = ff = Fraction(0)
    bound_terms = []
    for k in ks:
        for j in range(1, n):
            for i in range(1, n):
                s = Fraction(0)
                mag = 0.0
                for dz, dy, dx in offs:
                    w = _exact_weight(dim, abs(dx) + abs(dy) + abs(dz))
                    uv = float(u3[k + dz, j + dy, i + dx])
                    s += w * Fraction(uv)
                    mag += abs(float(w)) * abs(uv)
                fi = Fraction(float(f3[k, j, i]))
                r = fi - s / (hq * hq)
                rr += r * r
                ff += fi * fi
                bound_terms.append((abs(float(r)), abs(float(fi)) + mag / (h * h)))
    eps = np.finfo(np.float64).eps
    K, N = len(offs), len(bound_terms)
    err_rr = sum(2 * ar * (K + 8) * eps * m + ((K + 8) * eps * m) ** 2 for ar, m in bound_terms)
    err_rr += (N + 2) * eps * float(rr) * 1.01

    ld = oracle.residual_norms_ld(u, f, h)
    assert abs(ld[0] - float(rr)) <= 1e-15 * float(rr)
    assert abs(ld[1] - float(ff)) <= 1e-15 * float(ff)
    _, nrm = oracle.residual(u, f, h)
    assert abs(nrm[0] - float(rr)) <= err_rr
    assert abs(nrm[1] - float(ff)) <= (N + 2) * eps * float(ff)
    assert err_rr < 1e-11 * float(rr)  # the bound is not vacuous
    # a dropped term is far outside the bound: the residual without the last neighbour
    rr_bad = Fraction(0)
    for k in ks:
        for j in range(1, n):
            for i in range(1, n):
                s = sum(_exact_weight(dim, abs(dx) + abs(dy) + abs(dz)) * Fraction(float(u3[k + dz, j + dy, i + dx]))
                        for dz, dy, dx in offs[:-1])
                r = Fraction(float(f3[k, j, i])) - s / (hq * hq)
                rr_bad += r * r
    assert abs(float(rr_bad) - float(rr)) > 1e3 * err_rr


# ------------------------------------------------------------ iterative refinement

@pytest.mark.parametrize("prec", [0, 1, 2])
def test_ir_converges_to_closed_form(prec):
    n = 8
    h = 1.0 / n
    modes = (2, 3, 1)
    f = synth.sin_rhs(3, n, modes)
    lam = dr.symbol(3, [m * math.pi * h for m in modes])
    uh = h * h * f / lam
    x, hist, k, conv = oracle.ir_solve(np.zeros_like(f), f, h, 1e-10, 400, 8, prec)
    assert conv
    assert hist[-1] <= 1e-10
    assert _rel(x, uh) < 1e-8
    if prec == 0:
        # FP64 inner sweeps from e = 0 reproduce plain GS on x (Gauss-Seidel is a
        # stationary iteration), up to rounding.
        xg = oracle.gs_coloured(np.zeros_like(f), f, h, 8 * k)
        assert _rel(x, xg) < 1e-10


# ------------------------------------------------------------------ patch lattices

def test_single_patch_with_outer_boundary_is_plain_dirichlet_gs():
    lat = synth.PatchLattice(lat=(1, 1, 1), seed=2, u_random=True)
    u = lat.u.copy()
    p0 = lat.view(u, 0).copy()
    synth.zero_boundary(p0)
    out = oracle.patch_smooth(lat.lat, lat.np_sizes, lat.offsets, lat.u, lat.f, 3)
    n = int(lat.np_sizes[0])
    ref = oracle.gs_coloured(p0, lat.view(lat.f, 0), 1.0 / n, 3)
    assert np.array_equal(lat.view(out, 0), ref)


def test_equal_size_neighbours_copy_first_interior_layer():
    lat = synth.PatchLattice(lat=(2, 2, 1), seed=9, edges=(6,), u_random=True)
    u = oracle.patch_halo_fill(lat.lat, lat.np_sizes, lat.offsets, lat.u)
    a = lat.view(u, 0)  # at (0,0,0)
    b = lat.view(lat.u, 1)  # at (1,0,0): +x neighbour
    c = lat.view(lat.u, 2)  # at (0,1,0): +y neighbour
    d = lat.view(lat.u, 3)  # at (1,1,0): +x+y diagonal neighbour
    n = 6
    # +x face (i = n), away from edges: value of b at i=1, same (j,k)
    for k in range(1, n):
        for j in range(1, n):
            assert a[k, j, n] == b[k, j, 1]
            assert a[k, n, j] == c[k, 1, j]
        assert a[k, n, n] == d[k, 1, 1]
    # -x face and the z faces are on the outer boundary: 0
    assert np.all(a[:, :, 0] == 0.0)
    assert np.all(a[0, :, :] == 0.0) and np.all(a[n, :, :] == 0.0)
    # interior untouched
    assert np.array_equal(a[1:n, 1:n, 1:n], lat.view(lat.u, 0)[1:n, 1:n, 1:n])


def test_uneven_neighbour_nearest_index_ties_to_lower():
    # patch 0 with 8 cells next to patch 1 with 12 cells along +x
    lat = synth.PatchLattice(lat=(2, 1, 1), seed=1, edges=(8,))
    lat.np_sizes[:] = [8, 12]
    sizes = (lat.np_sizes.astype(np.int64) + 1) ** 3
    lat.offsets = np.array([0, sizes[0]], dtype=np.int64)
    total = int(sizes.sum())
    u = np.arange(total, dtype=np.float64) + 0.5  # every value distinct
    out = oracle.patch_halo_fill(lat.lat, lat.np_sizes, lat.offsets, u)
    a = out[:9 ** 3].reshape(9, 9, 9)
    b = u[9 ** 3:].reshape(13, 13, 13)
    # j = 1 -> 12/8 = 1.5 -> tie -> 1 ; j = 3 -> 4.5 -> 4 ; j = 5 -> 7.5 -> 7 ; j = 4 -> 6
    for j, jq in [(1, 1), (3, 4), (4, 6), (5, 7), (7, 10)]:
        assert a[4, j, 8] == b[6, jq, 1]  # k = 4 -> 6 exactly
    # tangential indices clamp into [1, n_q - 1]
    assert a[4, 0, 8] == 0.0  # j = 0 is on the -y outer boundary -> 0


def _collapsed_global(lat, L, n):
    """Dense solution of the global system on the collapsed grid of equal patches, and
    the map from patch interiors into it."""
    h = 1.0 / n
    N = tuple(L[a] * (n - 1) + 1 for a in range(3))  # cells per axis
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    F = np.zeros(shape)

    def block(p):
        px, py, pz = p % L[0], (p // L[0]) % L[1], p // (L[0] * L[1])
        return (slice(pz * (n - 1) + 1, pz * (n - 1) + n), slice(py * (n - 1) + 1, py * (n - 1) + n),
                slice(px * (n - 1) + 1, px * (n - 1) + n))

    npatch = L[0] * L[1] * L[2]
    for p in range(npatch):
        F[block(p)] = lat.view(lat.f, p)[1:n, 1:n, 1:n]
    A = dr.global_matrix(3, N, h)
    inner = dr.interior_mask(shape).ravel()
    U = np.zeros(F.size)
    U[inner] = np.linalg.solve(A[np.ix_(inner, inner)], F.ravel()[inner])
    return U.reshape(shape), block, npatch


@pytest.mark.parametrize("L,n", [((2, 2, 2), 4), ((3, 2, 1), 5)])
def test_equal_patches_converge_to_the_collapsed_global_solution(L, n):
    """Equal patches of n cells.  Vertex n of a patch and vertex 0 of its +x neighbour sit
    at the same point, yet both are halo: each is filled from the other patch's first
    interior layer.  So the interior vertices of all patches form one grid of L(n-1)
    unknowns per axis, and across an interface (face, edge or corner) a stencil's
    neighbour is the adjacent unknown of that grid, with h = 1/n in every stencil.  The
    patch iteration (halo fill, then a coloured GS sweep per patch) is a block splitting
    of that global system, so it must converge to the system's solution, computed here
    by a dense solve of the Kronecker-assembled matrix."""
    lat = synth.PatchLattice(lat=L, seed=5, edges=(n,))
    U, block, npatch = _collapsed_global(lat, L, n)
    out = oracle.patch_smooth(lat.lat, lat.np_sizes, lat.offsets, lat.u, lat.f, 300)
    scale = np.max(np.abs(U))
    err = max(np.max(np.abs(lat.view(out, p)[1:n, 1:n, 1:n] - U[block(p)])) for p in range(npatch))
    assert err <= 1e-12 * scale
    # the other reading, with the interface vertex an unknown shared by both patches
    # (a global grid of L n cells), is a different system and is far from the result
    N2 = tuple(L[a] * n for a in range(3))
    shape2 = (N2[2] + 1, N2[1] + 1, N2[0] + 1)
    F2 = np.zeros(shape2)
    for p in range(npatch):
        px, py, pz = p % L[0], (p // L[0]) % L[1], p // (L[0] * L[1])
        F2[pz * n + 1:pz * n + n, py * n + 1:py * n + n, px * n + 1:px * n + n] = lat.view(lat.f, p)[1:n, 1:n, 1:n]
    A2 = dr.global_matrix(3, N2, 1.0 / n)
    in2 = dr.interior_mask(shape2).ravel()
    U2 = np.zeros(F2.size)
    U2[in2] = np.linalg.solve(A2[np.ix_(in2, in2)], F2.ravel()[in2])
    U2 = U2.reshape(shape2)
    err2 = 0.0
    for p in range(npatch):
        px, py, pz = p % L[0], (p // L[0]) % L[1], p // (L[0] * L[1])
        g = U2[pz * n + 1:pz * n + n, py * n + 1:py * n + n, px * n + 1:px * n + n]
        err2 = max(err2, np.max(np.abs(lat.view(out, p)[1:n, 1:n, 1:n] - g)))
    assert err2 > 1e-3 * scale


def test_uneven_halo_is_the_nearest_vertex_by_exact_geometry():
    """The halo rule restated geometrically and evaluated by brute force in exact
    rational arithmetic, against the oracle's integer index formula, on every shell
    vertex of a 3 x 2 x 2 lattice of uneven patches (2 to 7 cells).  Shell vertex i
    (per axis) of patch p at lattice cell P sits at P + i / n_p; its outward direction d
    picks the neighbour cell Q = P + d (0 outside the lattice); per axis the source is
    the vertex t of Q, among all t = 0 .. n_q, whose position Q + t / n_q is nearest
    (the lower t on a tie), moved into Q's interior 1 .. n_q - 1."""
    from fractions import Fraction as Fr
    lat = synth.PatchLattice(lat=(3, 2, 2), seed=4, edges=(2, 3, 4, 5, 6, 7))
    sizes = (lat.np_sizes.astype(np.int64) + 1) ** 3
    u = np.arange(int(sizes.sum()), dtype=np.float64) + 0.25  # every value distinct
    out = oracle.patch_halo_fill(lat.lat, lat.np_sizes, lat.offsets, u)
    L = [int(v) for v in lat.lat]
    npatch = L[0] * L[1] * L[2]
    assert len(set(int(v) for v in lat.np_sizes)) >= 4  # genuinely uneven
    for p in range(npatch):
        P = (p % L[0], (p // L[0]) % L[1], p // (L[0] * L[1]))
        n = int(lat.np_sizes[p])
        got = lat.view(out, p)
        for k in range(n + 1):
            for j in range(n + 1):
                for i in range(n + 1):
                    idx = (i, j, k)
                    d = tuple(-1 if v == 0 else (1 if v == n else 0) for v in idx)
                    if d == (0, 0, 0):
                        continue
                    Q = tuple(P[a] + d[a] for a in range(3))
                    if any(Q[a] < 0 or Q[a] >= L[a] for a in range(3)):
                        assert got[k, j, i] == 0.0
                        continue
                    q = Q[0] + L[0] * (Q[1] + L[1] * Q[2])
                    m = int(lat.np_sizes[q])
                    src = []
                    for a in range(3):
                        x = P[a] + Fr(idx[a], n)
                        t = min(range(m + 1), key=lambda s: (abs(Q[a] + Fr(s, m) - x), s))
                        src.append(min(max(t, 1), m - 1))
                    assert got[k, j, i] == lat.view(u, q)[src[2], src[1], src[0]], (p, idx)
