"""Pins for the oracle's 5/7-point finite-difference functions (Fig. 1 middle; red-black
colouring of Section 3, pass order of Algorithm 1).  The dense matrix here is built
from 1D second differences by Kronecker sums, independently of the oracle."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import dense_reference as dr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_5pt():
    rows = []
    with open(os.path.join(GOLDEN, "fig1_5point_fd_stencil.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)  # rows dy = +1, 0, -1; columns dx = -1, 0, +1


def test_2d_weights_match_the_printed_stencil():
    paper = _paper_5pt()
    for r, dy in enumerate((1, 0, -1)):
        for c, dx in enumerate((-1, 0, 1)):
            assert oracle.fd_weight(2, dx, dy, 0) == paper[r, c]


def test_3d_weights_are_the_7_point_stencil():
    tot = 0.0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                w = oracle.fd_weight(3, dx, dy, dz)
                off = abs(dx) + abs(dy) + abs(dz)
                assert w == (6.0 if off == 0 else (-1.0 if off == 1 else 0.0))
                tot += w
    assert tot == 0.0


def _dense_fd(dim, n, h):
    """(sum over axes of kron(I, .., T, .., I)) / h^2, T = tridiag(-1, 2, -1), all vertices."""
    mats = []
    for a in range(dim):
        m = n[a] + 1
        T = 2.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
        mats.append(T)
    A = 0.0
    for axis in range(dim):
        term = None
        for b in reversed(range(dim)):
            f = mats[b] if b == axis else np.eye(n[b] + 1)
            term = f if term is None else np.kron(term, f)
        A = A + term
    return A / (h * h)


CASES = [(2, (5, 4)), (2, (6, 6)), (3, (3, 4, 5)), (3, (4, 4, 4))]


@pytest.mark.parametrize("dim,n", CASES)
def test_apply_equals_dense_kronecker(dim, n):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u = synth.uniform_field(shape, 3 + sum(n), zero_bc=False)
    y = oracle.fd_apply(u, h)
    yd = (_dense_fd(dim, n, h) @ u.ravel()).reshape(shape)
    inner = dr.interior_mask(shape)
    assert np.max(np.abs(y[inner] - yd[inner])) <= 1e-12 * np.max(np.abs(yd))
    assert np.all(y[~inner] == 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_exact_on_cubic_polynomials(dim):
    """Second differences are exact on cubics: A(x^2 + y^2 [+ z^2]) = -2d and
    A(x^3) = -6x at interior vertices when the boundary holds the same function."""
    n = 8
    h = 1.0 / n
    cs = synth.coords(dim, n)
    shape = synth.grid_shape(dim, n)
    inner = dr.interior_mask(shape)
    q = np.zeros(shape)
    for c in cs:
        q = q + c * c
    assert np.max(np.abs(oracle.fd_apply(q, h)[inner] + 2 * dim)) <= 1e-10
    x = np.broadcast_to(cs[0], shape)
    assert np.max(np.abs(oracle.fd_apply(x ** 3, h)[inner] + 6 * x[inner])) <= 1e-10


def _dense_gs_redblack(u0, f, h, sweeps):
    dim = u0.ndim
    shape = u0.shape
    n = tuple(s - 1 for s in reversed(shape))
    A = _dense_fd(dim, n, h)
    inner = dr.interior_mask(shape).ravel()
    idx = np.indices(shape).sum(axis=0).ravel()  # i + j (+ k)
    u = u0.ravel().copy()
    fr = f.ravel()
    for _ in range(sweeps):
        for parity in (1, 0):  # Algorithm 1: the odd set first
            for p in range(u.size):
                if inner[p] and idx[p] % 2 == parity:
                    off = A[p] @ u - A[p, p] * u[p]
                    u[p] = (fr[p] - off) / A[p, p]
    return u.reshape(shape)


@pytest.mark.parametrize("dim,n", CASES)
def test_redblack_gs_equals_dense_sequential(dim, n):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 13 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 14 + sum(n))
    got = oracle.fd_gs_redblack(u0, f, h, 2)
    ref = _dense_gs_redblack(u0, f, h, 2)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_pass_order_matters_and_is_odd_first():
    """One sweep from a field that differs between the orders: the odd pass reads the
    old even values; starting with the even pass would give a different result."""
    dim, n = 2, (6, 6)
    h = 1.0 / 6
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 99, zero_bc=False)
    f = synth.uniform_field(shape, 98)
    got = oracle.fd_gs_redblack(u0, f, h, 1)
    A = _dense_fd(dim, n, h)
    inner = dr.interior_mask(shape).ravel()
    par = np.indices(shape).sum(axis=0).ravel() % 2
    u = u0.ravel().copy()
    for parity in (0, 1):  # even first
        for p in range(u.size):
            if inner[p] and par[p] == parity:
                u[p] = (f.ravel()[p] - (A[p] @ u - A[p, p] * u[p])) / A[p, p]
    assert np.max(np.abs(got.ravel() - u)) > 1e-6


@pytest.mark.parametrize("dim,n", [(2, 24), (3, 10)])
def test_gs_converges_to_closed_form(dim, n):
    """Sine modes are eigenvectors of the FD operator, lambda = sum (2 - 2 cos theta_a),
    so the discrete solution for f = mode is h^2 f / lambda."""
    h = 1.0 / n
    modes = (1, 2, 1)
    f = synth.zero_boundary(np.ascontiguousarray(dr.sine_mode(dim, n, modes)))
    lam = sum(2 - 2 * math.cos(m * math.pi * h) for m in modes[:dim])
    uh = h * h * f / lam
    u = oracle.fd_gs_redblack(np.zeros_like(f), f, h, 3000)
    assert np.max(np.abs(u - uh)) <= 1e-9 * np.max(np.abs(uh))
    r, nrm = oracle.fd_residual(uh, f, h)
    assert math.sqrt(nrm[0] / nrm[1]) <= 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_jacobi_damps_a_mode_exactly(dim):
    """One Jacobi sweep multiplies a sine mode by 1 - omega lambda / (2d) (f = 0)."""
    n = 12
    h = 1.0 / n
    modes = (3, 1, 2)
    m = synth.zero_boundary(np.ascontiguousarray(dr.sine_mode(dim, n, modes)))
    lam = sum(2 - 2 * math.cos(k * math.pi * h) for k in modes[:dim])
    omega = 0.8
    got = oracle.fd_jacobi(m, np.zeros_like(m), h, omega, 1)
    assert np.max(np.abs(got - (1 - omega * lam / (2 * dim)) * m)) <= 1e-13


@pytest.mark.parametrize("dim,n", CASES)
def test_residual_definition(dim, n):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u = synth.uniform_field(shape, 31 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 32 + sum(n))
    r, nrm = oracle.fd_residual(u, f, h)
    yd = (_dense_fd(dim, n, h) @ u.ravel()).reshape(shape)
    inner = dr.interior_mask(shape)
    rd = np.where(inner, f - yd, 0.0)
    assert np.max(np.abs(r - rd)) <= 1e-12 * np.max(np.abs(yd))
    assert abs(nrm[0] - np.sum(rd[inner] ** 2)) <= 1e-10 * nrm[0]
    assert abs(nrm[1] - np.sum(f[inner] ** 2)) <= 1e-12 * nrm[1]


# ------------------------------------------------------------ expensive stencils S(k)

def test_cost_mode_none_is_the_plain_sweep():
    dim, n = 2, (9, 7)
    h = 1.0 / 9
    u0 = synth.uniform_field(synth.grid_shape(dim, n), 51, zero_bc=False)
    f = synth.uniform_field(u0.shape, 52)
    assert np.array_equal(oracle.fd_gs_redblack_cost(u0, f, h, 2, 0, 100), oracle.fd_gs_redblack(u0, f, h, 2))


@pytest.mark.parametrize("dim,n,i,j,k", [(2, (9, 7), 3, 4, 0), (3, (6, 5, 7), 2, 3, 4), (2, (300, 200), 250, 150, 0)])
@pytest.mark.parametrize("kmax", [1, 7, 100])
def test_cost_diagonal_closed_form(dim, n, i, j, k, kmax):
    """sum_{m=1..k} sin(m t) = sin(k t / 2) sin((k + 1) t / 2) / sin(t / 2)."""
    shape = synth.grid_shape(dim, n)
    idx = (((k - 1) * (n[1] - 1) if dim == 3 else 0) + (j - 1)) * (n[0] - 1) + (i - 1)
    t = idx * 2.0 ** -20
    sigma = math.sin(kmax * t / 2) * math.sin((kmax + 1) * t / 2) / math.sin(t / 2)
    want = 2 * dim + 2.0 ** -20 * sigma / kmax
    got = oracle.cost_diagonal(shape, 1, kmax, i, j, k)
    assert abs(got - want) <= 1e-15 * want


def test_cost_linear_pattern():
    """k runs linearly from 0 over the interior: the first 1/kmax of the vertices keep
    the plain diagonal, the last ones use k = kmax - 1."""
    dim, n, kmax = 2, (101, 41), 10
    shape = synth.grid_shape(dim, n)
    N = 100 * 40
    for idx in (0, 1, N // kmax - 1):
        j, i = 1 + idx // 100, 1 + idx % 100
        assert oracle.cost_diagonal(shape, 2, kmax, i, j) == 4.0
    idx = N - 1
    j, i = 1 + idx // 100, 1 + idx % 100
    t = idx * 2.0 ** -20
    kk = kmax * idx // N
    sigma = sum(math.sin(m * t) for m in range(1, kk + 1))
    assert kk == kmax - 1
    assert abs(oracle.cost_diagonal(shape, 2, kmax, i, j) - (4.0 + 2.0 ** -20 * sigma / kk)) <= 1e-15


@pytest.mark.parametrize("dim,n,mode", [(2, (6, 5), 1), (2, (6, 6), 2), (3, (4, 3, 5), 1)])
def test_cost_sweep_equals_dense_gs_with_perturbed_diagonal(dim, n, mode):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 61 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 62 + sum(n))
    kmax = 30
    A = _dense_fd(dim, n, h)
    inner = dr.interior_mask(shape)
    idxs = np.argwhere(inner)
    for ix in idxs:
        kk, jj, ii = (ix if dim == 3 else (0, ix[0], ix[1]))
        p = np.ravel_multi_index(tuple(ix), shape)
        A[p, p] = oracle.cost_diagonal(shape, mode, kmax, ii, jj, kk) / (h * h)
    par = np.indices(shape).sum(axis=0).ravel() % 2
    u = u0.ravel().copy()
    fr = f.ravel()
    innr = inner.ravel()
    for _ in range(2):
        for parity in (1, 0):
            for p in range(u.size):
                if innr[p] and par[p] == parity:
                    u[p] = (fr[p] - (A[p] @ u - A[p, p] * u[p])) / A[p, p]
    got = oracle.fd_gs_redblack_cost(u0, f, h, 2, mode, kmax)
    assert np.max(np.abs(got.ravel() - u)) <= 1e-12 * np.max(np.abs(u))
