"""Pins for the oracle's geometric multigrid (the sweeps as multigrid smoothers,
Section 1): each pin is fixed by the mathematics of the Q1 hierarchy, not by the
oracle's own code, so a wrong weight, offset, scale or transposition fails one."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import dense_reference as dr

SIZES = [(3, (4, 4, 4)), (3, (6, 4, 8)), (3, (8, 8, 8)), (2, (4, 4)), (2, (10, 6)), (2, (16, 16))]
# cubic grids with an odd cell count: coarse grid ceil(n/2), vertices not nested
ODD = [(3, (5, 5, 5)), (3, (9, 9, 9)), (2, (7, 7)), (2, (13, 13))]


def _nc(n):
    return tuple((m + 1) // 2 for m in n)


def _shape(dim, n):
    return synth.grid_shape(dim, n)


def _interior(a):
    return a[(slice(1, -1),) * a.ndim]


@pytest.mark.parametrize("dim,n", SIZES)
def test_galerkin_identity(dim, n):
    """R A_h P e = A_2h e on the coarse interior: the Q1 spaces are nested, so the
    Galerkin product of the fine operator is the coarse operator (FE stiffness
    K_2h = P^T K_h P; with A = K / h^d and R = P^T / 2^d this is R A_h P = A_2h)."""
    nc = _nc(n)
    h = 1.0 / max(n)
    ec = synth.uniform_field(_shape(dim, nc), 11 + sum(n))  # zero boundary
    fine = oracle.mg_prolong_add(ec, np.zeros(_shape(dim, n)))
    lhs = oracle.mg_restrict(oracle.apply_stencil(fine, h))
    rhs = oracle.apply_stencil(ec, 2.0 * h)
    assert np.max(np.abs(_interior(lhs) - _interior(rhs))) <= 1e-12 * np.max(np.abs(rhs))


@pytest.mark.parametrize("dim,n", SIZES + ODD)
def test_prolongation_reproduces_multilinear(dim, n):
    """d-linear interpolation is exact on functions linear in each coordinate, whether
    or not the coarse vertices are fine vertices."""
    nc = _nc(n)

    def g(shape, nn):
        if dim == 3:
            z, y, x = np.meshgrid(*[np.arange(s) / nn[a] for a, s in zip((2, 1, 0), shape)],
                                  indexing="ij")
            return 1 + 2 * x - 3 * y + 0.5 * z + x * y - y * z + 2 * x * y * z
        y, x = np.meshgrid(*[np.arange(s) / nn[a] for a, s in zip((1, 0), shape)], indexing="ij")
        return 1 + 2 * x - 3 * y + 1.5 * x * y

    gc = g(_shape(dim, nc), nc)
    gf = g(_shape(dim, n), n)
    got = oracle.mg_prolong_add(gc, np.zeros_like(gf))
    assert np.max(np.abs(_interior(got) - _interior(gf))) <= 1e-14
    assert np.all(got[(0,) * dim] == 0.0)  # the fine boundary is not touched


@pytest.mark.parametrize("dim,n", SIZES + ODD)
def test_restriction_is_scaled_transpose(dim, n):
    """<R r, e>_coarse (n/n_c)^d = <r, P e>_fine for interior-supported r, e."""
    nc = _nc(n)
    r = synth.uniform_field(_shape(dim, n), 21 + sum(n))
    e = synth.uniform_field(_shape(dim, nc), 31 + sum(n))
    lhs = float(np.sum(oracle.mg_restrict(r) * e)) * float(np.prod([a / b for a, b in zip(n, nc)]))
    rhs = float(np.sum(r * oracle.mg_prolong_add(e, np.zeros_like(r))))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(rhs), 1.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_restriction_of_constant(dim):
    """Full-weighting weights sum to one: a constant interior field restricts to the
    same constant at coarse vertices whose stencil stays inside the fine interior."""
    n = (8,) * dim
    r = synth.zero_boundary(np.full(_shape(dim, n), 3.25))
    rc = oracle.mg_restrict(r)
    inner2 = rc[(slice(2, -2),) * dim]
    assert np.all(inner2 == 3.25)
    assert np.all(rc[(0,) * dim] == 0.0)


def _interp_1d(nf, nc):
    """Dense 1D interpolation matrix from its definition: the coarse grid's hat
    function of vertex I evaluated at the fine vertex positions i / nf."""
    x = np.arange(nf + 1) / nf
    X = np.arange(nc + 1) / nc
    return np.maximum(0.0, 1.0 - np.abs(x[:, None] - X[None, :]) * nc)


@pytest.mark.parametrize("dim,n", SIZES + ODD)
def test_transfers_equal_dense_kronecker(dim, n):
    """P = kron of 1D hat-function matrices, R = (n_c/n)^d P^T, assembled densely."""
    nc = _nc(n)
    mats = [_interp_1d(n[a], nc[a]) for a in reversed(range(dim))]  # (z,) y, x order
    P = mats[0]
    for m in mats[1:]:
        P = np.kron(P, m)
    ec = synth.uniform_field(_shape(dim, nc), 41 + sum(n), zero_bc=False)
    rf = synth.uniform_field(_shape(dim, n), 42 + sum(n), zero_bc=False)
    inner_f = np.zeros(_shape(dim, n), dtype=bool)
    inner_f[(slice(1, -1),) * dim] = True
    pe = (P @ ec.ravel()).reshape(_shape(dim, n))
    got = oracle.mg_prolong_add(ec, np.zeros_like(rf))
    assert np.max(np.abs(got - np.where(inner_f, pe, 0.0))) <= 1e-14
    scale = float(np.prod([b / a for a, b in zip(n, nc)]))
    rc = (scale * (P.T @ rf.ravel())).reshape(_shape(dim, nc))
    synth.zero_boundary(rc)
    assert np.max(np.abs(oracle.mg_restrict(rf) - rc)) <= 1e-13


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 16), (2, 33), (3, 15)])
def test_mg_solve_reaches_closed_form(dim, n):
    """Sine modes are eigenvectors of S with eigenvalue lambda_S, so the discrete
    solution of A u = f for f = c * mode is u_h = h^2 f / lambda_S exactly."""
    h = 1.0 / n
    modes = (1, 2, 1)
    f = 7.0 * dr.sine_mode(dim, n, modes)
    f = synth.zero_boundary(np.ascontiguousarray(f))
    lam = dr.symbol(dim, [m * math.pi * h for m in modes])
    uh = h * h * f / lam
    u, rr, k, conv = oracle.mg_solve(np.zeros_like(f), f, h, 1e-12, 40)
    assert conv and k <= 12
    assert np.max(np.abs(u - uh)) <= 1e-10 * np.max(np.abs(uh))


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 16), (2, 63), (3, 17)])
def test_vcycle_contraction(dim, n):
    """V(2,2) with coloured GS: textbook contraction well below 0.1 per cycle on a
    random right-hand side (every frequency present)."""
    h = 1.0 / n
    f = synth.uniform_field(_shape(dim, (n,) * dim), 5)
    _, rr, k, _ = oracle.mg_solve(np.zeros_like(f), f, h, 1e-30, 5)  # stays above rounding
    rates = rr[2:] / rr[1:-1]
    assert np.all(rates < 0.1), rates


def test_levels():
    assert oracle.mg_levels(_shape(3, (32, 32, 32))) == 5  # 32, 16, 8, 4, 2
    assert oracle.mg_levels(_shape(3, (12, 12, 12))) == 3  # 12, 6, 3
    assert oracle.mg_levels(_shape(3, (255, 255, 255))) == 8  # 255, 128, ..., 2
    assert oracle.mg_levels(_shape(2, (7, 8))) == 1  # mixed parity, not square
    assert oracle.mg_levels(_shape(2, (12, 8))) == 3  # 12x8, 6x4, 3x2
    assert oracle.mg_levels(_shape(2, (8, 8)), max_levels=2) == 2
