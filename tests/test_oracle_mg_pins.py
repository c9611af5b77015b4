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


def _shape(dim, n):
    return synth.grid_shape(dim, n)


def _interior(a):
    return a[(slice(1, -1),) * a.ndim]


@pytest.mark.parametrize("dim,n", SIZES)
def test_galerkin_identity(dim, n):
    """R A_h P e = A_2h e on the coarse interior: the Q1 spaces are nested, so the
    Galerkin product of the fine operator is the coarse operator (FE stiffness
    K_2h = P^T K_h P; with A = K / h^d and R = P^T / 2^d this is R A_h P = A_2h)."""
    nc = tuple(m // 2 for m in n)
    h = 1.0 / max(n)
    ec = synth.uniform_field(_shape(dim, nc), 11 + sum(n))  # zero boundary
    fine = oracle.mg_prolong_add(ec, np.zeros(_shape(dim, n)))
    lhs = oracle.mg_restrict(oracle.apply_stencil(fine, h))
    rhs = oracle.apply_stencil(ec, 2.0 * h)
    assert np.max(np.abs(_interior(lhs) - _interior(rhs))) <= 1e-12 * np.max(np.abs(rhs))


@pytest.mark.parametrize("dim,n", SIZES)
def test_prolongation_reproduces_multilinear(dim, n):
    """d-linear interpolation is exact on functions linear in each coordinate."""
    nc = tuple(m // 2 for m in n)

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


@pytest.mark.parametrize("dim,n", SIZES)
def test_restriction_is_scaled_transpose(dim, n):
    """<R r, e>_coarse * 2^d = <r, P e>_fine for interior-supported r, e."""
    nc = tuple(m // 2 for m in n)
    r = synth.uniform_field(_shape(dim, n), 21 + sum(n))
    e = synth.uniform_field(_shape(dim, nc), 31 + sum(n))
    lhs = float(np.sum(oracle.mg_restrict(r) * e)) * 2 ** dim
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


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 16)])
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


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 16)])
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
    assert oracle.mg_levels(_shape(2, (7, 8))) == 1
    assert oracle.mg_levels(_shape(2, (8, 8)), max_levels=2) == 2
