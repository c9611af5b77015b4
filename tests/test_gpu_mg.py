"""Multigrid on the GPU (stencil_mg_*) against the oracle's V-cycle: the transfer
operators element by element, whole V-cycles, and the solve against the closed form."""
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

SIZES = [(3, (4, 4, 4)), (3, (6, 4, 8)), (3, (16, 12, 10)), (3, (64, 32, 34)), (3, (5, 5, 5)), (3, (33, 33, 33)),
         (2, (4, 4)), (2, (10, 6)), (2, (130, 66)), (2, (512, 200)), (2, (7, 7)), (2, (301, 301))]


@pytest.mark.parametrize("dim,n", SIZES)
@pytest.mark.parametrize("pad", [0, 3])
def test_restrict_matches_oracle(dim, n, pad):
    nc = tuple(m - 1 for m in reversed(oracle.coarse_shape(synth.grid_shape(dim, n))))
    h = 1.0 / max(n)
    rf = synth.uniform_field(synth.grid_shape(dim, n), 40 + sum(n), zero_bc=False)
    ref = oracle.mg_restrict(rf)
    rcd = to_dev(np.full(synth.grid_shape(dim, nc), np.nan), pad=pad)
    st.stencil_mg_restrict(to_dev(rf, pad=pad), rcd, h)
    torch.cuda.synchronize()
    assert rel_err(to_host(rcd), ref) <= 1e-14


@pytest.mark.parametrize("dim,n", SIZES)
@pytest.mark.parametrize("pad", [0, 5])
def test_prolong_add_matches_oracle(dim, n, pad):
    nc = tuple(m - 1 for m in reversed(oracle.coarse_shape(synth.grid_shape(dim, n))))
    h = 1.0 / max(n)
    ec = synth.uniform_field(synth.grid_shape(dim, nc), 50 + sum(n), zero_bc=False)
    uf = synth.uniform_field(synth.grid_shape(dim, n), 60 + sum(n), zero_bc=False)
    ref = oracle.mg_prolong_add(ec, uf)
    ufd = to_dev(uf, pad=pad)
    st.stencil_mg_prolong_add(to_dev(ec, pad=pad), ufd, h)
    torch.cuda.synchronize()
    got = to_host(ufd)
    assert rel_err(got, ref) <= 1e-14
    # the fine boundary is untouched
    for ax in range(dim):
        for side in (0, -1):
            idx = [slice(None)] * dim
            idx[ax] = side
            assert np.array_equal(got[tuple(idx)], uf[tuple(idx)])


@pytest.mark.parametrize("dim,n,levels", [(3, (16, 16, 16), 0), (3, (24, 16, 8), 0), (3, (32, 32, 32), 2),
                                          (3, (15, 15, 15), 0), (3, (19, 19, 19), 3),
                                          (2, (64, 64), 0), (2, (96, 40), 0), (2, (7, 9), 0), (2, (77, 77), 0)])
@pytest.mark.parametrize("pre,post", [(2, 2), (1, 0), (0, 3)])
def test_vcycle_matches_oracle(dim, n, levels, pre, post):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u0 = synth.uniform_field(shape, 70 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 80 + sum(n))
    L = oracle.mg_levels(shape, levels if levels else 64)
    ref = oracle.mg_vcycle(u0, f, h, L, pre, post, 10)
    ud = to_dev(u0, pad=2)
    st.stencil_mg_vcycle(ud, to_dev(f, pad=2), h, pre=pre, post=post, coarse_sweeps=10, max_levels=levels)
    torch.cuda.synchronize()
    got = to_host(ud)
    assert rel_err(got, ref) <= TOL_F64
    assert np.array_equal(got[(0,) * dim], u0[(0,) * dim])


@pytest.mark.parametrize("dim,n", [(3, 64), (2, 256), (3, 45), (2, 255)])
def test_mg_solve_closed_form_and_history(dim, n):
    h = 1.0 / n
    modes = (2, 3, 1)
    f = synth.zero_boundary(np.ascontiguousarray(14.0 * math.pi ** 2 * dr.sine_mode(dim, n, modes)))
    lam = dr.symbol(dim, [m * math.pi * h for m in modes])
    uh = h * h * f / lam
    ud = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    out = st.stencil_mg_solve(ud, to_dev(f), h, rel_tol=1e-10, max_cycles=30)
    assert out["converged"] and out["cycles"] <= 12
    assert out["levels"] == oracle.mg_levels(f.shape)
    hist = np.array(out["history"])
    assert np.all(hist[1:] < hist[:-1])
    assert rel_err(to_host(ud), uh) <= 1e-8
    # the oracle's own solve takes the same number of cycles and the same iterates
    if n <= 64:
        uo, rr, k, conv = oracle.mg_solve(np.zeros_like(f), f, h, 1e-10, 30)
        assert k == out["cycles"]
        assert rel_err(to_host(ud), uo) <= 1e-11


def test_mg_not_converged_and_bad_options():
    n = 16
    shape = synth.grid_shape(3, n)
    f = synth.uniform_field(shape, 3)
    ud = torch.zeros(shape, dtype=torch.float64, device="cuda")
    out = st.stencil_mg_solve(ud, to_dev(f), 1.0 / n, rel_tol=1e-30, max_cycles=2)
    assert not out["converged"] and out["cycles"] == 2
    with pytest.raises(st.StencilError):
        st.stencil_mg_vcycle(ud, to_dev(f), 1.0 / n, coarse_sweeps=0)
    with pytest.raises(st.StencilError):  # coarse grid of the wrong size
        st.stencil_mg_restrict(to_dev(f), torch.zeros(synth.grid_shape(3, 7), dtype=torch.float64,
                                                      device="cuda"), 1.0 / n)
    with pytest.raises(st.StencilError):  # mixed parity, not cubic: no coarse grid
        g = synth.grid_shape(3, (8, 7, 8))
        st.stencil_mg_restrict(torch.zeros(g, dtype=torch.float64, device="cuda"),
                               torch.zeros(synth.grid_shape(3, (4, 4, 4)), dtype=torch.float64, device="cuda"),
                               1.0 / 8)
