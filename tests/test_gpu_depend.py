"""Dependency-driven red-black sweeps (the GPU form of the paper's Hyb-depend variant):
the result equals the barrier-per-colour sweeps and the oracle's red-black sweep for any
task size and CTA count; a dependency that is never met ends in a timeout status that
the host reads, with the context still usable."""
import numpy as np
import pytest
import torch

import oracle
import paper_1810_04033_gb300 as st
import synth
from tests.parity_util import TOL_F64, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n,rows,cols,ctas", [
    (2, (64, 64), 0, 0, 0), (2, (301, 97), 3, 0, 5), (2, (30, 500), 1, 0, 0), (2, (2, 2), 1, 0, 1),
    (3, (24, 24, 24), 0, 0, 0), (3, (40, 17, 33), 1, 4, 3), (3, (9, 9, 70), 4, 3, 0), (3, (33, 65, 20), 2, 7, 0)])
@pytest.mark.parametrize("sweeps", [1, 4])
def test_depend_matches_oracle_and_barrier_sweeps(dim, n, rows, cols, ctas, sweeps):
    h = 1.0 / max(n)
    u0 = synth.uniform_field(synth.grid_shape(dim, n), 1200 + sum(n), zero_bc=False)
    f = synth.uniform_field(u0.shape, 1201 + sum(n))
    ud, fd = to_dev(u0, pad=3), to_dev(f, pad=3)
    out = st.stencil_smooth_depend(ud, fd, h, sweeps, rows=rows, cols=cols, ctas=ctas)
    assert out["status"] == 0
    bd = to_dev(u0, pad=3)
    st.stencil_smooth_coloured(bd, fd, h, sweeps, op=st.OP_FD)
    torch.cuda.synchronize()
    got = to_host(ud)
    # the same updates in the same per-vertex order: identical bits
    assert np.array_equal(got, to_host(bd))
    assert rel_err(got, oracle.fd_gs_redblack(u0, f, h, sweeps)) <= TOL_F64


def test_unmet_dependency_times_out_and_context_survives():
    dim, n = 2, (64, 256)
    h = 1.0 / 256
    u0 = synth.uniform_field(synth.grid_shape(dim, n), 1300, zero_bc=False)
    f = synth.uniform_field(u0.shape, 1301)
    fd = to_dev(f)
    # block 5 never reports progress.  With one CTA the tasks run in claim order, so the
    # first wait that runs out is phase 1 of block 4 waiting for block 5.
    out = st.stencil_smooth_depend(to_dev(u0), fd, h, 3, rows=8, ctas=1, max_wait_ns=2_000_000, test_stall=6)
    assert out["status"] == st.ETIMEDOUT and out["stalled_at"] == 5
    # with every CTA resident, all tasks are claimed at once and any wait in the cone of
    # block 5 (blocks 5 +- 6 over the 6 phases) may run out first
    out = st.stencil_smooth_depend(to_dev(u0), fd, h, 3, rows=8, max_wait_ns=2_000_000, test_stall=6)
    assert out["status"] == st.ETIMEDOUT and abs(out["stalled_at"] - 5) <= 6
    # the context still works: a normal run afterwards gives the oracle's result
    ud = to_dev(u0)
    assert st.stencil_smooth_depend(ud, fd, h, 2)["status"] == 0
    torch.cuda.synchronize()
    assert rel_err(to_host(ud), oracle.fd_gs_redblack(u0, f, h, 2)) <= TOL_F64


def test_depend_refuses_q1():
    u = torch.zeros(synth.grid_shape(2, (8, 8)), dtype=torch.float64, device="cuda")
    g = st.grid_for(u, 0.125, st.OP_Q1)
    o = st.DependOpts(0, 0, 0, 0, 0, -1, 0)
    rc = st.lib().stencil_smooth_depend(__import__("ctypes").byref(g), st._ptr(u), st._ptr(u.clone()), 1,
                                        __import__("ctypes").byref(o), None)
    assert rc == st.EINVAL


@pytest.mark.parametrize("dim,n", [(2, (61, 47)), (3, (13, 11, 17))])
@pytest.mark.parametrize("mode,kmax", [(st.COST_UNIFORM, 100), (st.COST_LINEAR, 100), (st.COST_NONE, 5)])
@pytest.mark.parametrize("depend", [None, {"rows": 3}, {"rows": 2, "cols": 4}])
def test_expensive_stencil_matches_oracle(dim, n, mode, kmax, depend):
    """S(k): k FP64 sin evaluations per update (uniform, or linear over the mesh); the
    GPU sin differs from the host's by a few ulp, far below the 2^-20 scale of the
    perturbation, so the result matches the oracle to FP64 tolerance."""
    h = 1.0 / max(n)
    u0 = synth.uniform_field(synth.grid_shape(dim, n), 1400 + sum(n), zero_bc=False)
    f = synth.uniform_field(u0.shape, 1401 + sum(n))
    ud = to_dev(u0, pad=2)
    assert st.stencil_smooth_expensive(ud, to_dev(f, pad=2), h, 2, mode, kmax, depend=depend) == 0
    torch.cuda.synchronize()
    got = to_host(ud)
    assert rel_err(got, oracle.fd_gs_redblack_cost(u0, f, h, 2, mode, kmax)) <= TOL_F64
    if mode != st.COST_NONE:
        # the perturbation is really applied: the plain sweep differs by far more than rounding
        assert rel_err(got, oracle.fd_gs_redblack(u0, f, h, 2)) > 1e-9
