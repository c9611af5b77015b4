"""The request server: continuous batching with admission by device-memory budget.

Each request's result equals the same request run alone (bit for bit: every request
uses its own buffers and deterministic kernels) and matches the oracle; host-made
failure paths (over-budget request, unknown ticket, wait timeout) return error codes.
"""
import numpy as np
import pytest

import oracle
import paper_1810_04033_gb300 as st
import synth
from tests.parity_util import TOL_F64, rel_err

pytestmark = pytest.mark.gpu

GB = 1 << 30


def test_seeded_rhs_matches_host_generator_and_oracle_smooth():
    n = 20
    srv = st.Server(4 * GB)
    t = srv.submit(st.REQ_SMOOTH, n, sweeps=20, f_seed=12345)
    res = srv.wait(t)
    assert res["status"] == 0 and res["iterations"] == 20
    u = srv.fetch(t, n)
    f = synth.splitmix_field(n, 12345)
    ref = oracle.gs_coloured(np.zeros_like(f), f, 1.0 / n, 20)
    assert rel_err(u, ref) <= TOL_F64
    srv.close()


def test_solve_request_matches_oracle_refinement():
    n = 16
    f = synth.uniform_field((n + 1,) * 3, 77)
    srv = st.Server(4 * GB, inner_dtype=st.F32)
    t = srv.submit(st.REQ_SOLVE, n, rel_tol=1e-8, f=f)
    res = srv.wait(t)
    assert res["status"] == 0 and res["relres"] <= 1e-8
    u = srv.fetch(t, n)
    xo, hist, k, conv = oracle.ir_solve(np.zeros_like(f), f, 1.0 / n, 1e-8, 100000, 8, 1)
    assert conv
    assert abs(k - res["iterations"]) <= 2
    assert rel_err(u, xo) <= 1e-6
    srv.close()


@pytest.mark.parametrize("n", [16, 24, 15])
def test_solve_request_multigrid_matches_oracle(n):
    """SOLVE with the multigrid solver: same V-cycles as the oracle's (V(2,2), 20
    coarsest sweeps), so the same cycle count and iterate; n = 15 coarsens to 8 (not nested)."""
    f = synth.splitmix_field(n, 991 + n)
    srv = st.Server(4 * GB, solver=st.SOLVER_MG)
    t = srv.submit(st.REQ_SOLVE, n, rel_tol=1e-9, f_seed=991 + n)
    res = srv.wait(t)
    assert res["status"] == 0 and res["relres"] <= 1e-9
    u = srv.fetch(t, n)
    uo, hist, k, conv = oracle.mg_solve(np.zeros_like(f), f, 1.0 / n, 1e-9, 100000, pre=2, post=2,
                                        coarse_sweeps=20)
    assert conv and k == res["iterations"]
    assert rel_err(u, uo) <= 1e-11
    srv.close()


def _mix(seed=3, count=24):
    g = synth.rng(seed)
    out = []
    for i in range(count):
        n = int(g.integers(6, 33))
        kind = st.REQ_SOLVE if g.random() < 0.5 else st.REQ_SMOOTH
        out.append(dict(kind=kind, n=n, sweeps=20, rel_tol=1e-8, f_seed=int(g.integers(0, 2 ** 40))))
    return out


def test_results_in_the_mix_equal_results_alone():
    reqs = _mix()
    # alone: one request at a time
    alone = []
    srv = st.Server(8 * GB, max_inflight=1, streams=1)
    for r in reqs:
        t = srv.submit(**r)
        srv.wait(t)
        alone.append(srv.fetch(t, r["n"]))
    srv.close()
    # in the mix: everything submitted at once, several streams, small budget so that
    # requests are admitted as others finish
    budget = 4 * 1024 * 1024
    srv = st.Server(budget, max_inflight=8, streams=4)
    tickets = [srv.submit(**r) for r in reqs]
    seen_pending = srv.stats()["pending"] > 0
    outs = []
    for t, r in zip(tickets, reqs):
        res = srv.wait(t)
        assert res["status"] == 0
        assert res["t_admit"] >= res["t_submit"] and res["t_done"] >= res["t_admit"]
        outs.append(srv.fetch(t, r["n"]))
    stats = srv.stats()
    srv.close()
    assert seen_pending
    assert stats["completed"] == len(reqs) and stats["hbm_used"] == 0
    for a, b in zip(alone, outs):
        assert np.array_equal(a, b)


def test_admission_refusal_unknown_ticket_and_timeout():
    srv = st.Server(16 * 1024 * 1024)  # 16 MiB budget
    with pytest.raises(st.StencilError) as ei:
        srv.submit(st.REQ_SMOOTH, 256, sweeps=1, f_seed=1)  # needs ~700 MB
    assert ei.value.code == -3
    with pytest.raises(st.StencilError) as ei:
        srv.wait(987654, timeout_us=0)
    assert ei.value.code == -7
    t = srv.submit(st.REQ_SOLVE, 24, rel_tol=0.0, f_seed=5)  # never converges before the cap
    with pytest.raises(st.StencilError) as ei:
        srv.wait(t, timeout_us=1)
    assert ei.value.code == -4
    assert srv.poll(t) is None or srv.poll(t)["status"] in (0, -6)
    srv.close()  # stops the engine with the solve still in progress
