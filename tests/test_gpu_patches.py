"""GPU parity of the patch batch (halo fill + coloured GS of every patch per sweep)
against the oracle's patch smoother on the same lattice, sizes and fields."""
import numpy as np
import pytest
import torch

import oracle
import paper_1810_04033_gb300 as st
import synth
from tests.parity_util import TOL_F64, rel_err

pytestmark = pytest.mark.gpu


def _run(lat, edges, seed, sweeps, u_random=True, tune=False):
    L = synth.PatchLattice(lat=lat, seed=seed, edges=edges, u_random=u_random)
    ref = oracle.patch_smooth(L.lat, L.np_sizes, L.offsets, L.u, L.f, sweeps)
    b = st.PatchBatch(L.np_sizes, L.offsets, L.neighbours27())
    ud = torch.from_numpy(L.u.copy()).cuda()
    fd = torch.from_numpy(L.f).cuda()
    if tune:
        before = ud.clone()
        t, c = b.autotune(ud, fd)
        assert t in (128, 256, 512) and c in (2, 4, 8)
        assert torch.equal(ud, before)  # autotuning works on a copy
    b.smooth(ud, fd, sweeps)
    torch.cuda.synchronize()
    got = ud.cpu().numpy()
    b.close()
    return got, ref, L


@pytest.mark.parametrize("lat,edges,sweeps", [((2, 2, 2), (4, 6, 8), 1), ((3, 2, 2), (4, 8, 12), 3),
                                              ((2, 3, 2), (8, 12, 16, 24, 32), 2), ((1, 1, 1), (2,), 2),
                                              ((4, 4, 4), (8, 12, 16, 24, 32), 2),
                                              ((2, 1, 1), (61, 64), 2), ((1, 2, 1), (3, 63), 1)])
def test_patch_batch_matches_oracle(lat, edges, sweeps):
    got, ref, _ = _run(lat, edges, 11, sweeps)
    assert rel_err(got, ref) <= TOL_F64


def test_patch_batch_per_patch_equals_standalone_gs_with_same_halo():
    """Patches are independent within a sweep: each patch equals a plain coloured GS of
    that patch alone after the halo fill (the paper's regular patches in a
    block-structured mesh)."""
    L = synth.PatchLattice(lat=(2, 2, 1), seed=4, edges=(6, 10), u_random=True)
    filled = oracle.patch_halo_fill(L.lat, L.np_sizes, L.offsets, L.u)
    b = st.PatchBatch(L.np_sizes, L.offsets, L.neighbours27())
    ud = torch.from_numpy(L.u.copy()).cuda()
    b.smooth(ud, torch.from_numpy(L.f).cuda(), 1)
    torch.cuda.synchronize()
    got = ud.cpu().numpy()
    for p in range(4):
        n = int(L.np_sizes[p])
        ref = oracle.gs_coloured(L.view(filled, p), L.view(L.f, p), 1.0 / n, 1)
        assert rel_err(L.view(got, p), ref) <= TOL_F64


def test_patch_batch_autotune_keeps_results():
    got, ref, _ = _run((2, 2, 2), (8, 12, 16), 5, 2, tune=True)
    assert rel_err(got, ref) <= TOL_F64


def test_patch_batch_rejects_bad_tables():
    with pytest.raises(st.StencilError):
        st.PatchBatch([8, 8], [0, 729], np.full((2, 27), 5, dtype=np.int32))  # neighbour 5 >= npatch
    with pytest.raises(st.StencilError):
        st.PatchBatch([1], [0], np.full((1, 27), -1, dtype=np.int32))  # n < 2
