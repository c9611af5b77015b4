"""Launch-shape tuning on the GPU: stencil_autotune records a shape per (call, grid);
the smoothers give the same bits under every chunking (3D planes per CTA, 2D rows per
warp; the 2D depth, one or two sweeps per pass, changes the fixed-point scale and so
the rounding), every shape stays within the FP64 bar of the oracle, and a saved cache
steers a fresh process through STENCIL_TUNING_CACHE."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_1810_04033_gb300 as st
import synth
from tests.parity_util import TOL_F64, apply_err, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (dim, n, pad): 64-byte pitches (TMA-staged kernels) and one odd pitch
GRIDS = [(3, (70, 45, 37), 1), (3, (24, 20, 18), 0), (2, (300, 270), 7), (2, (129, 97), 0)]
SHAPES_3D = {st.CALL_APPLY_ELEMENTWISE: [(c, 0) for c in (4, 8, 16, 32)],
             st.CALL_APPLY_STENCIL: [(c, 0) for c in (4, 8, 16, 32)],
             st.CALL_SMOOTH_COLOURED: [(c, 0) for c in (2, 4, 8, 16)],
             st.CALL_SMOOTH_JACOBI: [(c, 0) for c in (4, 8, 16, 32)]}
SHAPES_2D = {st.CALL_APPLY_ELEMENTWISE: [(r, 0) for r in (16, 32, 64, 256)],
             st.CALL_APPLY_STENCIL: [(r, 0) for r in (16, 64, 128)],
             st.CALL_SMOOTH_COLOURED: [(r, d) for r in (16, 64, 256, 1024) for d in (1, 2)],
             st.CALL_SMOOTH_JACOBI: [(r, d) for r in (16, 64, 256, 1024) for d in (1, 2)]}


def _like(u):
    """An array with u's shape and strides (padded rows included)."""
    return torch.empty_strided(u.size(), u.stride(), dtype=u.dtype, device=u.device)


def _run(call, u, f, h, sweeps=5):
    if call in (st.CALL_APPLY_ELEMENTWISE, st.CALL_APPLY_STENCIL):
        y = _like(u).fill_(float("nan"))
        form = st.FORM_ELEMENTWISE if call == st.CALL_APPLY_ELEMENTWISE else st.FORM_STENCIL
        st.stencil_apply(u, y, h, form)
        return y
    x = _like(u).copy_(u)
    if call == st.CALL_SMOOTH_COLOURED:
        st.stencil_smooth_coloured(x, f, h, sweeps)
    else:
        st.stencil_smooth_jacobi(x, f, _like(x), h, sweeps, 2.0 / 3.0)
    return x


def _ref(call, u, f, h, sweeps=5):
    if call == st.CALL_APPLY_ELEMENTWISE:
        return oracle.apply_elementwise(u, h)
    if call == st.CALL_APPLY_STENCIL:
        return oracle.apply_stencil(u, h)
    if call == st.CALL_SMOOTH_COLOURED:
        return oracle.gs_coloured(u, f, h, sweeps)
    return oracle.jacobi(u, f, h, 2.0 / 3.0, sweeps)


@pytest.mark.parametrize("dim,n,pad", GRIDS)
def test_every_shape_matches_the_oracle_and_smoothers_keep_their_bits(dim, n, pad):
    h = 1.0 / max(n)
    shape = synth.grid_shape(dim, n)
    u = synth.uniform_field(shape, 4000 + sum(n), zero_bc=False)
    f = synth.uniform_field(shape, 4001 + sum(n))
    ud, fd = to_dev(u, pad), to_dev(f, pad)
    st.stencil_tuning_clear()
    try:
        for call, shapes in (SHAPES_3D if dim == 3 else SHAPES_2D).items():
            # the 2D smoothers keep one fixed-point scale for the two sweeps of a pass,
            # so their bits depend on the depth (not on the rows): one base per depth
            base = {}
            for d in sorted({d for _, d in shapes}):
                if d:
                    st.stencil_tuning_set(ud, h, call, 256, d)
                base[d] = _run(call, ud, fd, h)
                st.stencil_tuning_set(ud, h, call, None)
            base.setdefault(0, _run(call, ud, fd, h))
            torch.cuda.synchronize()
            ref = _ref(call, u, f, h)
            for chunk, depth in shapes:
                st.stencil_tuning_set(ud, h, call, chunk, depth)
                got = _run(call, ud, fd, h)
                torch.cuda.synchronize()
                if call in (st.CALL_SMOOTH_COLOURED, st.CALL_SMOOTH_JACOBI):
                    assert torch.equal(got, base[depth]), (call, chunk, depth)
                    assert rel_err(to_host(got), ref) <= TOL_F64
                else:
                    assert apply_err(to_host(got), ref, u, h) <= TOL_F64, (call, chunk)
            st.stencil_tuning_set(ud, h, call, None)
    finally:
        st.stencil_tuning_clear()


def test_autotune_records_a_candidate_and_the_cache_steers_a_new_process(tmp_path):
    n = (96, 80, 64)
    h = 1.0 / 96
    shape = synth.grid_shape(3, n)
    u = synth.uniform_field(shape, 4100)
    ud = to_dev(u, 7)
    u2 = to_dev(synth.uniform_field(synth.grid_shape(2, (1000, 600)), 4101), 7)
    st.stencil_tuning_clear()
    try:
        got = {}
        for call, sweeps in ((st.CALL_APPLY_ELEMENTWISE, 0), (st.CALL_APPLY_STENCIL, 0),
                             (st.CALL_SMOOTH_COLOURED, 6), (st.CALL_SMOOTH_JACOBI, 6)):
            chunk, depth, ms = st.stencil_autotune(ud, h, call, sweeps)
            assert (chunk, depth) in SHAPES_3D[call] + [(32, 0)] and ms > 0
            assert st.stencil_tuning_get(ud, h, call)[:2] == (chunk, depth)
            got[call] = (chunk, depth)
            c2, d2, ms2 = st.stencil_autotune(u2, 1.0 / 1000, call, sweeps)
            assert ms2 > 0 and (d2 in (1, 2) if sweeps else d2 == 0)
        path = str(tmp_path / "cache.json")
        st.stencil_tuning_save(path)
        code = ("import paper_1810_04033_gb300 as st, torch\n"
                "u = torch.zeros(65, 81, 104, dtype=torch.float64, device='cuda')[..., :97]\n"
                "print(st.stencil_tuning_get(u, 1 / 96, %d))\n" % st.CALL_SMOOTH_COLOURED)
        env = dict(os.environ, STENCIL_TUNING_CACHE=path, PYTHONPATH=ROOT)
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT,
                             timeout=300)
        assert out.returncode == 0, out.stderr
        assert out.stdout.strip().startswith("(%d, %d," % got[st.CALL_SMOOTH_COLOURED]), out.stdout
    finally:
        st.stencil_tuning_clear()
