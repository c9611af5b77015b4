"""Every bounded device wait of the TMA-staged kernels completed: after the calls of the
whole suite before this file (and a round of TMA-staged calls here), the device status
flags are all clear.  No wait is made to run out: the GPU is never faulted or stalled
on purpose."""
import numpy as np
import pytest
import torch

import paper_1810_04033_gb300 as st
import synth
from tests.parity_util import to_dev

pytestmark = pytest.mark.gpu


def test_no_bounded_wait_ran_out():
    n = (64, 48, 40)
    h = 1.0 / 64
    shape = synth.grid_shape(3, n)
    u = to_dev(synth.uniform_field(shape, 5000), 7)
    f = to_dev(synth.uniform_field(shape, 5001), 7)
    y = to_dev(np.zeros(shape), 7)
    w = to_dev(np.zeros(shape), 7)
    st.stencil_apply(u, y, h, st.FORM_STENCIL)          # k_ops3t
    st.stencil_smooth_coloured(u, f, h, 4)                # k_gs_half_t
    st.stencil_smooth_jacobi(y, f, w, h, 4, 2.0 / 3.0)   # k_jac3_sweep
    u32 = to_dev(synth.uniform_field(shape, 5002), 3, dtype=torch.float32)  # pitch 68
    f32 = to_dev(synth.uniform_field(shape, 5003), 3, dtype=torch.float32)
    st.stencil_smooth_coloured(u32, f32, h, 3)            # k_gs_lp_t
    assert st.stencil_device_status() == 0
    assert st.stencil_device_status(clear=True) == 0
