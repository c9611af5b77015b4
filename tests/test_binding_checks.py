"""Argument checks of the Python binding that run before any library call, so that a
wrong buffer raises in Python instead of letting a kernel or a host copy touch memory
outside it.  Host-only: non-CUDA tensors and handles built without a library call."""
import numpy as np
import pytest
import torch

import paper_1810_04033_gb300 as st


def test_device_buffer_rejects_host_wrong_dtype_and_short_buffers():
    with pytest.raises(ValueError, match="CUDA"):
        st._device_buffer(torch.zeros(2, dtype=torch.float64), "norms2", None, 2)
    with pytest.raises(ValueError, match="CUDA"):
        st._device_buffer(np.zeros(2), "norms2", None, 2)
    with pytest.raises(ValueError, match="CUDA"):
        st._device_buffer(torch.zeros(2, dtype=torch.float64, device="meta"), "norms2", None, 2)


def test_residual_and_transfers_reject_host_tensors():
    u = torch.zeros(5, 5, dtype=torch.float64)
    with pytest.raises(ValueError):
        st.stencil_residual(u, u.clone(), 0.25, norms2=torch.zeros(2, dtype=torch.float64))
    with pytest.raises(ValueError):
        st.stencil_mg_restrict(torch.zeros(9, 9, 9, dtype=torch.float64), torch.zeros(5, 5, 5, dtype=torch.float64),
                               0.125)
    with pytest.raises(ValueError):
        st.stencil_mg_prolong_add(torch.zeros(5, 5, 5, dtype=torch.float64), torch.zeros(9, 9, 9, dtype=torch.float64),
                                  0.125)


def test_packed_numel_is_the_end_of_the_last_patch():
    assert st.packed_numel([], []) == 0
    assert st.packed_numel([2, 3], [0, 27]) == 27 + 64
    # offsets need not be sorted: the patch that ends last counts
    assert st.packed_numel([3, 2], [27, 0]) == 27 + 64
    assert st.packed_numel([4, 1], [0, 200]) == 208


def test_patch_batch_rejects_host_and_short_arrays():
    b = st.PatchBatch.__new__(st.PatchBatch)
    b._h, b.npatch, b.numel = None, 2, 91
    with pytest.raises(ValueError):
        b.smooth(torch.zeros(91, dtype=torch.float64), torch.zeros(91, dtype=torch.float64), 1)
    with pytest.raises(ValueError):
        b.autotune(torch.zeros(91, dtype=torch.float64), torch.zeros(91, dtype=torch.float64))


def _bare_server():
    s = st.Server.__new__(st.Server)
    s._h, s._n = None, {}
    return s


def test_server_submit_checks_array_lengths():
    s = _bare_server()
    with pytest.raises(ValueError, match=r"\(n\+1\)\^3 = 125"):
        s.submit(st.REQ_SMOOTH, 4, f=np.zeros(124))
    with pytest.raises(ValueError, match="u0"):
        s.submit(st.REQ_SMOOTH, 4, f=np.zeros(125), u0=np.zeros(126))


def test_server_fetch_sizes_by_the_ticket():
    s = _bare_server()
    with pytest.raises(st.StencilError) as e:
        s.fetch(7)
    assert e.value.code == st.ENOTFOUND
    s._n[7] = 16
    with pytest.raises(ValueError, match="n = 16"):
        s.fetch(7, 8)
