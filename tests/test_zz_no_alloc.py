"""The allocation-free residual entry point, rtlb_residual_noalloc.

It serves callers that cannot call cudaMalloc (allocator hooks, host
callbacks, processes whose device memory pool belongs to another framework,
real-time loops that must stay out of the allocator).  It must give the same
residual as the regular entry point, rtlb_last_residual, which uses a scratch
buffer owned by the context.  This file is collected last on purpose: a run
that stops at the first failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2609_23057_b300 import _lib
from paper_2609_23057_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc_residual(torch, old, new):
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    st = _lib.lib().rtlb_residual_noalloc(old.data_ptr(), new.data_ptr(), old.numel(),
                                          out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, _lib.STATUS_NAMES.get(st, st)
    d = out.cpu().numpy()
    assert d[2] == 0.0
    return d[0] / d[1]


def test_noalloc_matches_context_residual_on_two_calls_in_a_row():
    import torch
    from paper_2609_23057_b300.solver import solver_for
    assert torch.cuda.is_available()
    w = W.random_medium(45, 31, 4, 8, seed=31, n_phase=2, steps=2)
    s = solver_for(w, "fp32")
    s.set_state(torch.from_numpy(W.random_state(31, 45, 32, seed=32, dtype=np.float32)).cuda())
    for _ in range(2):
        old = s.get_state()
        s.step(1)
        new = s.get_state()
        ref = s.last_residual()
        got = _noalloc_residual(torch, old, new)
        assert ref > 0
        assert got == pytest.approx(ref, rel=1e-5)
    s.close()


def test_noalloc_rejects_oversize_and_bad_arguments():
    import torch
    a = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    L = _lib.lib()
    too_many = (1 << 30) + 4
    assert L.rtlb_residual_noalloc(a.data_ptr(), a.data_ptr(), too_many, out.data_ptr(), None) == 2
    assert L.rtlb_residual_noalloc(a.data_ptr(), a.data_ptr(), 6, out.data_ptr(), None) == 1
    assert L.rtlb_residual_noalloc(None, a.data_ptr(), 8, out.data_ptr(), None) == 1
    # host memory (pageable or pinned) is rejected before any launch
    h = np.zeros(8, np.float32)
    hp = torch.zeros(8, dtype=torch.float32).pin_memory()
    assert L.rtlb_residual_noalloc(h.ctypes.data, a.data_ptr(), 8, out.data_ptr(), None) == 1
    assert L.rtlb_residual_noalloc(a.data_ptr(), hp.data_ptr(), 8, out.data_ptr(), None) == 1
    ho = np.zeros(3, np.float64)
    assert L.rtlb_residual_noalloc(a.data_ptr(), a.data_ptr(), 8, ho.ctypes.data, None) == 1
    assert L.rtlb_residual_noalloc(a.data_ptr(), a.data_ptr(), 8, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0, 0.0]
