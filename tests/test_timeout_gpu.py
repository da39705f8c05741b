"""The bounded waits of the tensor-core kernels, made to run out on purpose.

rtlb_test_stall_next_step leaves one state load of the first CTA unissued, so
that CTA's converter warps wait for data that never arrives.  Nothing is in
flight for the missing load: the wait gives up after about 2 s, the CTA drains
what it did issue (loads and MMAs; on a CTA pair both CTAs wait for the even
CTA's final commit), frees its tensor memory and returns.  The next call that
reads the device error flag reports RTLB_E_TIMEOUT, and the context stays
usable: a step after it matches the oracle again.
"""
import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import oracle_problem, rel_err_I

pytestmark = pytest.mark.gpu

RTLB_E_TIMEOUT = 10


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.mark.parametrize("prec,nzen,naz,nx,nz", [
    ("bf16", 4, 8, 512, 4),      # single-CTA kernel, n = 32, 16 tiles
    ("bf16x2", 8, 8, 512, 4),    # CTA-pair kernel, n = 64, 8 tile pairs
])
def test_stalled_load_times_out_and_context_recovers(torch_cuda, orc, prec, nzen, naz, nx, nz):
    from paper_2609_23057_b300 import _lib
    from paper_2609_23057_b300.solver import solver_for
    w = W.random_medium(nx, nz, nzen, naz, seed=41, bc=(2, 0, 1, 1), n_phase=1, steps=1)
    S0 = W.random_state(nz, nx, w.n, seed=42, dtype=np.float32)
    s = solver_for(w, prec)
    dS0 = torch_cuda.from_numpy(S0).cuda()
    s.set_state(dS0)
    s.stall_next_step()
    s.step(1)                                     # the launch itself succeeds
    with pytest.raises(_lib.RtlbError) as ei:
        s.total_intensity()                       # reads (and clears) the error flag
    assert ei.value.status == RTLB_E_TIMEOUT
    # the hook disarms after one launch and the context keeps working
    s.set_state(dS0)
    s.step(2)
    s.total_intensity()
    got = s.get_state().cpu().numpy().astype(np.float64)
    s.close()
    ref = oracle_problem(orc, w).run(S0.astype(np.float64), 2)
    # bf16 operands: ~3.2e-3 per step on these media (see the tensor-core
    # parity tests), 1e-2 for two steps
    assert rel_err_I(got, ref) < 1e-2


def test_stall_hook_refused_without_tensor_cores(torch_cuda):
    from paper_2609_23057_b300 import _lib
    from paper_2609_23057_b300.solver import solver_for
    w = W.random_medium(64, 4, 4, 8, seed=43, n_phase=1, steps=1)
    s = solver_for(w, "fp32")
    with pytest.raises(_lib.RtlbError) as ei:
        s.stall_next_step()
    assert ei.value.status == 11
    s.close()
