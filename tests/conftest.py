import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def crop_ref_1000(orc):
    """The 256x256 crop [896,1152)^2 of the 2048x2048, n = 64 medium run for
    1000 steps from zero by the FP64 oracle (shared by the precision-form
    accuracy tests): (workload, oracle problem, state, top radiance)."""
    from paper_2609_23057_b300 import workloads as W
    from _util import oracle_problem
    w = W.precision_crop(steps=1000)
    P = oracle_problem(orc, w)
    ref = P.run(P.zero_state(), w.steps)
    return w, P, ref, P.radiance_out(ref, orc.SIDE_TOP)
