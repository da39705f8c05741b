"""GPU parity of the 3xTF32 tensor-core form (precision "tf32x3") with the
FP64 oracle, at the float32 path's tolerance.

Each operand of the scattered term beta * Z S~ is split into tf32 hi + lo
(about 22 significand bits together); the three products hi.hi, hi.lo and
lo.hi accumulate in float32, and the dropped lo.lo product is below 2^-22 of
each term.  The unscattered and forward-scattered light are applied in
float32 exactly as in the FP32 form.  So a step carries the float32 form's
error (a few units of 2^-24 per term): the same 1e-5 relative bound on I and
1e-5 absolute on the degree of polarization holds.  All calls go through the
C ABI.
"""
import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import abs_err_dop, oracle_problem, rel_err_I

pytestmark = pytest.mark.gpu

TOL_I = 1e-5
TOL_DOP = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _run(torch, w, S0, steps, prec="tf32x3"):
    from paper_2609_23057_b300.solver import solver_for
    s = solver_for(w, prec)
    if S0 is not None:
        s.set_state(torch.from_numpy(np.asarray(S0, np.float32)).cuda())
    s.step(steps)
    s.total_intensity()                       # surfaces a device-side timeout as an error
    got = s.get_state().cpu().numpy().astype(np.float64)
    s.close()
    return got


@pytest.mark.parametrize("nx,nz,nzen,naz,bc,nph", [
    (256, 8, 2, 4, (2, 0, 1, 1), 2),     # n = 8: one K chunk, converter group 1 idle
    (256, 8, 4, 4, (2, 0, 1, 1), 2),     # n = 16
    (384, 6, 4, 8, (2, 2, 1, 1), 2),     # n = 32, rows alternate class
    (130, 3, 4, 8, (1, 1, 0, 0), 1),     # one class, ragged last tile, periodic z
    (512, 128, 2, 4, (2, 0, 0, 0), 2),   # n = 8, several tiles per CTA
    (200, 7, 4, 8, (2, 0, 1, 1), 3),     # tiles straddling rows: mixed tiles on the CUDA cores
])
def test_tf32x3_matches_oracle(torch_cuda, orc, nx, nz, nzen, naz, bc, nph):
    w = W.random_medium(nx, nz, nzen, naz, seed=nx + 3 * nz, bc=bc, n_phase=nph, steps=4)
    w.phase_index = (np.arange(nz)[:, None] % nph * np.ones((1, nx))).astype(np.uint8)
    S0 = W.random_state(nz, nx, w.n, seed=nx + nz)
    ref = oracle_problem(orc, w).run(S0, w.steps)
    got = _run(torch_cuda, w, S0, w.steps)
    assert rel_err_I(got, ref) < TOL_I
    assert abs_err_dop(got, ref) < TOL_DOP
    # a real tensor-core result: the bf16 form of the same problem is far off
    assert rel_err_I(_run(torch_cuda, w, S0, w.steps, "bf16"), ref) > 10 * TOL_I


def test_tf32x3_crop128_100_steps(torch_cuda, orc):
    """The 128x128 centre crop of the 512x512, n = 32 steady-state medium, run
    as its own problem for 100 steps from zero (top beam, vacuum sides)."""
    w = W.steady().crop(192, 320, 192, 320)
    P = oracle_problem(orc, w)
    ref = P.run(P.zero_state(), 100)
    got = _run(torch_cuda, w, None, 100)
    assert rel_err_I(got, ref) < TOL_I
    assert abs_err_dop(got, ref) < TOL_DOP


def test_tf32x3_full_size_sampled_sites(torch_cuda, orc):
    """512x512, n = 32 (the steady-state workload in the launch configuration
    the benchmark times): one step from a random state; sampled sites
    recomputed by the oracle from their 3x3 neighbourhoods."""
    w = W.steady()
    rng = np.random.default_rng(17)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=23, dtype=np.float32)
    got = _run(torch_cuda, w, S0, 1)
    pts = [(0, 0), (w.nz - 1, w.nx - 1), (w.nz - 1, 0), (0, w.nx - 1), (w.nz // 2, w.nx // 2)] + \
          [tuple(rng.integers(0, [w.nz, w.nx])) for _ in range(27)]
    for z, x in pts:
        z0, z1 = max(z - 1, 0), min(z + 2, w.nz)
        x0, x1 = max(x - 1, 0), min(x + 2, w.nx)
        sub = w.crop(z0, z1, x0, x1)
        sub.bc = tuple(w.bc[k] if edge else 0 for k, edge in
                       enumerate([z1 == w.nz, z0 == 0, x0 == 0, x1 == w.nx]))
        ref = oracle_problem(orc, sub).step(S0[z0:z1, x0:x1].astype(np.float64))[z - z0, x - x0]
        assert rel_err_I(got[z, x], ref) < TOL_I, (z, x)
        assert abs_err_dop(got[z, x], ref) < TOL_DOP, (z, x)


def test_tf32x3_refuses_n64(torch_cuda):
    from paper_2609_23057_b300 import _lib
    from paper_2609_23057_b300.solver import Solver
    with pytest.raises(_lib.RtlbError) as ei:
        Solver(64, 4, 8, 8, precision="tf32x3")
    assert ei.value.status == 11
