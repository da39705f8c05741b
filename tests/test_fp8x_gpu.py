"""GPU parity and accuracy of the split FP8 tensor-core form ("fp8x").

Two checks, against two references:
- the form itself: orc_step_fp8x writes the split quantization out in float64
  (state operand in two e4m3 terms, table in three, five products kept).  Both
  sides take every quantization decision from the same float32 values, so one
  step agrees up to the tensor core's float32 accumulation: 1e-5 of the peak,
  as for the single-term FP8 form;
- the paper's method: orc_step, the FP64 step, on the 256x256 crop of the
  2048x2048, n = 64 cloud workload for 1000 steps.  The split form meets the
  1e-3 relative error on the top radiance and on its degree of polarization
  that the single-term form misses by 50x.
All calls go through the C ABI.
"""
import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import abs_err_dop, oracle_problem, rel_err_I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _run(torch, w, prec, S0, steps=1):
    from paper_2609_23057_b300.solver import solver_for
    s = solver_for(w, prec)
    s.set_state(torch.from_numpy(np.asarray(S0, np.float32)).cuda())
    s.step(steps)
    s.total_intensity()                       # surfaces a device-side timeout as an error
    got = s.get_state().cpu().numpy().astype(np.float64)
    s.close()
    return got


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("nx,nz,nzen,naz,n_phase", [(256, 8, 2, 4, 2), (256, 8, 4, 4, 2), (384, 6, 4, 8, 2),
                                                    (256, 4, 8, 8, 2), (130, 3, 4, 8, 1), (200, 7, 8, 8, 1),
                                                    (67, 5, 2, 4, 1), (512, 128, 2, 4, 2), (1024, 16, 8, 8, 2)])
def test_fp8x_one_step_matches_the_split_form(torch_cuda, orc, nx, nz, nzen, naz, n_phase):
    """Single-class 128-site tiles (rows alternate class, or one class with a
    ragged last tile), emission, polarized inflow on top, periodic sides; a
    random state; one step.  512x128 at n = 8 and 1024x16 at n = 64 give every
    CTA several tiles."""
    w = W.random_medium(nx, nz, nzen, naz, seed=nx + nz + naz, bc=(2, 0, 1, 1), n_phase=n_phase, steps=1)
    w.phase_index = (np.arange(nz)[:, None] % n_phase * np.ones((1, nx))).astype(np.uint8)
    S0 = W.random_state(nz, nx, w.n, seed=9, dtype=np.float32)
    P = oracle_problem(orc, w)
    ref = P.step_fp8x(S0.astype(np.float64))
    got = _run(torch_cuda, w, "fp8x", S0)
    assert _rel(got, ref) < TOL
    # a real approximation of the FP64 step, far closer than single e4m3
    plain = P.step(S0.astype(np.float64))
    single = P.step_fp8(S0.astype(np.float64))
    assert 0 < _rel(got, plain) < 0.1 * _rel(single, plain)


def test_fp8x_full_size_sampled_sites(torch_cuda, orc):
    """2048x2048, n = 64 (the benchmark's launch configuration), one step from
    a random state; sampled sites recomputed by the form's emulation from their
    3x3 neighbourhoods (mixed-class tiles run on the float32 CUDA-core
    kernel: those directions take the FP64 step)."""
    from test_fp8_gpu import _tile_pure
    w = W.precision(steps=1)
    rng = np.random.default_rng(13)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=31, dtype=np.float32)
    got = _run(torch_cuda, w, "fp8x", S0)
    cls = np.zeros((w.nz, w.nx), np.uint8) if w.phase_index is None else np.asarray(w.phase_index)
    pure = _tile_pure(cls.ravel())
    P0 = oracle_problem(orc, w)
    cx, cz = P0.cx, P0.cz
    pts = [(0, 0), (w.nz - 1, w.nx - 1), (w.nz - 1, 0), (0, w.nx - 1), (w.nz // 2, w.nx // 2),
           (1, 1), (w.nz - 2, 5)] + [tuple(rng.integers(0, [w.nz, w.nx])) for _ in range(17)]
    n_pure = 0
    for z, x in pts:
        z0, z1 = max(z - 1, 0), min(z + 2, w.nz)
        x0, x1 = max(x - 1, 0), min(x + 2, w.nx)
        sub = w.crop(z0, z1, x0, x1)
        sub.bc = tuple(w.bc[k] if edge else 0 for k, edge in
                       enumerate([z1 == w.nz, z0 == 0, x0 == 0, x1 == w.nx]))
        Psub = oracle_problem(orc, sub)
        Sin = S0[z0:z1, x0:x1].astype(np.float64)
        r8 = Psub.step_fp8x(Sin)[z - z0, x - x0]
        r32 = Psub.step(Sin)[z - z0, x - x0]
        ref = np.empty_like(r8)
        for d in range(w.n):
            zs, xs = z - cz[d], x - cx[d]
            if 0 <= zs < w.nz and 0 <= xs < w.nx and pure[(zs * w.nx + xs) // 128]:
                ref[d] = r8[d]
                n_pure += 1
            else:
                ref[d] = r32[d]
        assert np.abs(got[z, x] - ref).max() <= TOL * max(np.abs(S0).max(), 1e-30), (z, x)
    assert n_pure > 0


def test_fp8_forms_against_the_fp64_step_1000_steps(torch_cuda, orc, crop_ref_1000):
    """The 256x256 crop [896,1152)^2 of the 2048x2048, n = 64 medium, 1000
    steps from zero, against the FP64 oracle step (elementwise over the top
    radiance, entries below 1e-3 of the maximum compared against that floor).
    The split form meets 1e-3 on I and on the degree of polarization.  The
    single-term form is held to its measured error budget (5.6e-2 on I and
    4.2e-2 on the degree of polarization after 200 steps; the e4m3 table alone
    accounts for ~5e-2 in a CPU emulation): below 8e-2 and 6e-2, so that a
    regression of that form shows even though it misses 1e-3."""
    w, P, ref, top_ref = crop_ref_1000
    S0 = np.zeros((w.nz, w.nx, w.n, 4))
    for prec, tol_i, tol_p in (("fp8x", 1e-3, 1e-3), ("fp8", 8e-2, 6e-2)):
        got = _run(torch_cuda, w, prec, S0, w.steps)
        top = P.radiance_out(got, orc.SIDE_TOP)
        assert rel_err_I(top, top_ref, floor_frac=1e-3) < tol_i, prec
        assert abs_err_dop(top, top_ref, floor_frac=1e-3) < tol_p, prec


def test_fp8x_rejects_too_many_classes(torch_cuda):
    """n = 64 keeps the table scales of three terms per class in tensor
    memory beside the two state terms: two classes fit, three do not."""
    from paper_2609_23057_b300 import _lib
    from paper_2609_23057_b300.solver import solver_for

    def medium(k):
        w = W.random_medium(128, 2, 8, 8, seed=1, n_phase=1, steps=1)
        w.phase_specs = [("hg", 0.05 * c, -0.1) for c in range(k)]
        w.phase_index = (np.arange(w.nx * w.nz) % k).reshape(w.nz, w.nx).astype(np.uint8)
        return w

    with pytest.raises(_lib.RtlbError) as ei:
        solver_for(medium(3), "fp8x")
    assert ei.value.status == 11
    solver_for(medium(2), "fp8x").close()
