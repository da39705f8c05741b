"""GPU parity of the FP8 block-scaled tensor-core form (precision "fp8").

The oracle's orc_step_fp8 writes the form out in float64 from its definition
(e4m3 rounding, UE8M0 block scales, the float32 roundings of S~ and beta S~
before quantization).  The quantization decisions are taken from the same
float32 values on both sides, so one step must agree up to the tensor core's
float32 accumulation and the float32 part alpha S~ (a few float32 roundings of
entries of size <= max|S|): 1e-5 of the peak.  One e4m3 code taken
differently would move an entry by ~2^-4 of one product, far above that.

Tiles that mix phase classes run on the CUDA-core float32 kernel; the
full-size test takes each output direction's reference from the tile of the
site it streamed from.  All calls go through the C ABI.
"""
import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import oracle_problem

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _step(torch, w, prec, S0, steps=1):
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
                                                    (67, 5, 2, 4, 1), (512, 128, 2, 4, 2)])
def test_fp8_one_step_matches_the_fp8_form(torch_cuda, orc, nx, nz, nzen, naz, n_phase):
    """Single-class 128-site tiles (rows of 128-multiple width alternate class,
    or one class with a ragged last tile), emission, polarized inflow on top,
    periodic sides; a random state; one step.  512x128 at n = 8 gives every
    CTA several tiles, where a converter group without a slot (n = 8) must
    not run ahead of the other."""
    w = W.random_medium(nx, nz, nzen, naz, seed=nx + nz + naz, bc=(2, 0, 1, 1), n_phase=n_phase, steps=1)
    w.phase_index = (np.arange(nz)[:, None] % n_phase * np.ones((1, nx))).astype(np.uint8)
    S0 = W.random_state(nz, nx, w.n, seed=9, dtype=np.float32)
    ref = oracle_problem(orc, w).step_fp8(S0.astype(np.float64))
    got = _step(torch_cuda, w, "fp8", S0)
    assert _rel(got, ref) < TOL
    # and the form is a real approximation of the FP64 step, not a copy of it
    plain = oracle_problem(orc, w).step(S0.astype(np.float64))
    assert _rel(got, plain) > 10 * TOL


def _tile_pure(cls_flat, kTile=128):
    ntiles = (cls_flat.size + kTile - 1) // kTile
    pure = np.ones(ntiles, bool)
    for t in range(ntiles):
        seg = cls_flat[t * kTile:(t + 1) * kTile]
        pure[t] = np.all(seg == seg[0])
    return pure


def test_fp8_full_size_sampled_sites(torch_cuda, orc):
    """2048x2048, n = 64 (the precision workload's medium, two classes), one
    step from a random state in the launch configuration the benchmark times.
    Each sampled site is recomputed from its 3x3 neighbourhood by the FP8 form
    and by the float32-exact step; direction d takes the one matching the tile
    (pure -> FP8, mixed -> CUDA-core float32) of the site it came from."""
    w = W.precision(steps=1)
    rng = np.random.default_rng(11)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=29, dtype=np.float32)
    got = _step(torch_cuda, w, "fp8", S0)
    cls = np.zeros((w.nz, w.nx), np.uint8) if w.phase_index is None else np.asarray(w.phase_index)
    pure = _tile_pure(cls.ravel())
    P0 = oracle_problem(orc, w)
    cx, cz = P0.cx, P0.cz
    pts = [(0, 0), (w.nz - 1, w.nx - 1), (w.nz - 1, 0), (0, w.nx - 1), (w.nz // 2, w.nx // 2),
           (1, 1), (w.nz - 2, 5)] + [tuple(rng.integers(0, [w.nz, w.nx])) for _ in range(17)]
    n_pure = n_mixed = 0
    for z, x in pts:
        z0, z1 = max(z - 1, 0), min(z + 2, w.nz)
        x0, x1 = max(x - 1, 0), min(x + 2, w.nx)
        sub = w.crop(z0, z1, x0, x1)
        sub.bc = tuple(w.bc[k] if edge else 0 for k, edge in
                       enumerate([z1 == w.nz, z0 == 0, x0 == 0, x1 == w.nx]))
        Psub = oracle_problem(orc, sub)
        Sin = S0[z0:z1, x0:x1].astype(np.float64)
        r8 = Psub.step_fp8(Sin)[z - z0, x - x0]
        r32 = Psub.step(Sin)[z - z0, x - x0]
        ref = np.empty_like(r8)
        for d in range(w.n):
            zs, xs = z - cz[d], x - cx[d]
            if 0 <= zs < w.nz and 0 <= xs < w.nx and pure[(zs * w.nx + xs) // 128]:
                ref[d] = r8[d]
                n_pure += 1
            else:
                ref[d] = r32[d]          # mixed tile, or a ghost value (same in both)
                n_mixed += 1
        g = got[z, x]
        assert np.abs(g - ref).max() <= TOL * max(np.abs(S0).max(), 1e-30), (z, x)
    assert n_pure > 0


def test_fp8_rejects_too_many_classes(torch_cuda):
    """n = 64 keeps every class's table scales in tensor memory: 12 classes
    fit, 13 do not (RTLB_E_UNSUPPORTED from set_medium)."""
    from paper_2609_23057_b300 import _lib
    from paper_2609_23057_b300.solver import solver_for

    def medium(k):
        w = W.random_medium(128, 2, 8, 8, seed=1, n_phase=1, steps=1)
        w.phase_specs = [("hg", 0.05 * c, -0.1) for c in range(k)]
        w.phase_index = (np.arange(w.nx * w.nz) % k).reshape(w.nz, w.nx).astype(np.uint8)
        return w

    with pytest.raises(_lib.RtlbError) as ei:
        solver_for(medium(13), "fp8")
    assert ei.value.status == 11
    solver_for(medium(12), "fp8").close()
