"""GPU parity of the float32 fused step (CUDA cores) with the FP64 oracle.

Tolerances: 1e-5 relative on I (elementwise, entries below 1e-6 of the
maximum compared against that floor) and 1e-5 absolute on the degree of
polarization.  All calls go through the C ABI (librtlb.so)."""
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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _solver(w, precision="fp32"):
    from paper_2609_23057_b300.solver import solver_for
    return solver_for(w, precision)


def _state(s):
    return s.get_state().cpu().numpy().astype(np.float64)


def test_small_lattice_200_steps(torch_cuda, orc):
    """32x32, n = 8, tau 0.05, albedo 0.9, Rayleigh, emission 1e-3, top beam,
    200 steps (linear survival)."""
    w = W.small()
    ref = oracle_problem(orc, w).run(np.zeros((w.nz, w.nx, w.n, 4)), w.steps)
    s = _solver(w)
    s.step(w.steps)
    got = _state(s)
    assert rel_err_I(got, ref) < TOL_I
    assert abs_err_dop(got, ref) < TOL_DOP
    top = s.radiance_out("top").cpu().numpy()
    ref_top = oracle_problem(orc, w).radiance_out(ref, orc.SIDE_TOP)
    assert rel_err_I(top, ref_top) < TOL_I


CASES = [
    # nx, nz, n_zen, n_az, bc, n_phase, seed
    (37, 23, 2, 4, (2, 0, 0, 0), 2, 1),
    (129, 5, 4, 4, (2, 2, 2, 2), 3, 2),
    (64, 33, 4, 8, (1, 1, 1, 1), 2, 3),
    (70, 9, 8, 8, (2, 0, 1, 1), 4, 4),
    (3, 200, 8, 8, (0, 0, 0, 0), 1, 5),
    (1, 1, 4, 8, (2, 2, 2, 2), 2, 6),
    (17, 11, 3, 4, (2, 1, 2, 1)[:0] + (2, 0, 1, 1), 2, 7),   # n = 12: generic kernel
    (25, 13, 3, 5, (1, 1, 0, 0), 2, 8),                       # n = 15, odd zenith count (rest)
]


@pytest.mark.parametrize("nx,nz,nzen,naz,bc,nph,seed", CASES)
def test_random_media(torch_cuda, orc, nx, nz, nzen, naz, bc, nph, seed):
    """Odd sizes and ragged tiles, mixed phase classes within a tile, every
    boundary kind, polarized random initial state, 4 steps."""
    w = W.random_medium(nx, nz, nzen, naz, seed=seed, bc=bc, n_phase=nph, steps=4)
    S0 = W.random_state(nz, nx, w.n, seed=seed + 100)
    ref = oracle_problem(orc, w).run(S0, w.steps)
    s = _solver(w)
    s.set_state(torch_cuda.from_numpy(S0.astype(np.float32)).cuda())
    s.step(w.steps)
    got = _state(s)
    assert rel_err_I(got, ref) < TOL_I
    assert abs_err_dop(got, ref) < TOL_DOP
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    for side in range(4):
        ro = s.radiance_out(side).cpu().numpy()
        rr = oracle_problem(orc, w).radiance_out(ref, side)
        assert np.abs(ro - rr).max() <= 1e-5 * max(np.abs(rr).max(), 1e-30)
        # degree of polarization of the leaving radiance (Eq. 36), on entries
        # whose I is above 1e-6 of the side's maximum (zero elsewhere)
        dp = s.dop_out(side).cpu().numpy().astype(np.float64)
        mask = rr[..., 0] > 1e-6 * max(np.abs(rr[..., 0]).max(), 1e-300)
        assert np.abs(dp - orc.dop(rr))[mask].max(initial=0.0) < TOL_DOP
        assert np.all(dp[rr[..., 0] == 0] == 0)


def test_steady_state_small(torch_cuda, orc):
    """run_to_steady on a 24x16 cloud medium (n = 32): converges, takes about
    as many steps as the oracle's own iteration, and the state equals the
    oracle's after the same number of steps."""
    w = W.cloud("cloud24x16", 24, 16, 4, 8, seed=0, steps=0)
    P = oracle_problem(orc, w)
    _, t_ref, _ = P.run_to_steady(P.zero_state(), 1e-6, 20000)
    s = _solver(w)
    steps, res, ok = s.run_to_steady(1e-6, 20000, check_every=1)
    assert ok and res < 1e-6
    assert abs(steps - t_ref) <= max(3, 0.02 * t_ref)
    ref = P.run(P.zero_state(), steps)
    got = _state(s)
    assert rel_err_I(got, ref) < TOL_I
    assert abs_err_dop(got, ref) < TOL_DOP


def test_steady_state_lattice512_crop128(torch_cuda, orc):
    """run_to_steady (residual < 1e-6, cap 4000, checked every step) on the
    128x128 centre crop of the 512x512, n = 32 steady-state medium, run as its
    own problem: the step count within 2 % of the oracle's own iteration, and
    the state after those steps within 1e-5 of the oracle's."""
    w = W.steady().crop(192, 320, 192, 320)
    P = oracle_problem(orc, w)
    _, t_ref, r_ref = P.run_to_steady(P.zero_state(), 1e-6, 4000)
    assert r_ref < 1e-6
    s = _solver(w)
    steps, res, ok = s.run_to_steady(1e-6, 4000, check_every=1)
    assert ok and res < 1e-6
    assert abs(steps - t_ref) <= max(2, 0.02 * t_ref)
    ref = P.run(P.zero_state(), steps)
    got = _state(s)
    s.close()
    assert rel_err_I(got, ref) < TOL_I
    assert abs_err_dop(got, ref) < TOL_DOP


def test_residual_and_total_intensity(torch_cuda, orc):
    w = W.random_medium(40, 30, 4, 4, seed=9, steps=1)
    S0 = W.random_state(30, 40, 16, seed=10)
    P = oracle_problem(orc, w)
    S1 = P.step(S0)
    s = _solver(w)
    s.set_state(S0.astype(np.float32))           # host pointer path
    s.step(1)
    r = s.last_residual()
    assert r == pytest.approx(orc.residual(S0, S1), rel=1e-5)
    assert s.total_intensity() == pytest.approx(S1[..., 0].sum(), rel=1e-6)
    host = np.zeros((30, 40, 16, 4), np.float32)
    s._check(__import__("paper_2609_23057_b300._lib", fromlist=["lib"]).lib().rtlb_get_state(
        s._ctx, host.ctypes.data, None))
    assert np.array_equal(host, s.get_state().cpu().numpy())


def test_full_size_sampled_sites(torch_cuda, orc):
    """2048x2048, n = 64 (the measured workload, same launch configuration):
    one step from a random state, then the oracle computes sampled outputs one
    by one from the 3x3 neighbourhood of each sampled site."""
    w = W.precision(steps=1)
    rng = np.random.default_rng(0)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=21, dtype=np.float32)
    s = _solver(w)
    s.set_state(torch_cuda.from_numpy(S0).cuda())
    s.step(1)
    got = s.get_state().cpu().numpy()
    pts = [(0, 0), (w.nz - 1, w.nx - 1), (w.nz - 1, 0), (0, w.nx - 1), (w.nz // 2, w.nx // 2),
           (w.nz // 2 - 1, 7)] + [tuple(rng.integers(0, [w.nz, w.nx])) for _ in range(26)]
    for z, x in pts:
        z0, z1 = max(z - 1, 0), min(z + 2, w.nz)
        x0, x1 = max(x - 1, 0), min(x + 2, w.nx)
        # boundary kinds only matter where the window touches the lattice edge
        bc = tuple(w.bc[k] if edge else 0 for k, edge in
                   enumerate([z1 == w.nz, z0 == 0, x0 == 0, x1 == w.nx]))
        sub = w.crop(z0, z1, x0, x1)
        sub.bc = bc
        ref = oracle_problem(orc, sub).step(S0[z0:z1, x0:x1].astype(np.float64))
        g = got[z, x].astype(np.float64)
        r = ref[z - z0, x - x0]
        assert rel_err_I(g, r) < TOL_I, (z, x)
        assert abs_err_dop(g, r) < TOL_DOP, (z, x)


def test_error_codes(torch_cuda):
    from paper_2609_23057_b300 import _lib
    from paper_2609_23057_b300.solver import Solver, phase_rayleigh
    s = Solver(8, 8, 2, 4)
    with pytest.raises(_lib.RtlbError) as ei:
        s.step(1)
    assert ei.value.status == 5                              # step before set_medium
    Z = phase_rayleigh(2, 4)
    tau = np.full((8, 8), 0.1, np.float32)
    alb = np.full((8, 8), 0.5, np.float32)
    s.set_medium(tau, alb, Z)
    bad = alb.copy()
    bad[3, 3] = 1.5
    with pytest.raises(_lib.RtlbError) as ei:
        s.set_medium(tau, bad, Z)
    assert ei.value.status == 3
    bad = tau.copy()
    bad[0, 0] = np.nan
    with pytest.raises(_lib.RtlbError) as ei:
        s.set_medium(bad, alb, Z)
    assert ei.value.status == 8
    big = np.full((8, 8), 5.0, np.float32)                  # linear survival: albedo*tau > 1
    with pytest.raises(_lib.RtlbError) as ei:
        s.set_medium(big, alb, Z)
    assert ei.value.status == 3
    with pytest.raises(_lib.RtlbError) as ei:
        s.set_medium(tau, alb, Z, phase_index=np.full((8, 8), 2, np.uint8))
    assert ei.value.status == 3
    s.set_boundary("left", "periodic")
    with pytest.raises(_lib.RtlbError) as ei:
        s.step(1)
    assert ei.value.status == 5                              # unpaired periodic side
    s.set_boundary("right", "periodic")
    s.step(2)                                                # the context is still usable
    assert s.steps_done == 2
    with pytest.raises(_lib.RtlbError) as ei:
        s.set_boundary("top", "inflow", None)
    assert ei.value.status == 1


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_table_variants(torch_cuda, orc, prec):
    """Depolarized Rayleigh (rho = 0.0279) and the intensity-conserving
    correction of an HG table: the library's own tables, run on the GPU,
    against the oracle's tables and step."""
    from paper_2609_23057_b300 import solver as SV
    w = W.random_medium(150, 8, 4, 8, seed=13, bc=(2, 0, 1, 1), n_phase=2, steps=4)
    w.phase_index = (np.arange(w.nz)[:, None] % 2 * np.ones((1, w.nx))).astype(np.uint8)
    mu, phi = orc.direction_grid(4, 8)
    Zo = np.stack([orc.phase_table_spec(mu, phi, ("rayleigh", 0.0279)),
                   orc.conserve_intensity(orc.phase_table_spec(mu, phi, ("hg", 0.85, -0.1)))])
    Zl = np.stack([SV.phase_rayleigh(4, 8, depol=0.0279),
                   SV.conserve_intensity(SV.phase_hg(4, 8, 0.85, -0.1))])
    P = orc.Problem(w.nx, w.nz, mu, phi, w.tau, w.albedo, w.emission, w.phase_index.astype(np.int32), Zo,
                    surv_mode=w.surv_mode, bc=w.bc, inflow=w.inflow)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=14)
    ref = P.run(S0, w.steps)
    s = SV.Solver(w.nx, w.nz, 4, 8, precision=prec, survival="exp")
    s.set_medium(w.tau.astype(np.float32), w.albedo.astype(np.float32), Zl,
                 emission=w.emission.astype(np.float32), phase_index=w.phase_index)
    for side in range(4):
        s.set_boundary(side, w.bc[side], w.inflow[side] if w.bc[side] == 2 else None)
    s.set_state(torch_cuda.from_numpy(S0.astype(np.float32)).cuda())
    s.step(w.steps)
    s.total_intensity()
    got = s.get_state().cpu().numpy().astype(np.float64)
    s.close()
    tol = TOL_I if prec == "fp32" else 5e-5
    assert rel_err_I(got, ref) < tol
    assert abs_err_dop(got, ref) < tol
