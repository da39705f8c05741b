"""GPU parity of semi-Lagrangian bilinear streaming (Eq. 33-38) with the FP64
oracle, through the C ABI: the collision pass of every precision followed by
the four-tap gather, on both lattice planes and every boundary kind, the
transposed gather of the adjoint, and sampled sites of the 2048x2048, n = 64
workload in the benchmark's launch configuration.

Tolerances as for the nearest-offset scheme: the gather is a convex
combination (weights sum to one), so it adds at most a few float32 roundings
per step: 1e-5 relative for the float32 path; the tensor-core forms keep
their own bounds (bf16: ~2u per step on the scattered part)."""
import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import abs_err_dop, oracle_problem, rel_err_I

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -9
TOL_TC = {"bf16": 1e-2, "bf16x2": 1e-2, "bf16x3": 5e-5}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _run(torch, w, prec, S0, steps, sides=()):
    from paper_2609_23057_b300.solver import solver_for
    s = solver_for(w, prec)
    s.set_state(torch.from_numpy(np.asarray(S0, np.float32)).cuda())
    s.step(steps)
    s.total_intensity()
    got = s.get_state().cpu().numpy().astype(np.float64)
    outs = [s.radiance_out(side).cpu().numpy().astype(np.float64) for side in sides]
    s.close()
    return got, outs


CASES = [
    (37, 23, 2, 4, (2, 0, 1, 1), "xz", 2),
    (64, 17, 4, 8, (1, 1, 2, 0), "xy", 2),
    (5, 3, 4, 4, (2, 2, 2, 2), "xz", 1),
    (1, 2, 2, 4, (1, 1, 1, 1), "xy", 1),     # lattice narrower than the taps' reach
    (2, 1, 3, 6, (1, 1, 1, 1), "xz", 1),
    (130, 9, 8, 8, (2, 0, 0, 0), "xz", 2),
    (33, 31, 4, 4, (0, 0, 0, 0), "xy", 3),
]


@pytest.mark.parametrize("nx,nz,nzen,naz,bc,plane,nph", CASES)
def test_fp32_random_media(torch_cuda, orc, nx, nz, nzen, naz, bc, plane, nph):
    w = W.random_medium(nx, nz, nzen, naz, seed=nx * 7 + nz, bc=bc, n_phase=nph, steps=6)
    w.scheme, w.plane = "bilinear", plane
    S0 = W.random_state(nz, nx, w.n, seed=nx + 3)
    P = oracle_problem(orc, w)
    ref = P.run(S0, w.steps)
    got, outs = _run(torch_cuda, w, "fp32", S0, w.steps, sides=range(4))
    assert rel_err_I(got, ref) < 1e-5
    assert abs_err_dop(got, ref) < 1e-5
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    for side, ro in enumerate(outs):
        rr = P.radiance_out(ref, side)
        assert np.abs(ro - rr).max() <= 1e-5 * max(np.abs(rr).max(), 1e-30)


@pytest.mark.parametrize("nzen,naz", [(2, 4), (4, 4), (4, 8), (8, 8)])
@pytest.mark.parametrize("prec", ["bf16", "bf16x2", "bf16x3"])
def test_tensor_core_forms(torch_cuda, orc, nzen, naz, prec):
    if prec == "bf16x3" and nzen * naz == 64:
        pytest.skip("split operands for n = 64 exceed shared memory")
    w = W.random_medium(256, 6, nzen, naz, seed=nzen * naz, bc=(2, 0, 1, 1), n_phase=2, steps=3)
    w.phase_index = (np.arange(w.nz)[:, None] % 2 * np.ones((1, w.nx))).astype(np.uint8)
    w.scheme, w.plane = "bilinear", "xz"
    S0 = W.random_state(w.nz, w.nx, w.n, seed=9)
    ref = oracle_problem(orc, w).run(S0, w.steps)
    got, _ = _run(torch_cuda, w, prec, S0, w.steps)
    assert rel_err_I(got, ref) < TOL_TC[prec]
    assert abs_err_dop(got, ref) < TOL_TC[prec]


def test_offset_azimuths_on_the_horizontal_lattice(torch_cuda, orc):
    """Table 1's azimuth set offset by 22.5 deg (no nearest D2Q9 offset
    exists) on the paper's 16x16 horizontal lattice, recycling boundaries,
    central source, 64 steps."""
    from paper_2609_23057_b300.solver import Solver, phase_rayleigh
    mu = np.array([-0.5] * 4 + [0.5] * 4)
    phi = np.radians([22.5, 112.5, 202.5, 292.5] * 2)
    nx = nz = 16
    tau = np.full((nz, nx), np.float32(2.5 / 16))
    alb = np.full((nz, nx), np.float32(0.2))
    em = np.zeros((nz, nx), np.float32)
    em[7:9, 7:9] = np.float32(1 / 16 / 8)
    Zo = orc.phase_table(mu, phi)
    P = orc.Problem(nx, nz, mu, phi, tau, alb, em, None, Zo, bc=(1, 1, 1, 1), scheme="bilinear",
                    plane=orc.PLANE_XY)
    ref = P.run(P.zero_state(), 64)
    s = Solver(nx, nz, 2, 4, mu=mu, phi=phi, streaming="bilinear", plane="xy")
    s.set_medium(tau, alb, phase_rayleigh(2, 4, mu, phi)[None], emission=em)
    for side in range(4):
        s.set_boundary(side, "periodic")
    s.step(64)
    got = s.get_state().cpu().numpy().astype(np.float64)
    s.close()
    assert rel_err_I(got, ref) < 1e-5
    assert abs_err_dop(got, ref) < 1e-5


@pytest.mark.parametrize("plane,bc", [("xz", (2, 0, 0, 0)), ("xy", (1, 1, 2, 0))])
def test_adjoint(torch_cuda, orc, plane, bc):
    from paper_2609_23057_b300.solver import solver_for
    w = W.random_medium(19, 11, 4, 4, seed=61, bc=bc, n_phase=2, steps=10, surv_mode=1)
    w.tau = np.minimum(w.tau, 0.9)
    w.scheme, w.plane = "bilinear", plane
    P = oracle_problem(orc, w)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=4)
    seed = np.random.default_rng(5).standard_normal((w.nx, w.n, 4)).astype(np.float32).astype(np.float64)
    rt, ra, rZ, rS = P.adjoint(S0, w.steps, seed, want_S0=True)
    s = solver_for(w, "fp32")
    s.set_state(torch_cuda.from_numpy(S0.astype(np.float32)).cuda())
    gt, ga, gZ, gS = s.adjoint(w.steps, torch_cuda.from_numpy(seed.astype(np.float32)).cuda(), checkpoint_every=4,
                               want_S0=True)
    SN = s.get_state().cpu().numpy()
    s.close()
    rel = lambda a, b: float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300))
    assert rel(gt.cpu().numpy(), rt) < 1e-4
    assert rel(ga.cpu().numpy(), ra) < 1e-4
    assert rel(gZ, rZ) < 1e-4
    assert rel(gS.cpu().numpy(), rS) < 1e-4
    assert rel(SN, P.run(S0, w.steps)) < 1e-5


@pytest.mark.parametrize("prec", ["fp32", "bf16x2"])
def test_full_size_sampled_sites(torch_cuda, orc, prec):
    """2048x2048, n = 64, one step from a random state; each sampled site is
    recomputed by the oracle from its 5x5 neighbourhood (the taps reach two
    cells)."""
    w = W.precision(steps=1)
    w.scheme = "bilinear"
    rng = np.random.default_rng(3)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=23, dtype=np.float32)
    from paper_2609_23057_b300.solver import solver_for
    s = solver_for(w, prec)
    s.set_state(torch_cuda.from_numpy(S0).cuda())
    s.step(1)
    s.total_intensity()
    got = s.get_state().cpu().numpy()
    s.close()
    pts = [(0, 0), (w.nz - 1, w.nx - 1), (w.nz - 1, 0), (0, w.nx - 1), (w.nz // 2, w.nx // 2),
           (1, 1), (w.nz - 2, 5)] + [tuple(rng.integers(0, [w.nz, w.nx])) for _ in range(17)]
    tol = 1e-5 if prec == "fp32" else 2 * 2 * U_BF16
    for z, x in pts:
        z0, z1 = max(z - 2, 0), min(z + 3, w.nz)
        x0, x1 = max(x - 2, 0), min(x + 3, w.nx)
        sub = w.crop(z0, z1, x0, x1)
        sub.bc = tuple(w.bc[k] if edge else 0 for k, edge in
                       enumerate([z1 == w.nz, z0 == 0, x0 == 0, x1 == w.nx]))
        ref = oracle_problem(orc, sub).step(S0[z0:z1, x0:x1].astype(np.float64))
        g, r = got[z, x].astype(np.float64), ref[z - z0, x - x0]
        assert rel_err_I(g, r) < tol, (z, x)
        if prec == "fp32":
            assert abs_err_dop(g, r) < 1e-5, (z, x)


def _settle_each_step(s, w):
    """Re-set one boundary to its own kind: the library then ends the
    deferred streaming of the last step with the gather kernel, so the next
    step loads a state, as in the two-pass form."""
    inflow = None if w.inflow is None else w.inflow[0]
    s.set_boundary(0, w.bc[0], inflow if w.bc[0] == 2 else None)


@pytest.mark.parametrize("prec,nzen,naz,mixed,bc,nx,nz", [("bf16", 4, 4, False, (2, 0, 1, 1), 256, 7),
                                                           ("bf16x2", 4, 8, True, (2, 0, 1, 1), 256, 7),
                                                           ("bf16x3", 4, 8, False, (2, 2, 0, 0), 256, 7),
                                                           ("bf16", 4, 8, True, (0, 0, 0, 0), 256, 7),
                                                           ("bf16x2", 4, 4, False, (1, 1, 2, 0), 256, 6),
                                                           ("bf16", 4, 8, False, (1, 1, 1, 1), 128, 3)])
def test_gather_form_equals_two_pass(torch_cuda, prec, nzen, naz, mixed, bc, nx, nz):
    """The gather form (each step gathers the previous step's P while
    loading: the tensor-core bf16 forms at n in {16, 32} with nx % 128 == 0)
    against the two-pass form (collision pass, then the gather kernel) on the
    same inputs: identical bits for the state, the readouts, the residual and
    a following adjoint.  Boundaries: top inflow, periodic x, vacuum bottom
    (ghost values written into the staged windows), inflow top and bottom,
    all vacuum (the TMA's zero fill), periodic z with inflow on the left, and
    periodic on both axes on a lattice one tile wide and three rows high
    (every tile an edge tile, windows wrapping on both sides); `mixed` puts a
    class boundary inside tiles (those tiles run on the CUDA-core kernel, also
    gathering)."""
    from paper_2609_23057_b300.solver import solver_for
    w = W.random_medium(nx, nz, nzen, naz, seed=nzen * naz + 5, bc=bc, n_phase=2, steps=5)
    if mixed:
        w.phase_index = ((np.arange(w.nx)[None, :] >= 100) * np.ones((w.nz, 1))).astype(np.uint8)
    else:
        w.phase_index = (np.arange(w.nz)[:, None] % 2 * np.ones((1, w.nx))).astype(np.uint8)
    w.scheme, w.plane = "bilinear", "xz"
    S0 = torch_cuda.from_numpy(W.random_state(w.nz, w.nx, w.n, seed=2, dtype=np.float32)).cuda()
    seed = torch_cuda.from_numpy(np.random.default_rng(8).standard_normal((w.nx, w.n, 4)).astype(np.float32)).cuda()
    res = []
    for settle in (False, True):
        s = solver_for(w, prec)
        assert s.gather_form
        assert (s.mixed_tiles > 0) == mixed
        s.set_state(S0)
        for _ in range(w.steps):
            s.step(1)
            if settle:
                _settle_each_step(s, w)
        st = s.get_state().cpu().numpy()
        top = s.radiance_out(0).cpu().numpy()
        dop = s.dop_out(0).cpu().numpy()
        r = s.last_residual()
        tot = s.total_intensity()
        s.step(2)
        st2 = s.get_state().cpu().numpy()
        gt, ga, gZ, _ = s.adjoint(3, seed, checkpoint_every=2)
        res.append((st, top, dop, r, tot, st2, gt.cpu().numpy(), ga.cpu().numpy(), gZ))
        s.close()
    a, b = res
    for k in range(len(a)):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def test_run_to_steady_gather_form(torch_cuda, orc):
    """run_to_steady through the gather form (residual between two gathered
    states, bf16x3 at n = 16) against the oracle: the same step count within
    one, the final state within the form's bound."""
    from paper_2609_23057_b300.solver import solver_for
    w = W.random_medium(128, 12, 4, 4, seed=77, bc=(2, 0, 1, 1), n_phase=1, steps=1)
    w.scheme, w.plane = "bilinear", "xz"
    P = oracle_problem(orc, w)
    s = solver_for(w, "bf16x3")
    assert s.gather_form
    taken, r, ok = s.run_to_steady(1e-6, 2000, check_every=1)
    got = s.get_state().cpu().numpy().astype(np.float64)
    s.close()
    ref, rtaken, _ = P.run_to_steady(P.zero_state(), 1e-6, 2000)
    assert ok and abs(taken - rtaken) <= 0.02 * rtaken + 1
    assert rel_err_I(got, ref) < TOL_TC["bf16x3"]


def test_batch_rejects_bilinear_channels(torch_cuda):
    from paper_2609_23057_b300 import _lib
    from paper_2609_23057_b300.solver import Batch, solver_for
    w = W.random_medium(128, 4, 2, 4, seed=1, n_phase=1, steps=1)
    w.scheme = "bilinear"
    s = solver_for(w, "bf16")
    with pytest.raises(_lib.RtlbError) as ei:
        Batch([s])
    assert ei.value.status == 11
    s.close()
