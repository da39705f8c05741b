"""GPU adjoint (rtlb_adjoint) against the FP64 oracle adjoint, against central
finite differences of the FP64 oracle, and an exact linearity identity at the
full 1024x256 size.  Tolerance 1e-4 relative (float32 arithmetic accumulated
over the steps; the oracle adjoint itself is pinned to finite differences at
1e-6)."""
import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import oracle_problem

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300))


def _gpu_adjoint(torch, w, S0, nsteps, seed, K, prec="fp32"):
    from paper_2609_23057_b300.solver import solver_for
    s = solver_for(w, prec)
    s.set_state(torch.from_numpy(np.asarray(S0, np.float32)).cuda())
    gt, ga, gZ, gS = s.adjoint(nsteps, torch.from_numpy(np.asarray(seed, np.float32)).cuda(), checkpoint_every=K,
                               want_S0=True)
    out = (gt.cpu().numpy(), ga.cpu().numpy(), gZ, gS.cpu().numpy(), s.get_state().cpu().numpy())
    s.close()
    return out


@pytest.mark.parametrize("K", [1, 5, 12])
@pytest.mark.parametrize("nx,nz,nzen,naz,bc,surv,absm,nph", [
    (13, 9, 2, 4, (2, 0, 0, 0), 1, 0, 2),
    (20, 7, 4, 4, (2, 0, 1, 1), 0, 0, 3),
    (17, 11, 4, 8, (1, 1, 2, 0), 1, 1, 2),
    (9, 6, 8, 8, (2, 2, 0, 0), 1, 0, 2),
])
def test_adjoint_matches_oracle(torch_cuda, orc, nx, nz, nzen, naz, bc, surv, absm, nph, K):
    """K = 1 keeps every state (no recomputation), K = 5 three segments of
    5, 5 and 2 steps, K = 12 one segment."""
    w = W.random_medium(nx, nz, nzen, naz, seed=nx * nz, bc=bc, n_phase=nph, steps=12, surv_mode=surv)
    w.tau = np.minimum(w.tau, 0.9)
    w.abs_mode = absm
    P = oracle_problem(orc, w)
    S0 = W.random_state(nz, nx, w.n, seed=4)
    seed = np.random.default_rng(5).standard_normal((nx, w.n, 4)).astype(np.float32).astype(np.float64)
    rt, ra, rZ, rS = P.adjoint(S0, w.steps, seed, want_S0=True)
    gt, ga, gZ, gS, SN = _gpu_adjoint(torch_cuda, w, S0, w.steps, seed, K=K)
    assert _rel(gt, rt) < TOL
    assert _rel(ga, ra) < TOL
    assert _rel(gZ, rZ) < TOL
    assert _rel(gS, rS) < TOL
    # the state afterwards is the forward result
    assert _rel(SN, P.run(S0, w.steps)) < 1e-5


@pytest.mark.parametrize("K", [1, 5])
@pytest.mark.parametrize("nx,nz,nzen,naz,bc,nph", [
    (130, 5, 2, 4, (2, 0, 1, 1), 2),
    (256, 6, 4, 4, (2, 0, 0, 0), 2),
    (384, 4, 4, 8, (1, 1, 2, 0), 2),       # n = 32: tensor-core reverse step too
])
def test_adjoint_with_tf32x3_forward(torch_cuda, orc, nx, nz, nzen, naz, bc, nph, K):
    """A TF32X3 context runs the adjoint's forward pass and replays on the
    3xTF32 tensor-core step (float32 accuracy): gradients against the oracle
    adjoint at the same 1e-4, rows alternating class so most tiles are
    single-class (the rest run on the CUDA cores)."""
    w = W.random_medium(nx, nz, nzen, naz, seed=nx + 7 * nz, bc=bc, n_phase=nph, steps=9, surv_mode=1)
    w.tau = np.minimum(w.tau, 0.9)
    w.phase_index = (np.arange(nz)[:, None] % nph * np.ones((1, nx))).astype(np.uint8)
    P = oracle_problem(orc, w)
    S0 = W.random_state(nz, nx, w.n, seed=4)
    seed = np.random.default_rng(5).standard_normal((nx, w.n, 4)).astype(np.float32).astype(np.float64)
    rt, ra, rZ, rS = P.adjoint(S0, w.steps, seed, want_S0=True)
    gt, ga, gZ, gS, SN = _gpu_adjoint(torch_cuda, w, S0, w.steps, seed, K=K, prec="tf32x3")
    assert _rel(gt, rt) < TOL
    assert _rel(ga, ra) < TOL
    assert _rel(gZ, rZ) < TOL
    assert _rel(gS, rS) < TOL
    assert _rel(SN, P.run(S0, w.steps)) < 1e-5


@pytest.mark.parametrize("nzen,naz", [(2, 4), (4, 4), (4, 8)])
def test_adjoint_many_chunks_per_block(torch_cuda, orc, nzen, naz):
    """A lattice of 30,560 sites (477.5 chunks of 64 sites, so several chunks
    per block of the table-gradient sweep and a ragged last chunk), classes
    mixed inside chunks, n = 8, 16 and 32 directions."""
    w = W.random_medium(191, 160, nzen, naz, seed=7, bc=(2, 0, 1, 1), n_phase=3, steps=4, surv_mode=1)
    w.tau = np.minimum(w.tau, 0.9)
    w.abs_mode = 0
    P = oracle_problem(orc, w)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=4)
    seed = np.random.default_rng(5).standard_normal((w.nx, w.n, 4)).astype(np.float32).astype(np.float64)
    rt, ra, rZ, rS = P.adjoint(S0, w.steps, seed, want_S0=True)
    gt, ga, gZ, gS, _ = _gpu_adjoint(torch_cuda, w, S0, w.steps, seed, K=2)
    assert _rel(gt, rt) < TOL
    assert _rel(ga, ra) < TOL
    assert _rel(gZ, rZ) < TOL
    assert _rel(gS, rS) < TOL


@pytest.mark.parametrize("nx,nz,bc,nph,K,nzen,naz", [
    (256, 6, (2, 0, 1, 1), 2, 5, 4, 8),      # rows alternate class, 128 | nx: every tile single-class
    (200, 7, (2, 0, 0, 0), 2, 1, 4, 8),      # tiles straddle rows: single-class and mixed tiles
    (130, 3, (1, 1, 2, 0), 1, 4, 4, 8),      # one class, ragged last tile, periodic z
    (384, 4, (2, 2, 1, 1), 3, 12, 4, 8),
    (256, 6, (2, 0, 1, 1), 2, 5, 2, 4),      # n = 8: one staging slot per tile, K padded to 64
    (130, 3, (1, 1, 2, 0), 1, 4, 2, 4),
    (256, 6, (2, 0, 1, 1), 2, 5, 4, 4),      # n = 16
    (384, 4, (2, 2, 1, 1), 3, 12, 4, 4),
    (200, 7, (2, 0, 0, 0), 2, 1, 4, 4),      # mixed tiles at n = 16: the CUDA-core lambda form
])
def test_adjoint_tensor_core_reverse_step(torch_cuda, orc, nx, nz, bc, nph, K, nzen, naz):
    """n in {8, 16, 32}: the reverse step runs on the tensor cores over
    single-class 128-site tiles in the transposed-stream form (at n = 32 the
    mixed tiles on a CUDA-core variant of that form; at n = 8 and 16 a medium
    with mixed tiles keeps the CUDA-core lambda form); gradients and dL/dS0
    against the oracle adjoint."""
    w = W.random_medium(nx, nz, nzen, naz, seed=nx + nz, bc=bc, n_phase=nph, steps=9, surv_mode=1)
    w.tau = np.minimum(w.tau, 0.9)
    w.phase_index = (np.arange(nz)[:, None] % nph * np.ones((1, nx))).astype(np.uint8)
    P = oracle_problem(orc, w)
    S0 = W.random_state(nz, nx, w.n, seed=4)
    seed = np.random.default_rng(5).standard_normal((nx, w.n, 4)).astype(np.float32).astype(np.float64)
    rt, ra, rZ, rS = P.adjoint(S0, w.steps, seed, want_S0=True)
    gt, ga, gZ, gS, SN = _gpu_adjoint(torch_cuda, w, S0, w.steps, seed, K=K)
    assert _rel(gt, rt) < TOL
    assert _rel(ga, ra) < TOL
    assert _rel(gZ, rZ) < TOL
    assert _rel(gS, rS) < TOL
    assert _rel(SN, P.run(S0, w.steps)) < 1e-5


def test_adjoint_workspace_reuse(torch_cuda, orc):
    """Calls on one context reuse (and grow) the workspace: the same call
    repeated gives the same bits, a larger call after a smaller one and a
    call after rtlb_release_workspace still match the oracle."""
    from paper_2609_23057_b300.solver import solver_for
    w = W.random_medium(17, 11, 4, 4, seed=3, bc=(2, 0, 1, 1), n_phase=2, steps=12, surv_mode=1)
    w.tau = np.minimum(w.tau, 0.9)
    P = oracle_problem(orc, w)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=4)
    seed = np.random.default_rng(5).standard_normal((w.nx, w.n, 4)).astype(np.float32).astype(np.float64)
    rt, ra, rZ, rS = P.adjoint(S0, w.steps, seed, want_S0=True)
    s = solver_for(w, "fp32")
    S0d = torch_cuda.from_numpy(np.asarray(S0, np.float32)).cuda()
    seedd = torch_cuda.from_numpy(np.asarray(seed, np.float32)).cuda()
    outs = []
    for K, release in ((12, False), (12, False), (1, False), (5, True), (1, False)):
        if release:
            s.release_workspace()
        s.set_state(S0d)
        gt, ga, gZ, gS = s.adjoint(w.steps, seedd, checkpoint_every=K, want_S0=True)
        gt, ga, gS = gt.cpu().numpy(), ga.cpu().numpy(), gS.cpu().numpy()
        assert _rel(gt, rt) < TOL and _rel(ga, ra) < TOL and _rel(gZ, rZ) < TOL and _rel(gS, rS) < TOL
        outs.append((gt, ga, gZ, gS))
    s.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def _crop32_target(orc, w, nsteps):
    """Seeded target of the differentiation workload: the top radiance of a
    forward with tau x 1.1 in the cloud cells (class 1), times 1 + 0.05 N(0, 1)
    (seed 2)."""
    wt = W.adjoint(steps=nsteps).crop(112, 144, 496, 528)
    wt.tau = np.where(wt.phase_index == 1, wt.tau * 1.1, wt.tau)
    Pt = oracle_problem(orc, wt)
    top = Pt.radiance_out(Pt.run(Pt.zero_state(), nsteps), orc.SIDE_TOP)
    return top * (1.0 + 0.05 * np.random.default_rng(2).standard_normal(top.shape))


def test_adjoint_crop32_fd_and_g(torch_cuda, orc):
    """The differentiation workload (1024x256, n = 32, medium seed 2) on its
    32x32 crop (rows 112-143 across the cloud top, columns 496-527), run as
    its own problem for 1000 steps.  Loss: squared error of the top I, Q, U
    against the seeded target.  Checks: the GPU adjoint (checkpoint every 50
    steps) against the FP64 oracle adjoint (1e-4 of the largest gradient);
    the oracle adjoint against the oracle's central differences (1e-4) at 64
    random cells for tau and 16 for albedo, and the GPU gradient against the
    same differences within the sum of the two bounds; dL/dg
    (rtlb_phase_hg_grad) against a central difference in g.  The step is
    h = 5e-4: with h = 1e-3 the central difference's own truncation error
    (proportional to h^2) reaches 1.1e-4 of the largest gradient on this crop
    (cell (30, 17): -5.12435e-5 at h = 1e-3, -5.12372e-5 at 5e-4, adjoint
    -5.12350e-5), so it would not resolve 1e-4.  The differences
    run 200 steps: on this crop the top radiance after 200 steps equals the
    1000-step one to ~1e-11 relative (asserted), so the two losses are the
    same function to that accuracy, and 2 x 82 oracle forwards of 200 steps
    take a minute where 1000 steps would take five."""
    from paper_2609_23057_b300.solver import phase_hg_grad
    full_steps, fd_steps = 1000, 200
    w = W.adjoint(steps=full_steps).crop(112, 144, 496, 528)
    P = oracle_problem(orc, w)
    S0 = np.zeros((w.nz, w.nx, w.n, 4))
    target = _crop32_target(orc, w, fd_steps)
    m = np.zeros_like(target)
    m[..., :3] = 1.0
    top_full = P.radiance_out(P.run(S0, full_steps), orc.SIDE_TOP)
    top_fd = P.radiance_out(P.run(S0, fd_steps), orc.SIDE_TOP)
    assert np.abs(top_fd - top_full).max() <= 1e-10 * np.abs(top_full).max()

    def loss(Pp):
        top = Pp.radiance_out(Pp.run(S0, fd_steps), orc.SIDE_TOP)
        return float(np.sum(m * (top - target) ** 2))

    seed = 2 * m * (top_full - target)
    rt, ra, rZ = P.adjoint(S0, full_steps, seed)
    gt, ga, gZ, _, _ = _gpu_adjoint(torch_cuda, w, S0, full_steps, seed, K=50)
    assert _rel(gt, rt) < TOL and _rel(ga, ra) < TOL and _rel(gZ, rZ) < TOL
    rng = np.random.default_rng(5)
    h = 5e-4
    for field, grad, ref, count in (("tau", gt, rt, 64), ("albedo", ga, ra, 16)):
        cells = [tuple(c) for c in rng.integers(0, [w.nz, w.nx], size=(count, 2))]
        for z, x in cells:
            vals = []
            for sgn in (1, -1):
                Pp = oracle_problem(orc, w)
                getattr(Pp, field)[z, x] += sgn * h
                vals.append(loss(Pp))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - ref[z, x]) <= TOL * np.abs(ref).max(), (field, z, x)
            assert abs(fd - grad[z, x]) <= 2 * TOL * np.abs(ref).max(), (field, z, x)
    # cloud g (class 1 is HG with g = 0.85).  The loss curves strongly in g
    # near the forward peak: a central difference with h = 1e-3 carries ~2e-4
    # relative truncation error, so this one uses h = 1e-4 (~2e-6).
    g_adj = phase_hg_grad(w.n_zen, w.n_az, 0.85, -0.1, gZ[1])
    mu, phi = orc.direction_grid(w.n_zen, w.n_az)
    hz = 1e-6
    dZ_orc = (orc.phase_table_spec(mu, phi, ("hg", 0.85 + hz, -0.1)) -
              orc.phase_table_spec(mu, phi, ("hg", 0.85 - hz, -0.1))) / (2 * hz)
    assert g_adj == pytest.approx(float(np.sum(dZ_orc * rZ[1])), rel=TOL)
    hg = 1e-4
    vals = []
    for sgn in (1, -1):
        ww = W.adjoint(steps=fd_steps).crop(112, 144, 496, 528)
        ww.phase_specs = [("rayleigh",), ("hg", 0.85 + sgn * hg, -0.1)]
        vals.append(loss(oracle_problem(orc, ww)))
    g_fd = (vals[0] - vals[1]) / (2 * hg)
    assert g_adj == pytest.approx(g_fd, rel=TOL)


def test_adjoint_full_size_fd_of_gpu_forward(torch_cuda):
    """1024x256, n = 32, 1000 steps, checkpoint every 50 (the differentiation
    workload at full size): grad_tau and grad_albedo against central
    differences (h = 1e-3) of the float32 GPU forward, at the four cells
    where each gradient is largest and at four random cloud cells for tau.
    The forward is float32: a perturbed run differs from the base run by
    rounding noise of ~1e-7 of each top-radiance entry besides the effect of
    h, which limits what a difference quotient resolves (the first run of this
    test saw 2.7e-3 relative at an albedo cell whose gradient is 0.8 of the
    largest); the tolerance is 1e-3 of the largest gradient plus 1e-2 of the
    cell's own value.  The 32x32 crop test holds the adjoint to 1e-4 against
    the FP64 oracle."""
    from paper_2609_23057_b300.solver import solver_for
    w = W.adjoint(steps=1000)
    zero = torch_cuda.zeros((w.nz, w.nx, w.n, 4), dtype=torch_cuda.float32, device="cuda")

    def top_after(ww):
        s = solver_for(ww, "fp32")
        s.set_state(zero)
        s.step(ww.steps)
        top = s.radiance_out("top").cpu().numpy().astype(np.float64)
        s.close()
        return top

    wt = W.adjoint(steps=1000)
    wt.tau = np.where(wt.phase_index == 1, wt.tau * 1.1, wt.tau)
    target = top_after(wt) * (1.0 + 0.05 * np.random.default_rng(2).standard_normal((w.nx, w.n, 4)))
    m = np.zeros_like(target)
    m[..., :3] = 1.0
    top0 = top_after(w)
    seed = 2 * m * (top0 - target)
    s = solver_for(w, "fp32")
    s.set_state(zero)
    gt, ga, _, _ = s.adjoint(w.steps, torch_cuda.from_numpy(seed.astype(np.float32)).cuda(), checkpoint_every=50)
    gt, ga = gt.cpu().numpy().astype(np.float64), ga.cpu().numpy().astype(np.float64)
    s.close()

    def loss(ww):
        return float(np.sum(m * (top_after(ww) - target) ** 2))

    rng = np.random.default_rng(6)
    cloud = np.argwhere(w.phase_index == 1)
    h = 1e-3
    for field, grad in (("tau", gt), ("albedo", ga)):
        cells = [tuple(c) for c in np.argwhere(np.abs(grad) >= np.sort(np.abs(grad).ravel())[-4])[:4]]
        if field == "tau":
            cells += [tuple(cloud[k]) for k in rng.integers(0, len(cloud), 4)]
        for z, x in cells:
            vals, xs = [], []
            for sgn in (1, -1):
                ww = W.adjoint(steps=1000)
                arr = getattr(ww, field).copy()
                arr[z, x] = float(np.float32(arr[z, x] + sgn * h))   # the value the library sees
                xs.append(arr[z, x])
                setattr(ww, field, arr)
                vals.append(loss(ww))
            fd = (vals[0] - vals[1]) / (xs[0] - xs[1])
            assert abs(fd - grad[z, x]) <= 1e-3 * np.abs(grad).max() + 1e-2 * abs(grad[z, x]), \
                (field, z, x, fd, grad[z, x])


def test_adjoint_full_size_linearity(torch_cuda):
    """1024x256, n = 32, 1000 steps, checkpoint every 50: the map S^0 -> top
    radiance is affine, so for any direction dS, <grad_S0, dS> equals the
    change of <seed, top radiance> when S^0 moves by dS."""
    from paper_2609_23057_b300.solver import solver_for
    w = W.adjoint(steps=1000)
    rng = np.random.default_rng(3)
    seed = rng.standard_normal((w.nx, w.n, 4)).astype(np.float32)
    dS = torch_cuda.from_numpy(W.random_state(w.nz, w.nx, w.n, seed=7, dtype=np.float32)).cuda()
    s = solver_for(w, "fp32")
    zero = torch_cuda.zeros_like(dS)
    s.set_state(zero)
    gt, ga, gZ, gS = s.adjoint(w.steps, torch_cuda.from_numpy(seed).cuda(), checkpoint_every=50, want_S0=True)
    top0 = s.radiance_out("top").cpu().numpy().astype(np.float64)
    s.set_state(dS)
    s.step(w.steps)
    top1 = s.radiance_out("top").cpu().numpy().astype(np.float64)
    s.close()
    lhs = float(np.sum(seed * (top1 - top0)))
    rhs = float(torch_cuda.sum(gS.double() * dS.double()).item())
    assert np.isfinite(gt.cpu().numpy()).all() and np.isfinite(ga.cpu().numpy()).all()
    assert rhs == pytest.approx(lhs, rel=1e-4)


def test_autograd_function(torch_cuda, orc):
    """torch.autograd through top_radiance: gradients equal the oracle
    adjoint for tau and albedo and a central difference for g."""
    from paper_2609_23057_b300.solver import Solver, top_radiance
    w = W.adjoint(steps=60).crop(118, 134, 40, 60)
    s = Solver(w.nx, w.nz, w.n_zen, w.n_az, precision="fp32", survival="exp")
    s.set_boundary("top", "inflow", w.inflow[0])
    tau = torch_cuda.tensor(w.tau, dtype=torch_cuda.float32, device="cuda", requires_grad=True)
    alb = torch_cuda.tensor(w.albedo, dtype=torch_cuda.float32, device="cuda", requires_grad=True)
    g = torch_cuda.tensor(0.85, dtype=torch_cuda.float64, device="cuda", requires_grad=True)
    out = top_radiance(tau, alb, g, s, w.phase_specs, hg_index=1, phase_index=w.phase_index, nsteps=w.steps,
                       checkpoint_every=20)
    weight = torch_cuda.linspace(0.5, 1.5, out.numel(), device="cuda").reshape(out.shape)
    (out * weight).sum().backward()
    P = oracle_problem(orc, w)
    rt, ra, _ = P.adjoint(np.zeros((w.nz, w.nx, w.n, 4)), w.steps, weight.cpu().numpy().astype(np.float64))
    assert _rel(tau.grad.cpu().numpy(), rt) < TOL
    assert _rel(alb.grad.cpu().numpy(), ra) < TOL
    h = 1e-4
    vals = []
    for sgn in (1, -1):
        ww = W.adjoint(steps=60).crop(118, 134, 40, 60)
        ww.phase_specs = [("rayleigh",), ("hg", 0.85 + sgn * h, -0.1)]
        Pp = oracle_problem(orc, ww)
        top = Pp.radiance_out(Pp.run(np.zeros((w.nz, w.nx, w.n, 4)), w.steps), orc.SIDE_TOP)
        vals.append(float(np.sum(weight.cpu().numpy() * top)))
    assert g.grad.item() == pytest.approx((vals[0] - vals[1]) / (2 * h), rel=1e-4)
    s.close()
