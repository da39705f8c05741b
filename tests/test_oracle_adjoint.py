"""Pins of the oracle's reverse-mode gradients: central finite differences of
the FP64 forward solver (the loss is linear in the outgoing radiance,
L = <w, radiance_out(top, S^N)>), for per-cell extinction and albedo, table
entries and the initial state, in every survival / absorption mode."""
import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import oracle_problem


def _loss(orc, P, S0, nsteps, w):
    return float(np.sum(w * P.radiance_out(P.run(S0, nsteps), orc.SIDE_TOP)))


@pytest.mark.parametrize("surv,absm,bc", [(1, 0, (2, 0, 0, 0)), (0, 0, (2, 0, 1, 1)), (1, 1, (1, 1, 2, 0))])
def test_adjoint_matches_central_differences(orc, surv, absm, bc):
    w = W.random_medium(7, 6, 2, 4, seed=40 + surv + 2 * absm, bc=bc, n_phase=2, steps=6, surv_mode=surv)
    w.tau = np.minimum(w.tau, 0.9)
    w.abs_mode = absm
    P = oracle_problem(orc, w)
    rng = np.random.default_rng(1)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=3)
    wt = rng.standard_normal((w.nx, w.n, 4))
    gt, ga, gZ, gS = P.adjoint(S0, w.steps, wt, want_S0=True)
    L0 = _loss(orc, P, S0, w.steps, wt)
    assert np.isfinite(L0)

    def fd(mutate):
        h = 1e-6
        vals = []
        for sgn in (1, -1):
            Pp = oracle_problem(orc, w)
            S = S0.copy()
            mutate(Pp, S, sgn * h)
            vals.append(_loss(orc, Pp, S, w.steps, wt))
        return (vals[0] - vals[1]) / (2 * h)

    cells = [(0, 0), (w.nz - 1, 3), (2, w.nx - 1), (3, 4), (w.nz - 2, 1)]
    for z, x in cells:
        def mt(Pp, S, h, z=z, x=x):
            Pp.tau[z, x] += h
        def ma(Pp, S, h, z=z, x=x):
            Pp.albedo[z, x] += h
        assert fd(mt) == pytest.approx(gt[z, x], rel=1e-6, abs=1e-9)
        assert fd(ma) == pytest.approx(ga[z, x], rel=1e-6, abs=1e-9)
    for c, r, k in [(0, 0, 0), (1, 5, 9), (0, 13, 2), (1, 31, 30), (0, 7, 22)]:
        def mz(Pp, S, h, c=c, r=r, k=k):
            Pp.Z[c, r, k] += h
        assert fd(mz) == pytest.approx(gZ[c, r, k], rel=1e-6, abs=1e-9)
    for idx in [(0, 0, 0, 0), (5, 6, 4, 1), (2, 3, 7, 2), (4, 1, 3, 3)]:
        def ms(Pp, S, h, idx=idx):
            S[idx] += h
        assert fd(ms) == pytest.approx(gS[idx], rel=1e-6, abs=1e-9)


def test_adjoint_dot_product_identity(orc):
    """For the linear part of one step (no sources), <T C x, y> = <x, C^T T^T y>:
    the gradient of L(S0) = <y, S^1> w.r.t. S0 is C^T T^T y.  With the loss
    read only on the top row, pick y there and compare with an explicit
    brute-force Jacobian-vector product."""
    w = W.random_medium(5, 4, 2, 4, seed=9, bc=(0, 0, 1, 1), n_phase=2, steps=1, emission=False)
    P = oracle_problem(orc, w)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((w.nz, w.nx, w.n, 4))
    y = rng.standard_normal((w.nx, w.n, 4))
    _, _, _, gS = P.adjoint(np.zeros_like(x), 1, y, want_S0=True)
    lhs = np.sum(y * P.radiance_out(P.step(x), orc.SIDE_TOP))   # linear: no inflow, no emission
    rhs = np.sum(x * gS)
    assert lhs == pytest.approx(rhs, rel=1e-13)


@pytest.mark.parametrize("plane,bc", [("xz", (2, 0, 0, 0)), ("xy", (1, 1, 2, 0))])
def test_bilinear_adjoint_matches_central_differences(orc, plane, bc):
    """Semi-Lagrangian streaming (Eq. 34): the transposed step spreads each
    entry back over its four taps."""
    w = W.random_medium(7, 6, 2, 4, seed=77, bc=bc, n_phase=2, steps=5, surv_mode=1)
    w.tau = np.minimum(w.tau, 0.9)
    w.scheme, w.plane = "bilinear", plane
    P = oracle_problem(orc, w)
    rng = np.random.default_rng(8)
    S0 = W.random_state(w.nz, w.nx, w.n, seed=9)
    wt = rng.standard_normal((w.nx, w.n, 4))
    gt, ga, gZ, gS = P.adjoint(S0, w.steps, wt, want_S0=True)

    def fd(mutate):
        h = 1e-6
        vals = []
        for sgn in (1, -1):
            Pp = oracle_problem(orc, w)
            S = S0.copy()
            mutate(Pp, S, sgn * h)
            vals.append(_loss(orc, Pp, S, w.steps, wt))
        return (vals[0] - vals[1]) / (2 * h)

    for z, x in [(0, 0), (w.nz - 1, 3), (2, w.nx - 1), (3, 4)]:
        def mt(Pp, S, h, z=z, x=x):
            Pp.tau[z, x] += h
        assert fd(mt) == pytest.approx(gt[z, x], rel=1e-6, abs=1e-9)
    for c, r, k in [(0, 0, 0), (1, 5, 9), (0, 13, 2)]:
        def mz(Pp, S, h, c=c, r=r, k=k):
            Pp.Z[c, r, k] += h
        assert fd(mz) == pytest.approx(gZ[c, r, k], rel=1e-6, abs=1e-9)
    for idx in [(0, 0, 0, 0), (5, 6, 4, 1), (2, 3, 7, 2)]:
        def ms(Pp, S, h, idx=idx):
            S[idx] += h
        assert fd(ms) == pytest.approx(gS[idx], rel=1e-6, abs=1e-9)
