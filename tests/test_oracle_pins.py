"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage (section / equation) or the identity it checks.
None of them compares the oracle with itself through a retyped formula: they
use values the paper prints, closed forms, invariants, special cases that
reduce to a hand-written loop, and brute-force linear solves on tiny lattices.
"""
import math
import os

import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import oracle_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def _unit(mu, phi):
    st = np.sqrt(1 - mu ** 2)
    return np.stack([st * np.cos(phi), st * np.sin(phi), mu], -1)


# ------------------------------------------------------------ Mueller matrices

@pytest.mark.parametrize("theta_deg", [0.0, 17.0, 60.0, 75.5, 90.0, 104.5, 151.0, 180.0])
def test_rayleigh_spectrum(orc, theta_deg):
    """Eq. 16-19: P~(theta) is symmetric with eigenvalues {1, cos^2, cos, cos}."""
    c = math.cos(math.radians(theta_deg))
    P = orc.rayleigh_matrix(c)
    assert np.allclose(P, P.T)
    ev = np.sort(np.linalg.eigvalsh(P))
    assert np.allclose(ev, np.sort([1.0, c * c, c, c]), atol=1e-14)


def test_rayleigh_continuum_normalization(orc):
    """Eq. 16: the 3/(8 pi) prefactor makes the (1,1) element integrate to one
    over the sphere (int P11 dOmega = 1)."""
    x, wq = np.polynomial.legendre.leggauss(64)
    vals = np.array([orc.rayleigh_matrix(c)[0, 0] for c in x])
    integral = 2 * math.pi * np.sum(wq * vals) * 3 / (8 * math.pi)
    assert abs(integral - 1.0) < 1e-13


def test_hg_continuum_normalization_and_stokes_criterion(orc):
    """HG cloud matrix: the scalar phase function integrates to 4 pi (mean 1),
    its first moment is g, and every element pair satisfies p^2 + q^2 = 1."""
    x, wq = np.polynomial.legendre.leggauss(400)
    for g in (0.0, 0.5, 0.85):
        M = np.array([orc.hg_matrix(c, g, -0.1) for c in x])
        h = M[:, 0, 0]
        assert abs(0.5 * np.sum(wq * h) - 1.0) < 1e-6
        assert abs(0.5 * np.sum(wq * h * x) - g) < 1e-6
        p, q = M[:, 0, 1] / h, M[:, 2, 2] / h
        assert np.allclose(p, -0.1 * (1 - x ** 2))
        assert np.allclose(p ** 2 + q ** 2, 1.0)


@pytest.mark.parametrize("a,b", [(0.3, 0.4), (-1.1, 2.5), (0.0, math.pi / 2)])
def test_rotation_group(orc, a, b):
    """Eq. 21/22: R(a) R(b) = R(a + b), R(pi) = I, and the action on (Q, U)."""
    assert np.allclose(orc.rotation(a) @ orc.rotation(b), orc.rotation(a + b), atol=1e-14)
    assert np.allclose(orc.rotation(math.pi), np.eye(4), atol=1e-14)
    S = np.array([1.0, 0.3, -0.2, 0.1])
    out = orc.rotation(a) @ S
    c, s = math.cos(2 * a), math.sin(2 * a)
    assert np.allclose(out, [1.0, 0.3 * c - 0.2 * s, -0.2 * c - 0.3 * s, 0.1])


# ---------------------------------------------------------------- phase table

def test_single_scatter_dop_matches_paper(orc):
    """Sec. 3.2.2 (Fig. 16): at step 1, light scattered from natural light at
    60/120 deg has DOP 0.6000 and at 75.5/104.5 deg 9/17.  For each outgoing
    direction, sum the contributions of all incoming directions at that
    scattering angle (the field is isotropic at step 1)."""
    gold = _load_golden("single_scatter_dop_n8.txt")
    mu, phi = orc.direction_grid(2, 4)
    Z = orc.phase_table(mu, phi)
    om = _unit(mu, phi)
    for o in range(8):
        for ang, want in gold:
            acc = np.zeros(4)
            for i in range(8):
                t = math.degrees(math.acos(np.clip(om[o] @ om[i], -1, 1)))
                if abs(t - ang) < 0.1:
                    acc += Z[4 * o:4 * o + 4, 4 * i:4 * i + 4] @ np.array([1.0, 0, 0, 0])
            assert acc[0] > 0
            assert abs(orc.dop(acc) - want) < 1e-12, (o, ang)


def test_literal_azimuth_frame_reading_would_fail_the_paper_values(orc):
    """Documents the reading of Eq. 15: with psi_out - psi_in equal to the
    azimuth difference (90 deg here) the two 75.5-deg contributions keep DOP
    15/17, not the 9/17 the paper reports; the geometric frame angle gives
    |cos 2 psi| = 0.6 and hence 9/17."""
    c = 0.25                               # cos(75.5 deg)
    P = orc.rayleigh_matrix(c)
    lit = orc.rotation(-math.pi / 2) @ P @ orc.rotation(0.0) @ np.array([1.0, 0, 0, 0])
    assert abs(orc.dop(lit) - 15 / 17) < 1e-12


@pytest.mark.parametrize("nzen,naz", [(2, 4), (4, 8), (8, 8), (3, 6), (1, 4)])
def test_table_normalization(orc, nzen, naz):
    """Eq. 17 / 26: column-normalized weights sum to one (sum_o Z11(o,i) = 1);
    the U and V rows of the I column vanish in total (no net circular or
    oblique polarization is created from natural light)."""
    mu, phi = orc.direction_grid(nzen, naz)
    for spec in [("rayleigh",), ("hg", 0.85, -0.1)]:
        Z = orc.phase_table_spec(mu, phi, spec)
        n = len(mu)
        for i in range(n):
            assert abs(Z[0::4, 4 * i].sum() - 1.0) < 1e-13
            assert abs(Z[2::4, 4 * i].sum()) < 1e-13
            assert abs(Z[3::4, 4 * i].sum()) < 1e-13
        assert np.all(Z[0::4, 0::4] >= 0)


@pytest.mark.parametrize("nzen,naz", [(2, 4), (4, 8), (8, 8), (3, 6)])
def test_reciprocity(orc, nzen, naz):
    """Mueller reciprocity for the un-normalized blocks:
    M(o, i) = D M(-i, -o)^T D with D = diag(1, 1, -1, 1)."""
    mu, phi = orc.direction_grid(nzen, naz)
    n = len(mu)

    def opposite(k):
        for j in range(n):
            if abs(mu[j] + mu[k]) < 1e-12 and abs(math.cos(phi[j] - phi[k] - math.pi) - 1) < 1e-12:
                return j
        raise AssertionError("grid not symmetric")

    D = np.diag([1.0, 1.0, -1.0, 1.0])
    for spec in [(orc.PHASE_RAYLEIGH, 0, 0), (orc.PHASE_HG, 0.85, -0.1)]:
        for o in range(n):
            for i in range(n):
                M, _ = orc.rpr_block(mu[o], phi[o], mu[i], phi[i], *spec)
                mi, mo = opposite(i), opposite(o)
                M2, _ = orc.rpr_block(mu[mi], phi[mi], mu[mo], phi[mo], *spec)
                assert np.abs(M - D @ M2.T @ D).max() < 1e-13 * max(1.0, np.abs(M).max())


def test_blocks_preserve_the_stokes_cone(orc):
    """Every block maps physically realizable Stokes vectors (I >= |QUV|) to
    realizable ones, so the step keeps I^2 >= Q^2 + U^2 + V^2."""
    rng = np.random.default_rng(5)
    mu, phi = orc.direction_grid(4, 8)
    n = len(mu)
    v = rng.standard_normal((200, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    S = np.concatenate([np.ones((200, 1)), v], 1).T           # on the cone surface
    for spec in [("rayleigh",), ("hg", 0.85, -0.1)]:
        Z = orc.phase_table_spec(mu, phi, spec)
        for o in range(0, n, 3):
            for i in range(0, n, 5):
                out = Z[4 * o:4 * o + 4, 4 * i:4 * i + 4] @ S
                assert np.all(out[0] + 1e-14 >= np.linalg.norm(out[1:], axis=0))


def test_degenerate_pairs(orc):
    """Forward scattering is the identity; backscattering in the meridian
    plane is diag(1, 1, -1, -1) (P~(pi) with no frame rotation)."""
    M, w = orc.rpr_block(0.3, 1.0, 0.3, 1.0)
    assert np.allclose(M, np.eye(4)) and w == pytest.approx(1.0)
    M, _ = orc.rpr_block(-0.3, 1.0 + math.pi, 0.3, 1.0)
    assert np.allclose(M, np.diag([1.0, 1.0, -1.0, -1.0]))


# ----------------------------------------------------------------- streaming

def test_stream_offsets_n8(orc):
    """n = 8 (Sec. 3.2.1: 2 zenith x 4 azimuth): projections (+-0.866, +-0.5)
    go to the diagonals and the phi = 90/270 deg ones straight up/down."""
    mu, phi = orc.direction_grid(2, 4)
    cx, cz = orc.stream_offsets(mu, phi)
    assert list(cx) == [1, 0, -1, 0, 1, 0, -1, 0]
    assert list(cz) == [-1, -1, -1, -1, 1, 1, 1, 1]


def test_stream_offsets_rest_and_axis(orc):
    """An odd zenith count puts mu = 0 in the grid: phi = 0 / pi stream along
    +-x and phi = 90/270 deg have a zero projection and rest."""
    mu, phi = orc.direction_grid(1, 4)
    cx, cz = orc.stream_offsets(mu, phi)
    assert list(cx) == [1, 0, -1, 0] and list(cz) == [0, 0, 0, 0]


def test_stream_offsets_brute_force(orc):
    """Offsets equal the neighbour direction of smallest angle to the
    projection, found by brute force over the 8 unit offsets."""
    offs = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    for nzen, naz in [(4, 8), (8, 8), (3, 6), (4, 4), (5, 7)]:
        mu, phi = orc.direction_grid(nzen, naz)
        cx, cz = orc.stream_offsets(mu, phi)
        for d in range(len(mu)):
            px, pz = math.sqrt(1 - mu[d] ** 2) * math.cos(phi[d]), mu[d]
            if math.hypot(px, pz) < 1e-12:
                assert (cx[d], cz[d]) == (0, 0)
                continue
            ang = [math.acos(np.clip((px * a + pz * b) / math.hypot(px, pz) / math.hypot(a, b), -1, 1))
                   for a, b in offs]
            assert (cx[d], cz[d]) == offs[int(np.argmin(ang))]


def test_stream_offset_tie_is_rejected(orc):
    """A projection exactly between two offsets (22.5 deg) has no nearest one."""
    mu = math.sin(math.radians(22.5))
    with pytest.raises(ValueError):
        orc.stream_offsets(np.array([mu]), np.array([0.0]))


# ------------------------------------------------------------ closed forms

def _vacuum_problem(orc, nx, nz, nzen, naz, tau, w0, e, bc=(0, 0, 0, 0), inflow=None,
                    spec=("rayleigh",), surv=0, absm=0, Z=None):
    mu, phi = orc.direction_grid(nzen, naz)
    if Z is None:
        Z = orc.phase_table_spec(mu, phi, spec)
    return orc.Problem(nx, nz, mu, phi, tau, w0, e, None, Z, surv_mode=surv, abs_mode=absm,
                       bc=bc, inflow=inflow)


def test_beer_lambert_direct_beam(orc):
    """Sec. 2.1.4 (Beer-Lambert transmission) + streaming: with no scattering
    and no emission, the top beam on direction 0 (offset (1, -1)) reaches the
    k-th row below the top as exp(-k tau) in the lit region x >= k and is zero
    in the shadow x < k."""
    nx, nz, tau = 12, 10, 0.3
    inflow = W.top_beam(8)
    P = _vacuum_problem(orc, nx, nz, 2, 4, tau, 0.0, None, bc=(2, 0, 0, 0), inflow=inflow)
    S = P.run(P.zero_state(), nz + 2)
    for k in range(nz):
        z = nz - 1 - k
        for x in range(nx):
            want = math.exp(-k * tau) if x >= k else 0.0
            assert S[z, x, 0, 0] == pytest.approx(want, rel=1e-13, abs=1e-300)
    assert np.all(S[..., 1:, :] == 0) and np.all(S[..., 0, 1:] == 0)


def test_taylor_absorption(orc):
    """Sec. 2.1.4: the first-order Taylor form attenuates by 1 - k_abs dt."""
    inflow = W.top_beam(8)
    P = _vacuum_problem(orc, 6, 6, 2, 4, 0.2, 0.0, None, bc=(2, 0, 0, 0), inflow=inflow, absm=1)
    S = P.run(P.zero_state(), 8)
    assert S[2, 5, 0, 0] == pytest.approx(0.8 ** 3, rel=1e-14)


def test_emission_geometric_series(orc):
    """Eq. 6/8 (source added every step without depletion) + absorption:
    after t steps a cell with at least t upstream cells holds
    e A (1 - A^t) / (1 - A), A = exp(-tau)."""
    nx = nz = 16
    tau, e, t = 0.25, 0.01, 5
    P = _vacuum_problem(orc, nx, nz, 2, 4, tau, 0.0, e)
    S = P.run(P.zero_state(), t)
    A = math.exp(-tau)
    want = e * A * (1 - A ** t) / (1 - A)
    assert S[8, 8, :, 0] == pytest.approx(np.full(8, want), rel=1e-13)
    assert np.all(S[..., 1:] == 0)
    # direction 0 streams by (1, -1): at x = 1 the upstream chain holds one
    # cell, at x = 0 none (left ghost, vacuum)
    assert S[8, 1, 0, 0] == pytest.approx(e * A, rel=1e-13)
    assert S[8, 0, 0, 0] == 0.0


def test_energy_split_matches_paper(orc):
    """Sec. 3.2.1: with dt = 1/16, k_ext = 2.5, k_scat = 0.5 about 97% of the
    energy stays unscattered per step and ~3% is redistributed."""
    nx, ny, kext, ksca, surv, tol = _load_golden("energy_split.txt")[0]
    dt = min(1 / nx, 1 / ny)
    tau, w0 = kext * dt, ksca / kext
    # one collision of a unit I beam at one site: the unscattered part is
    # what stays in the incoming direction minus its forward-scattered share.
    mu, phi = orc.direction_grid(2, 4)
    Z = orc.phase_table(mu, phi)
    P = orc.Problem(1, 1, mu, phi, tau, w0, None, None, Z, bc=(1, 1, 1, 1))
    S = P.zero_state()
    S[0, 0, 0, 0] = 1.0
    out = P.step(S)
    A = math.exp(-(1 - w0) * tau)
    unscattered = A * (1 - w0 * tau)
    scattered = out[0, 0, :, 0].sum() - unscattered
    assert abs(unscattered / (unscattered + scattered) - surv) < tol
    assert scattered == pytest.approx(A * w0 * tau, rel=1e-13)


def test_conservation_scalar_table(orc):
    """Albedo 1, no absorption, no emission, periodic on both axes: with the
    I-only part of the table, total intensity is conserved exactly."""
    mu, phi = orc.direction_grid(4, 8)
    Z = orc.phase_table(mu, phi)
    Zs = np.zeros_like(Z)
    Zs[0::4, 0::4] = Z[0::4, 0::4]
    P = _vacuum_problem(orc, 9, 7, 4, 8, 0.4, 1.0, None, bc=(1, 1, 1, 1), Z=Zs)
    S = W.random_state(7, 9, 32, seed=3)
    tot0 = S[..., 0].sum()
    S = P.run(S, 25)
    assert S[..., 0].sum() == pytest.approx(tot0, rel=1e-13)


def test_conservation_drift_polarized_table(orc):
    """With the full polarized table sum_o Z12(o, i) != 0 on a discrete grid,
    so total I changes each step by exactly sum_i (1 - s) (sum_o Z12) Q_i
    (and the U, V columns contribute sum_o Z13 = sum_o Z14 = 0)."""
    mu, phi = orc.direction_grid(2, 4)
    Z = orc.phase_table(mu, phi)
    tau = 0.4
    P = _vacuum_problem(orc, 5, 4, 2, 4, tau, 1.0, None, bc=(1, 1, 1, 1), Z=Z)
    S = W.random_state(4, 5, 8, seed=4)
    s = 1 - tau
    z12 = np.array([Z[0::4, 4 * i + 1].sum() for i in range(8)])
    z13 = np.array([Z[0::4, 4 * i + 2].sum() for i in range(8)])
    z14 = np.array([Z[0::4, 4 * i + 3].sum() for i in range(8)])
    assert np.abs(z12).max() > 1e-3 and np.abs(z13).max() < 1e-13 and np.abs(z14).max() < 1e-13
    out = P.step(S)
    predicted = S[..., 0].sum() + (1 - s) * np.sum(S[..., 1] * z12)
    assert out[..., 0].sum() == pytest.approx(predicted, rel=1e-13)


def test_stokes_criterion_over_a_run(orc):
    """I^2 >= Q^2 + U^2 + V^2 holds at every site and direction along a run
    with polarized inflow, two phase classes and all boundary kinds."""
    w = W.random_medium(11, 9, 4, 8, seed=7, bc=(2, 0, 1, 1), surv_mode=0)
    w.albedo = np.minimum(w.albedo, 1.0 / np.maximum(w.tau, 1e-9))   # linear survival >= 0
    P = oracle_problem(orc, w)
    S = W.random_state(9, 11, 32, seed=8)
    for _ in range(6):
        S = P.step(S)
        assert np.all(S[..., 0] ** 2 * (1 + 1e-12) + 1e-300 >= (S[..., 1:] ** 2).sum(-1))


def test_periodic_translation(orc):
    """'Shifts taken modulo' (Eq. 39 text): with no extinction a single entry
    travels around a periodic lattice and returns after nx steps."""
    mu, phi = orc.direction_grid(1, 4)            # d = 0 streams along +x
    P = orc.Problem(7, 3, mu, phi, 0.0, 0.0, None, None, orc.phase_table(mu, phi),
                    bc=(1, 1, 1, 1))
    S = P.zero_state()
    S[1, 2, 0] = [1.0, 0.2, -0.1, 0.05]
    out = P.run(S, 3)
    assert np.array_equal(out[1, 5, 0], S[1, 2, 0])
    assert np.array_equal(P.run(S, 7), S)


# -------------------------------------------------- brute-force linear algebra

def _dense_operator(orc, P):
    """The affine step S' = T (C S + c0) + b as explicit matrices, assembled
    from the problem definition (independent index arithmetic)."""
    nx, nz, n = P.nx, P.nz, P.n
    K = 4 * n
    N = nx * nz * K
    Cm = np.zeros((N, N))
    c0 = np.zeros(N)
    T = np.zeros((N, N))
    b = np.zeros(N)
    E = np.zeros(K)
    E[0::4] = 1.0
    for z in range(nz):
        for x in range(nx):
            st = z * nx + x
            tau, w0 = P.tau[z, x], P.albedo[z, x]
            e = 0.0 if P.emission is None else P.emission[z, x]
            Zc = P.Z[0 if P.cls is None else P.cls[z, x]]
            A = math.exp(-(1 - w0) * tau)
            s = 1 - w0 * tau if P.surv_mode == 0 else math.exp(-w0 * tau)
            blk = A * (s * np.eye(K) + (1 - s) * Zc)
            Cm[st * K:(st + 1) * K, st * K:(st + 1) * K] = blk
            c0[st * K:(st + 1) * K] = blk @ (e * E)
    per_x = P.bc[2] == 1
    per_z = P.bc[0] == 1
    for z in range(nz):
        for x in range(nx):
            for d in range(n):
                xs, zs = x - P.cx[d], z - P.cz[d]
                if per_x:
                    xs %= nx
                if per_z:
                    zs %= nz
                row = ((z * nx + x) * n + d) * 4
                if 0 <= xs < nx and 0 <= zs < nz:
                    col = ((zs * nx + xs) * n + d) * 4
                    for s_ in range(4):
                        T[row + s_, col + s_] = 1.0
                else:
                    side = 0 if zs >= nz else 1 if zs < 0 else 2 if xs < 0 else 3
                    if P.bc[side] == 2:
                        b[row:row + 4] = P.inflow[side, d]
    return T, Cm, c0, b


@pytest.mark.parametrize("size,bc", [(4, (2, 0, 0, 0)), (6, (2, 0, 1, 1)), (5, (0, 0, 0, 0))])
def test_steady_state_dense_solve(orc, size, bc):
    """Eq. 1 with the time derivative set to zero: the fixed point of the
    lattice step equals the dense LU solve of (I - T C) S = T c0 + b."""
    w = W.random_medium(size, size, 2, 4, seed=size, bc=bc, n_phase=2)
    w.tau = np.minimum(w.tau, 0.9)
    P = oracle_problem(orc, w)
    T, Cm, c0, b = _dense_operator(orc, P)
    N = T.shape[0]
    Sx = np.linalg.solve(np.eye(N) - T @ Cm, T @ c0 + b)
    S, steps, r = P.run_to_steady(P.zero_state(), 1e-14, 20000)
    assert r < 1e-14
    assert np.abs(S.ravel() - Sx).max() <= 1e-11 * np.abs(Sx).max()


def test_time_dependent_dense_powers(orc):
    """The first ten steps equal repeated application of the assembled affine
    operator (brute force on a 4x3 lattice, n = 8, two classes)."""
    w = W.random_medium(4, 3, 2, 4, seed=11, bc=(2, 1, 0, 0)[:1] + (0, 0, 0), n_phase=2)
    P = oracle_problem(orc, w)
    T, Cm, c0, b = _dense_operator(orc, P)
    S = W.random_state(3, 4, 8, seed=12)
    v = S.ravel().copy()
    for _ in range(10):
        S = P.step(S)
        v = T @ (Cm @ v + c0) + b
        assert np.abs(S.ravel() - v).max() <= 1e-13 * np.abs(v).max()


def test_two_direction_lattice_reproduces_hand_d1q2_loop(orc):
    """Sec. 3.1: a 2D lattice restricted to the +-x directions reproduces a
    1D two-velocity (D1Q2) loop written by hand: scattering splits evenly
    between forward and backward (Rayleigh weights a(0) = a(pi) = 1), and
    the back-scattered Stokes vector flips U and V."""
    mu = np.array([0.0, 0.0])
    phi = np.array([0.0, math.pi])
    Z = orc.phase_table(mu, phi)
    nx, tau, w0, e, steps = 32, 2.5 / 32, 0.2, 1.0 / 32, 40
    em = np.zeros((1, nx))
    em[0, 12:20] = e
    P = orc.Problem(nx, 1, mu, phi, tau, w0, em, None, Z, bc=(0, 0, 0, 0))
    S = P.run(P.zero_state(), steps)
    # hand loop, intensity only (the source is unpolarized and Q stays 0)
    A, s = math.exp(-(1 - w0) * tau), 1 - w0 * tau
    fwd, bwd = np.zeros(nx), np.zeros(nx)
    for _ in range(steps):
        f, g = fwd + em[0], bwd + em[0]
        pf = A * (s * f + (1 - s) * 0.5 * (f + g))
        pb = A * (s * g + (1 - s) * 0.5 * (f + g))
        fwd = np.concatenate([[0.0], pf[:-1]])
        bwd = np.concatenate([pb[1:], [0.0]])
    assert np.allclose(S[0, :, 0, 0], fwd, rtol=1e-14, atol=0)
    assert np.allclose(S[0, :, 1, 0], bwd, rtol=1e-14, atol=0)


def test_residual_and_radiance_out(orc):
    """Residual = max|S_new - S_old| / max|S_new|; radiance_out(top) keeps
    the top row for directions leaving through the top (cz = +1) only."""
    a = np.array([1.0, -2.0, 3.0])
    b = np.array([1.5, -2.0, 2.0])
    assert orc.residual(a, b) == pytest.approx(1.0 / 2.0)
    w = W.small(steps=1)
    P = oracle_problem(orc, w)
    S = W.random_state(w.nz, w.nx, w.n, seed=1)
    out = P.radiance_out(S, orc.SIDE_TOP)
    for d in range(8):
        if P.cz[d] == 1:
            assert np.array_equal(out[:, d], S[-1, :, d])
        else:
            assert np.all(out[:, d] == 0)
    left = P.radiance_out(S, orc.SIDE_LEFT)
    for d in range(8):
        assert np.array_equal(left[:, d], S[:, 0, d] if P.cx[d] == -1 else 0 * S[:, 0, d])


# ----------------------------------------------------------- table variants

def test_depolarized_rayleigh_limits(orc):
    """Hansen & Travis (1974) depolarized Rayleigh matrix: rho = 0 is Eq. 16;
    the (1,1) element stays normalized over the sphere; unpolarized light
    scattered at 90 deg has degree of polarization (1 - rho) / (1 + rho)."""
    for c in (-0.7, 0.0, 0.3, 1.0):
        assert np.allclose(orc.rayleigh_depol_matrix(c, 0.0), orc.rayleigh_matrix(c), atol=1e-15)
    x, wq = np.polynomial.legendre.leggauss(64)
    for rho in (0.0, 0.0279, 0.1):
        vals = np.array([orc.rayleigh_depol_matrix(c, rho)[0, 0] for c in x])
        assert abs(2 * math.pi * np.sum(wq * vals) * 3 / (8 * math.pi) - 1.0) < 1e-13
        P = orc.rayleigh_depol_matrix(0.0, rho)
        assert abs(abs(P[0, 1]) / P[0, 0] - (1 - rho) / (1 + rho)) < 1e-14


def test_depolarized_table_keeps_normalization_and_cone(orc):
    mu, phi = orc.direction_grid(4, 8)
    Z = orc.phase_table_spec(mu, phi, ("rayleigh", 0.0279))
    for i in range(32):
        assert abs(Z[0::4, 4 * i].sum() - 1.0) < 1e-13
    rng = np.random.default_rng(1)
    v = rng.standard_normal((3, 100))
    S = np.vstack([np.ones(100), v / np.linalg.norm(v, axis=0)])
    for o in range(0, 32, 5):
        for i in range(0, 32, 3):
            out = Z[4 * o:4 * o + 4, 4 * i:4 * i + 4] @ S
            assert np.all(out[0] + 1e-14 >= np.linalg.norm(out[1:], axis=0))


def test_conservative_table_conserves_polarized_intensity(orc):
    """With the intensity-conserving correction the total intensity is
    conserved exactly at albedo 1 even for polarized light (the plain table
    drifts by sum (1-s) (sum_o Z12) Q per step)."""
    mu, phi = orc.direction_grid(2, 4)
    Z = orc.conserve_intensity(orc.phase_table(mu, phi))
    for i in range(8):
        assert abs(Z[0::4, 4 * i].sum() - 1.0) < 1e-14
        for k in (1, 2, 3):
            assert abs(Z[0::4, 4 * i + k].sum()) < 1e-14
    P = orc.Problem(5, 4, mu, phi, 0.4, 1.0, None, None, Z, bc=(1, 1, 1, 1))
    S = W.random_state(4, 5, 8, seed=4)
    tot0 = S[..., 0].sum()
    assert P.run(S, 20)[..., 0].sum() == pytest.approx(tot0, rel=1e-13)
