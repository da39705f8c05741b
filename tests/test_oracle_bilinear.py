"""Pins of the oracle's semi-Lagrangian bilinear streaming (Eq. 33-38) and of
the lattice-plane choice, against closed forms that do not reuse the oracle's
tap construction: a point source spreads as the product of two binomial laws
whose mean moves by the direction's displacement every step; the streamed
field is the bilinear interpolation of the old one at the departure point
x - l (the textbook semi-Lagrangian definition, ghost cells included); lattice-
aligned directions reduce to the nearest-offset scheme; a uniform inflow fills
the lattice."""
import math

import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import oracle_problem

DIRS = [(0.3, 0.4), (-0.8, 2.5), (0.55, 4.0), (-0.2, 5.9), (0.95, 1.3)]


def _identity_problem(orc, nx, nz, mu, phi, plane, bc=(1, 1, 1, 1), inflow=None, scheme="bilinear"):
    """tau = 0: no absorption, survival s = 1 (LINEAR), so a step is pure streaming."""
    mu, phi = np.asarray(mu, float), np.asarray(phi, float)
    Z = orc.phase_table(mu, phi)
    return orc.Problem(nx, nz, mu, phi, np.zeros((nz, nx)), np.full((nz, nx), 0.5), None, None, Z,
                       bc=bc, inflow=inflow, scheme=scheme, plane=plane)


def _projection(mu, phi, plane):
    st = math.sqrt(1 - mu * mu)
    return (st * math.cos(phi), mu) if plane == 0 else (st * math.cos(phi), st * math.sin(phi))


@pytest.mark.parametrize("plane", [0, 1])
def test_tap_weights_are_a_distribution_with_mean_l(orc, plane):
    mu = np.array([m for m, _ in DIRS])
    phi = np.array([p for _, p in DIRS])
    ox, oz, w, lx, lz = orc.bilinear_taps(mu, phi, plane)
    for d in range(len(mu)):
        px, pz = _projection(mu[d], phi[d], plane)
        assert lx[d] == pytest.approx(px, abs=1e-15) and lz[d] == pytest.approx(pz, abs=1e-15)
        assert (w[d] >= 0).all() and w[d].sum() == pytest.approx(1.0, abs=1e-15)
        assert np.dot(w[d], ox[d]) == pytest.approx(px, abs=1e-15)
        assert np.dot(w[d], oz[d]) == pytest.approx(pz, abs=1e-15)


@pytest.mark.parametrize("plane", [0, 1])
def test_point_source_spreads_binomially(orc, plane):
    """t steps of pure streaming of a unit pulse: per axis, a sum of t
    independent moves of floor(l) + Bernoulli(frac(l)) cells."""
    nx = nz = 41
    t = 8
    for mu_d, phi_d in DIRS:
        P = _identity_problem(orc, nx, nz, [mu_d], [phi_d], plane)
        S = P.zero_state()
        stokes = np.array([1.0, 0.3, -0.2, 0.1])
        S[20, 20, 0] = stokes
        S = P.run(S, t)
        lx, lz = _projection(mu_d, phi_d, plane)
        expect = np.zeros((nz, nx))
        bx, fx = math.floor(lx), lx - math.floor(lx)
        bz, fz = math.floor(lz), lz - math.floor(lz)
        for kx in range(t + 1):
            for kz in range(t + 1):
                p = (math.comb(t, kx) * fx ** kx * (1 - fx) ** (t - kx) *
                     math.comb(t, kz) * fz ** kz * (1 - fz) ** (t - kz))
                expect[20 + t * bz + kz, 20 + t * bx + kx] += p
        for s in range(4):
            assert np.abs(S[:, :, 0, s] - stokes[s] * expect).max() < 1e-14
        # the centre of mass moved by t * l
        zz, xx = np.mgrid[0:nz, 0:nx]
        I = S[:, :, 0, 0]
        assert (I * xx).sum() == pytest.approx(20 + t * lx, abs=1e-12)
        assert (I * zz).sum() == pytest.approx(20 + t * lz, abs=1e-12)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (2, 2, 2, 2), (1, 1, 2, 0), (2, 0, 1, 1)])
@pytest.mark.parametrize("plane", [0, 1])
def test_step_is_bilinear_interpolation_at_the_departure_point(orc, bc, plane):
    """New value at node (x, z) = bilinear interpolation of the old field,
    extended by the ghost layer (vacuum 0, inflow vector, periodic wrap), at
    the departure point (x - lx, z - lz)."""
    nx, nz = 7, 5
    mu = np.array([m for m, _ in DIRS])
    phi = np.array([p for _, p in DIRS])
    n = len(mu)
    rng = np.random.default_rng(11)
    inflow = rng.uniform(0, 1, (4, n, 4))
    P = _identity_problem(orc, nx, nz, mu, phi, plane, bc=bc, inflow=inflow)
    S0 = rng.uniform(0, 1, (nz, nx, n, 4))
    S1 = P.step(S0)

    def node(x, z, d):
        if bc[2] == 1:
            x %= nx
        if bc[0] == 1:
            z %= nz
        side = 0 if z >= nz else 1 if z < 0 else 2 if x < 0 else 3 if x >= nx else -1
        if side < 0:
            return S0[z, x, d]
        return inflow[side, d] if bc[side] == 2 else np.zeros(4)

    for d in range(n):
        lx, lz = _projection(mu[d], phi[d], plane)
        for z in range(nz):
            for x in range(nx):
                px, pz = x - lx, z - lz
                x0, z0 = math.floor(px), math.floor(pz)
                tx, tz = px - x0, pz - z0
                v = ((1 - tx) * (1 - tz) * node(x0, z0, d) + tx * (1 - tz) * node(x0 + 1, z0, d) +
                     (1 - tx) * tz * node(x0, z0 + 1, d) + tx * tz * node(x0 + 1, z0 + 1, d))
                assert np.abs(S1[z, x, d] - v).max() < 1e-14


def test_lattice_aligned_directions_reduce_to_nearest(orc):
    """Horizontal lattice (x, y), directions in the plane (mu = 0) along the
    axes: every displacement is a lattice vector and bilinear streaming is the
    nearest-offset step, on a random scattering medium with mixed boundaries."""
    w = W.random_medium(9, 8, 1, 4, seed=5, n_phase=2, steps=6, bc=(2, 0, 1, 1))
    w.plane = "xy"
    Pn = oracle_problem(orc, w)
    w.scheme = "bilinear"
    Pb = oracle_problem(orc, w)
    assert np.array_equal(Pn.cx, [1, 0, -1, 0]) and np.array_equal(Pn.cz, [0, 1, 0, -1])
    S0 = W.random_state(w.nz, w.nx, w.n, seed=2)
    assert np.array_equal(Pn.run(S0, 6), Pb.run(S0, 6))


def test_xy_plane_n8_streams_along_the_axes(orc):
    """The paper's 2D runs (Sec. 3.2.1): 2 zenith x 4 azimuth directions on the
    horizontal lattice move only east / north / west / south."""
    mu, phi = orc.direction_grid(2, 4)
    cx, cz = orc.stream_offsets(mu, phi, orc.PLANE_XY)
    assert np.array_equal(cx, [1, 0, -1, 0] * 2) and np.array_equal(cz, [0, 1, 0, -1] * 2)
    ox, oz, w, lx, lz = orc.bilinear_taps(mu, phi, orc.PLANE_XY)
    assert np.allclose(np.abs(lx) + np.abs(lz), math.sqrt(0.75), atol=1e-15)
    assert (lx * lz == 0).all()


def test_uniform_inflow_fills_the_lattice(orc):
    """Periodic in x, inflow on top, vacuum below, no medium: directions moving
    down converge to the inflow vector everywhere, those moving up stay 0."""
    mu, phi = orc.direction_grid(2, 4)
    n = len(mu)
    inflow = np.zeros((4, n, 4))
    inflow[0, :, :] = [1.0, 0.2, -0.1, 0.05]
    P = _identity_problem(orc, 6, 5, mu, phi, 0, bc=(2, 0, 1, 1), inflow=inflow)
    S = P.run(P.zero_state(), 300)
    down = mu < 0
    assert np.abs(S[:, :, down] - inflow[0, 0]).max() < 1e-12
    assert np.abs(S[:, :, ~down]).max() == 0.0


def test_periodic_streaming_conserves_every_component(orc):
    mu = np.array([m for m, _ in DIRS])
    phi = np.array([p for _, p in DIRS])
    P = _identity_problem(orc, 8, 6, mu, phi, 0)
    S0 = np.random.default_rng(3).standard_normal((6, 8, len(mu), 4))
    S = P.run(S0, 25)
    assert np.abs(S.sum(axis=(0, 1)) - S0.sum(axis=(0, 1))).max() < 1e-12


def test_radiance_out_uses_the_sense_of_motion(orc):
    mu = np.array([0.3, -0.3, 0.0])
    phi = np.array([0.2, 0.2, 0.0])
    P = _identity_problem(orc, 4, 3, mu, phi, 0, bc=(0, 0, 0, 0))
    assert np.array_equal(P.cz, [1, -1, 0]) and np.array_equal(P.cx, [1, 1, 1])
    S = np.random.default_rng(1).uniform(0, 1, (3, 4, 3, 4))
    top = P.radiance_out(S, orc.SIDE_TOP)
    assert np.array_equal(top[:, 0], S[2, :, 0]) and not top[:, 1:].any()
