"""The synthetic inputs follow their stated recipe: the two-layer cloud medium
(clear air over a log-normal cloud, correlated over 16 cells), the small
Rayleigh lattice, the 256 spectral channels and the top beam.  Every medium
value is float32-representable, so the oracle and the library see the same
numbers."""
import math

import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W


def _f32_exact(a):
    a = np.asarray(a)
    return np.array_equal(a.astype(np.float32).astype(a.dtype), a)


@pytest.mark.parametrize("nx,nz,seed", [(512, 512, 0), (1024, 256, 2), (256, 192, 1)])
def test_cloud_medium_recipe(nx, nz, seed):
    tau, alb, cls = W.cloud_medium(nx, nz, seed)
    assert tau.shape == alb.shape == cls.shape == (nz, nx)
    cloud = np.zeros((nz, nx), bool)
    cloud[: nz // 2] = True                     # z increases upward: the cloud is the lower half
    assert np.all(cls[cloud] == 1) and np.all(cls[~cloud] == 0)
    assert np.all(tau[~cloud] == np.float32(0.01)) and np.all(alb[~cloud] == np.float32(0.8))
    assert np.all(alb[cloud] == np.float32(0.95))
    lg = np.log(tau[cloud].astype(np.float64))
    # re-standardized over the cloud cells: ln tau has mean ln 0.2 and std 0.5
    # (up to the float32 rounding of tau)
    assert abs(lg.mean() - math.log(0.2)) < 1e-6 and abs(lg.std() - 0.5) < 1e-6
    assert _f32_exact(tau) and _f32_exact(alb)
    # spatial correlation over ~16 cells: neighbours are strongly correlated,
    # cells 64 apart much less
    z = (lg.reshape(nz // 2, nx) - lg.mean()) / lg.std()
    c1 = np.mean(z[:, 1:] * z[:, :-1])
    c64 = np.mean(z[:, 64:] * z[:, :-64])
    assert c1 > 0.95 and abs(c64) < 0.5


def test_same_seed_same_medium():
    a = W.cloud_medium(256, 128, 3)
    b = W.cloud_medium(256, 128, 3)
    c = W.cloud_medium(256, 128, 4)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])


def test_small_lattice_recipe():
    w = W.small()
    assert (w.nx, w.nz, w.n) == (32, 32, 8) and w.steps == 200
    assert np.all(w.tau == np.float32(0.05)) and np.all(w.albedo == np.float32(0.9))
    assert np.all(w.emission == np.float32(1e-3)) and w.phase_specs == [("rayleigh",)]
    assert w.bc == (W.BC_INFLOW, W.BC_VACUUM, W.BC_VACUUM, W.BC_VACUUM) and w.surv_mode == W.SURV_LINEAR


def test_top_beam():
    b = W.top_beam(8)
    assert b.shape == (4, 8, 4)
    want = np.zeros((4, 8, 4))
    want[0, 0] = (1.0, 0.0, 0.0, 0.0)           # side 0 is the top; direction 0 points down
    assert np.array_equal(b, want)


def test_channels_recipe():
    ws = W.channels(count=256, steps=10)
    assert len(ws) == 256
    split = {8: (2, 4), 16: (4, 4), 32: (4, 8)}
    for w in ws:
        assert w.nx in (64, 128, 256, 512) and w.nz in (64, 128, 256)
        assert (w.n_zen, w.n_az) == split[w.n]
        a = float(w.albedo[0, 0])
        assert np.all(w.albedo == w.albedo[0, 0]) and 0.5 <= a <= 0.999
        (kind, m, g, pol), = w.phase_specs
        assert kind == "mix" and 0.0 <= m <= 1.0 and 0.0 <= g <= 0.9
        assert w.phase_index is None and _f32_exact(w.tau)
    # every direction count and lattice size occurs
    assert {w.n for w in ws} == {8, 16, 32}
    assert {w.nx for w in ws} == {64, 128, 256, 512} and {w.nz for w in ws} == {64, 128, 256}
