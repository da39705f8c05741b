"""Seeded synthetic inputs for the polarized lattice-Boltzmann RT step.

This module only draws input arrays (media, boundary Stokes vectors, initial
states) and names phase-matrix *parameters*; it holds none of the method's
arithmetic (no phase tables, no step coefficients, no streaming).  Both the CUDA
path and the FP64 oracle read their inputs from here.

Every floating-point medium array is rounded to float32 and returned as float64,
so the oracle (float64) and the CUDA library (float32 inputs) see identical
values.

Workloads (sizes follow the paper's lattice form: an (x, z) lattice, n
directions = n_zen x n_az, four Stokes components per direction):

- ``small``:      32x32, n=8 (2x4), tau 0.05, albedo 0.9, Rayleigh, emission 1e-3,
                  top beam I=1 on direction 0, vacuum elsewhere, 200 steps, seed 0.
- ``steady``:     512x512, n=32 (4x8), two-layer cloud medium (seed 0), run to a
                  residual below 1e-6 (cap 4000 steps).
- ``precision``:  2048x2048, n=64 (8x8), the same medium generator with seed 1,
                  1000 steps; error measured on the crop rows/cols [896, 1152).
- ``channels``:   256 independent spectral channels with mixed lattice sizes and
                  direction counts (seeded).
- ``adjoint``:    1024x256, n=32, medium seed 2, 1000 steps, loss on top I,Q,U.
- ``paper_2d``:   the paper's 16x16 horizontal-lattice runs (n=8, central source,
                  recycling or absorbing boundaries, 64 steps).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

SURV_LINEAR, SURV_EXP = 0, 1
ABS_BEER_LAMBERT, ABS_TAYLOR = 0, 1
BC_VACUUM, BC_PERIODIC, BC_INFLOW = 0, 1, 2
SIDE_TOP, SIDE_BOTTOM, SIDE_LEFT, SIDE_RIGHT = 0, 1, 2, 3


def _f32(a) -> np.ndarray:
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    nz: int
    n_zen: int
    n_az: int
    tau: np.ndarray                  # [nz][nx] per-step extinction optical depth
    albedo: np.ndarray               # [nz][nx] single-scattering albedo
    emission: Optional[np.ndarray]   # [nz][nx] per-step isotropic unpolarized emission
    phase_index: Optional[np.ndarray]  # [nz][nx] uint8 phase-class index
    phase_specs: List[Tuple]         # ("rayleigh",) | ("hg", g, pol_amp) | ("mix", m, g, pol_amp)
    bc: Tuple[int, int, int, int] = (BC_VACUUM,) * 4   # top, bottom, left, right
    inflow: Optional[np.ndarray] = None  # [4][n][4] ghost Stokes vectors per side
    surv_mode: int = SURV_LINEAR
    abs_mode: int = ABS_BEER_LAMBERT
    steps: int = 1
    seed: int = 0
    scheme: str = "nearest"          # streaming: "nearest" (D2Q9 offset) | "bilinear" (Eq. 34)
    plane: str = "xz"                # lattice plane the directions project on: "xz" | "xy"

    @property
    def n(self) -> int:
        return self.n_zen * self.n_az

    @property
    def sites(self) -> int:
        return self.nx * self.nz

    def crop(self, z0: int, z1: int, x0: int, x1: int, name: Optional[str] = None) -> "Workload":
        """The medium window [z0,z1) x [x0,x1) run as a problem of its own,
        with the same boundary kinds and inflow."""
        sl = (slice(z0, z1), slice(x0, x1))
        return dataclasses.replace(
            self, name=name or f"{self.name}_crop", nx=x1 - x0, nz=z1 - z0,
            tau=self.tau[sl].copy(), albedo=self.albedo[sl].copy(),
            emission=None if self.emission is None else self.emission[sl].copy(),
            phase_index=None if self.phase_index is None else self.phase_index[sl].copy())


def top_beam(n: int, direction: int = 0, stokes=(1.0, 0.0, 0.0, 0.0)) -> np.ndarray:
    """Inflow table [4][n][4] with a collimated beam entering through the top
    side on one direction; the other sides' ghost values are zero."""
    inflow = np.zeros((4, n, 4))
    inflow[SIDE_TOP, direction] = stokes
    return inflow


def random_state(nz: int, nx: int, n: int, seed: int, scale: float = 1.0,
                 dtype=np.float64) -> np.ndarray:
    """A physically realizable random Stokes field S[z][x][d][4]: I >= |(Q,U,V)|.
    Values are float32-representable; ``dtype=np.float32`` skips the float64
    temporaries for large lattices (same values)."""
    rng = np.random.default_rng(seed)
    out = np.empty((nz, nx, n, 4), np.float32)
    rows = max(1, (1 << 22) // max(1, nx * n))
    for z0 in range(0, nz, rows):
        z1 = min(nz, z0 + rows)
        shp = (z1 - z0, nx, n)
        I = rng.uniform(0.1, 1.0, shp).astype(np.float32) * np.float32(scale)
        v = rng.standard_normal(shp + (3,), dtype=np.float32)
        v /= np.linalg.norm(v, axis=-1, keepdims=True)
        p = rng.uniform(0.0, 1.0, shp).astype(np.float32)
        out[z0:z1, ..., 0] = I
        out[z0:z1, ..., 1:] = (I * p * np.float32(0.999))[..., None] * v
    return out if dtype == np.float32 else out.astype(dtype)


def _gaussian_smooth(field: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(field, sigma=sigma, mode="reflect")


def cloud_medium(nx: int, nz: int, seed: int):
    """Two-layer medium: clear air (upper half, optical depth 0.01 per cell,
    albedo 0.8, Rayleigh class 0) over a cloud layer (lower half, log-normal
    optical depth with median 0.2 and sigma 0.5, spatially correlated by a
    Gaussian filter of 16 cells, albedo 0.95, Henyey-Greenstein class 1)."""
    rng = np.random.default_rng(seed)
    g = _gaussian_smooth(rng.standard_normal((nz, nx)), 16.0)
    cloud = np.zeros((nz, nx), bool)
    cloud[: nz // 2] = True
    gc = g[cloud]
    g = (g - gc.mean()) / gc.std()
    tau = np.where(cloud, np.exp(math.log(0.2) + 0.5 * g), 0.01)
    albedo = np.where(cloud, 0.95, 0.8)
    cls = np.where(cloud, 1, 0).astype(np.uint8)
    return _f32(tau), _f32(albedo), cls


CLOUD_SPECS = [("rayleigh",), ("hg", 0.85, -0.1)]


def small(steps: int = 200) -> Workload:
    nx = nz = 32
    n = 8
    return Workload("lattice32_n8_fp64ref", nx, nz, 2, 4,
                    tau=_f32(np.full((nz, nx), 0.05)), albedo=_f32(np.full((nz, nx), 0.9)),
                    emission=_f32(np.full((nz, nx), 1e-3)), phase_index=None,
                    phase_specs=[("rayleigh",)], inflow=top_beam(n),
                    bc=(BC_INFLOW, BC_VACUUM, BC_VACUUM, BC_VACUUM),
                    surv_mode=SURV_LINEAR, steps=steps, seed=0)


def cloud(name: str, nx: int, nz: int, n_zen: int, n_az: int, seed: int, steps: int) -> Workload:
    tau, albedo, cls = cloud_medium(nx, nz, seed)
    n = n_zen * n_az
    return Workload(name, nx, nz, n_zen, n_az, tau=tau, albedo=albedo, emission=None,
                    phase_index=cls, phase_specs=list(CLOUD_SPECS), inflow=top_beam(n),
                    bc=(BC_INFLOW, BC_VACUUM, BC_VACUUM, BC_VACUUM),
                    surv_mode=SURV_EXP, steps=steps, seed=seed)


def steady(seed: int = 0) -> Workload:
    return cloud("lattice512_n32_steady", 512, 512, 4, 8, seed, 4000)


def precision(seed: int = 1, steps: int = 1000) -> Workload:
    return cloud("lattice2048_n64", 2048, 2048, 8, 8, seed, steps)


PRECISION_CROP = (896, 1152, 896, 1152)


def precision_crop(seed: int = 1, steps: int = 1000) -> Workload:
    return precision(seed, steps).crop(*PRECISION_CROP, name="lattice2048_n64_crop256")


def adjoint(seed: int = 2, steps: int = 1000) -> Workload:
    return cloud("lattice1024x256_n32_adjoint", 1024, 256, 4, 8, seed, steps)


def channels(count: int = 256, seed: int = 3, steps: int = 500) -> List[Workload]:
    """Independent spectral channels: lattice from {64,128,256,512} x
    {64,128,256}, n from {8,16,32}, optical-depth scale log-uniform in
    [0.01, 1], albedo uniform in [0.5, 0.999], and a Rayleigh/HG mixture with
    weight m ~ U[0,1] and g ~ U[0,0.9]."""
    rng = np.random.default_rng(seed)
    split = {8: (2, 4), 16: (4, 4), 32: (4, 8)}
    out = []
    for c in range(count):
        nx = int(rng.choice([64, 128, 256, 512]))
        nz = int(rng.choice([64, 128, 256]))
        n = int(rng.choice([8, 16, 32]))
        scale = math.exp(rng.uniform(math.log(0.01), math.log(1.0)))
        w0 = rng.uniform(0.5, 0.999)
        m, g = rng.uniform(0.0, 1.0), rng.uniform(0.0, 0.9)
        tau, _, _ = cloud_medium(nx, nz, seed * 1000 + c)
        nzen, naz = split[n]
        out.append(Workload(f"channel{c}", nx, nz, nzen, naz, tau=_f32(tau * scale),
                            albedo=_f32(np.full((nz, nx), w0)), emission=None, phase_index=None,
                            phase_specs=[("mix", m, g, -0.1)], inflow=top_beam(n),
                            bc=(BC_INFLOW, BC_VACUUM, BC_VACUUM, BC_VACUUM),
                            surv_mode=SURV_EXP, steps=steps, seed=seed))
    return out


def paper_2d(bc: str = "recycle", scheme: str = "nearest", steps: int = 64) -> Workload:
    """The paper's 2D runs (Sec. 3.2.1, Figs. 10-12): a horizontal 16x16
    lattice, 2 zenith x 4 azimuth directions, Rayleigh scattering, Beer-Lambert
    absorption, k_ext = 2.5 and k_scat = 0.5 with dt = 1/16 (tau = 2.5/16,
    albedo 0.2), an unpolarized source J = 1 shared equally by the directions
    on the four central sites (e = dt J / 8 per direction and step), recycling
    ("recycle") or absorbing ("absorb") boundaries, 64 steps."""
    N = 16
    em = np.zeros((N, N))
    em[7:9, 7:9] = 1.0 / 16 / 8
    kind = BC_PERIODIC if bc == "recycle" else BC_VACUUM
    return Workload(f"paper2d_{bc}_{scheme}", N, N, 2, 4, tau=_f32(np.full((N, N), 2.5 / 16)),
                    albedo=_f32(np.full((N, N), 0.2)), emission=_f32(em), phase_index=None,
                    phase_specs=[("rayleigh",)], inflow=None, bc=(kind,) * 4, surv_mode=SURV_LINEAR,
                    steps=steps, seed=0, scheme=scheme, plane="xy")


def random_medium(nx: int, nz: int, n_zen: int, n_az: int, seed: int, n_phase: int = 2,
                  bc=(BC_INFLOW, BC_VACUUM, BC_VACUUM, BC_VACUUM), steps: int = 5,
                  surv_mode: int = SURV_EXP, emission: bool = True) -> Workload:
    """Unstructured random medium for parity edge cases (odd sizes, mixed phase
    classes per tile, all boundary kinds)."""
    rng = np.random.default_rng(seed)
    n = n_zen * n_az
    tau = rng.uniform(0.0, 1.5, (nz, nx))
    albedo = rng.uniform(0.0, 1.0, (nz, nx))
    em = rng.uniform(0.0, 1e-2, (nz, nx)) if emission else None
    cls = rng.integers(0, n_phase, (nz, nx)).astype(np.uint8)
    specs = [("rayleigh",), ("hg", 0.85, -0.1), ("hg", 0.5, -0.05), ("mix", 0.3, 0.7, -0.1)][:n_phase]
    inflow = np.zeros((4, n, 4))
    for side in range(4):
        if bc[side] == BC_INFLOW:
            I = rng.uniform(0.5, 1.0, n)
            q = rng.uniform(-0.3, 0.3, (n, 3))
            inflow[side] = np.concatenate([I[:, None], q * I[:, None]], 1)
    return Workload(f"random{nx}x{nz}_n{n}", nx, nz, n_zen, n_az, tau=_f32(tau),
                    albedo=_f32(albedo), emission=None if em is None else _f32(em),
                    phase_index=cls, phase_specs=specs, bc=tuple(bc), inflow=_f32(inflow),
                    surv_mode=surv_mode, steps=steps, seed=seed)
