"""FP64 CPU oracle for the polarized lattice-Boltzmann radiative-transfer step.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library; the C source (``rtlb_oracle.c``) documents the readings of the
paper it fixes.  This module only marshals numpy arrays into that library.

State layout: ``S[z][x][d][s]`` float64, s = (I, Q, U, V), d = i_zen * n_az + i_az.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SURV_LINEAR, SURV_EXP = 0, 1
ABS_BEER_LAMBERT, ABS_TAYLOR = 0, 1
BC_VACUUM, BC_PERIODIC, BC_INFLOW = 0, 1, 2
SIDE_TOP, SIDE_BOTTOM, SIDE_LEFT, SIDE_RIGHT = 0, 1, 2, 3
PHASE_RAYLEIGH, PHASE_HG, PHASE_RAYLEIGH_DEPOL = 0, 1, 2
PLANE_XZ, PLANE_XY = 0, 1

_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    """Load (building on first use) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_direction_grid.argtypes = [C.c_int, C.c_int, _dp, _dp]
        L.orc_stream_offset.argtypes = [C.c_double, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_stream_offset.restype = C.c_int
        L.orc_plane_offset.argtypes = [C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_plane_offset.restype = C.c_int
        L.orc_lattice_projection.argtypes = [C.c_double, C.c_double, C.c_int, C.POINTER(C.c_double),
                                             C.POINTER(C.c_double)]
        L.orc_bilinear_taps.argtypes = [C.c_double, C.c_double, C.c_int, _ip, _ip, _dp,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_rotation.argtypes = [C.c_double, _dp]
        L.orc_rayleigh_matrix.argtypes = [C.c_double, _dp]
        L.orc_hg_matrix.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
        L.orc_rpr_block.argtypes = [C.c_double] * 4 + [C.c_int, C.c_double, C.c_double, _dp,
                                                       C.POINTER(C.c_double)]
        L.orc_phase_table.argtypes = [C.c_int, _dp, _dp, C.c_int, C.c_double, C.c_double, _dp]
        step_args = [C.c_int, C.c_int, C.c_int, C.c_int, _ip, _ip, _dp, _dp, _dp, C.c_void_p, C.c_void_p,
                     _dp, C.c_int, C.c_int, _ip, _dp]
        L.orc_step.argtypes = step_args + [_dp, _dp]
        L.orc_run.argtypes = step_args + [_dp, C.c_int]
        L.orc_step_fp8.argtypes = step_args[:12] + [C.c_int] + step_args[12:] + [_dp, _dp]
        L.orc_step_fp8x.argtypes = step_args[:12] + [C.c_int] + step_args[12:] + [_dp, _dp]
        L.orc_e4m3.argtypes = [C.c_double]
        L.orc_e4m3.restype = C.c_double
        L.orc_fp8_exponent.argtypes = [C.c_double, C.c_int]
        L.orc_fp8_exponent.restype = C.c_int
        L.orc_run_to_steady.argtypes = step_args + [_dp, C.c_double, C.c_int, C.POINTER(C.c_double)]
        L.orc_run_to_steady.restype = C.c_int
        L.orc_residual.argtypes = [C.c_size_t, _dp, _dp]
        L.orc_residual.restype = C.c_double
        L.orc_radiance_out.argtypes = [C.c_int, C.c_int, C.c_int, _ip, _ip, C.c_int, _dp, _dp]
        L.orc_dop.argtypes = [_dp]
        L.orc_dop.restype = C.c_double
        L.orc_num_threads.restype = C.c_int
        L.orc_rayleigh_depol_matrix.argtypes = [C.c_double, C.c_double, _dp]
        L.orc_conserve_intensity.argtypes = [C.c_int, _dp]
        L.orc_adjoint.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _ip, _ip, _dp, _ip, _dp, _dp,
                                  C.c_void_p, C.c_void_p, _dp, C.c_int, C.c_int, C.c_int, _ip, _dp, _dp,
                                  C.c_int, _dp, _dp, _dp, _dp, C.c_void_p]
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().orc_num_threads()


# ------------------------------------------------------------------ geometry

def direction_grid(n_zen: int, n_az: int):
    """(mu, phi) of the uniform n_zen x n_az grid, float64 arrays of length n."""
    n = n_zen * n_az
    mu, phi = np.zeros(n), np.zeros(n)
    lib().orc_direction_grid(n_zen, n_az, mu, phi)
    return mu, phi


def stream_offsets(mu, phi, plane=PLANE_XZ):
    """Integer D2Q9 offsets (cx, cz) per direction; raises on a tie."""
    n = len(mu)
    cx, cz = np.zeros(n, np.int32), np.zeros(n, np.int32)
    for d in range(n):
        a, b = C.c_int(), C.c_int()
        if lib().orc_plane_offset(float(mu[d]), float(phi[d]), int(plane), C.byref(a), C.byref(b)):
            raise ValueError(f"direction {d} lies exactly between two lattice offsets")
        cx[d], cz[d] = a.value, b.value
    return cx, cz


def lattice_projection(mu, phi, plane=PLANE_XZ):
    """(px, pz) arrays: each direction's projection on the lattice plane."""
    px, pz = np.zeros(len(mu)), np.zeros(len(mu))
    for d in range(len(mu)):
        a, b = C.c_double(), C.c_double()
        lib().orc_lattice_projection(float(mu[d]), float(phi[d]), int(plane), C.byref(a), C.byref(b))
        px[d], pz[d] = a.value, b.value
    return px, pz


def bilinear_taps(mu, phi, plane=PLANE_XZ):
    """Semi-Lagrangian taps (Eq. 33-34): offsets ox, oz [n][4] (int32),
    weights w [n][4] and the displacement lx, lz [n]."""
    n = len(mu)
    ox, oz, w = np.zeros((n, 4), np.int32), np.zeros((n, 4), np.int32), np.zeros((n, 4))
    lx, lz = np.zeros(n), np.zeros(n)
    for d in range(n):
        a, b, c = np.zeros(4, np.int32), np.zeros(4, np.int32), np.zeros(4)
        x, z = C.c_double(), C.c_double()
        lib().orc_bilinear_taps(float(mu[d]), float(phi[d]), int(plane), a, b, c, C.byref(x), C.byref(z))
        ox[d], oz[d], w[d], lx[d], lz[d] = a, b, c, x.value, z.value
    return ox, oz, w, lx, lz


def rotation(psi: float) -> np.ndarray:
    R = np.zeros(16)
    lib().orc_rotation(float(psi), R)
    return R.reshape(4, 4)


def rayleigh_matrix(cos_t: float) -> np.ndarray:
    P = np.zeros(16)
    lib().orc_rayleigh_matrix(float(cos_t), P)
    return P.reshape(4, 4)


def hg_matrix(cos_t: float, g: float, pol_amp: float) -> np.ndarray:
    P = np.zeros(16)
    lib().orc_hg_matrix(float(cos_t), float(g), float(pol_amp), P)
    return P.reshape(4, 4)


def rayleigh_depol_matrix(cos_t: float, rho: float) -> np.ndarray:
    P = np.zeros(16)
    lib().orc_rayleigh_depol_matrix(float(cos_t), float(rho), P)
    return P.reshape(4, 4)


def conserve_intensity(Z) -> np.ndarray:
    """Intensity-conserving copy of a normalized table (see the C source)."""
    Z = np.array(Z, np.float64, order="C", copy=True)
    lib().orc_conserve_intensity(Z.shape[0] // 4, Z)
    return Z


def rpr_block(mu_o, phi_o, mu_i, phi_i, kind=PHASE_RAYLEIGH, g=0.0, pol_amp=0.0):
    """Un-normalized rotation-phase-rotation block M(o, i) and its scalar weight."""
    M = np.zeros(16)
    w = C.c_double()
    lib().orc_rpr_block(float(mu_o), float(phi_o), float(mu_i), float(phi_i), int(kind),
                        float(g), float(pol_amp), M, C.byref(w))
    return M.reshape(4, 4), w.value


def phase_table(mu, phi, kind=PHASE_RAYLEIGH, g=0.0, pol_amp=0.0) -> np.ndarray:
    """Normalized 4n x 4n redistribution table Z (row = outgoing, col = incoming)."""
    n = len(mu)
    Z = np.zeros((4 * n) * (4 * n))
    lib().orc_phase_table(n, np.ascontiguousarray(mu, np.float64),
                          np.ascontiguousarray(phi, np.float64), int(kind), float(g),
                          float(pol_amp), Z)
    return Z.reshape(4 * n, 4 * n)


def phase_table_spec(mu, phi, spec) -> np.ndarray:
    """Table for a phase-class spec tuple: ("rayleigh",) or ("rayleigh", rho)
    with depolarization factor rho, ("hg", g, pol_amp) or ("mix", m, g,
    pol_amp) = m * rayleigh + (1 - m) * hg (both normalized)."""
    kind = spec[0]
    if kind == "rayleigh":
        if len(spec) > 1 and spec[1]:
            return phase_table(mu, phi, PHASE_RAYLEIGH_DEPOL, spec[1])
        return phase_table(mu, phi, PHASE_RAYLEIGH)
    if kind == "hg":
        return phase_table(mu, phi, PHASE_HG, spec[1], spec[2])
    if kind == "mix":
        m = spec[1]
        return m * phase_table(mu, phi, PHASE_RAYLEIGH) + (1 - m) * phase_table(
            mu, phi, PHASE_HG, spec[2], spec[3])
    raise ValueError(f"unknown phase spec {spec!r}")


# ------------------------------------------------------------------ solver

class Problem:
    """Medium, geometry and boundaries of one lattice, in oracle form (float64).

    scheme "nearest" streams each direction to its nearest D2Q9 offset;
    "bilinear" uses the four weighted translations of Eq. 34.  plane selects
    the lattice plane the directions are projected on (PLANE_XZ or PLANE_XY).
    """

    def __init__(self, nx, nz, mu, phi, tau, albedo, emission, cls, Z,
                 surv_mode=SURV_LINEAR, abs_mode=ABS_BEER_LAMBERT,
                 bc=(BC_VACUUM,) * 4, inflow=None, offsets=None, scheme="nearest", plane=PLANE_XZ):
        self.nx, self.nz, self.n = int(nx), int(nz), len(mu)
        self.mu = np.ascontiguousarray(mu, np.float64)
        self.phi = np.ascontiguousarray(phi, np.float64)
        self.scheme, self.plane = scheme, int(plane)
        if scheme == "nearest":
            cx, cz = offsets if offsets is not None else stream_offsets(self.mu, self.phi, self.plane)
            self.cx = np.ascontiguousarray(cx, np.int32)
            self.cz = np.ascontiguousarray(cz, np.int32)
            self.ntap = 1
            self.tx, self.tz = self.cx.copy(), self.cz.copy()
            self.tw = np.ones(self.n)
        elif scheme == "bilinear":
            ox, oz, w, lx, lz = bilinear_taps(self.mu, self.phi, self.plane)
            self.ntap = 4
            self.tx = np.ascontiguousarray(ox.ravel(), np.int32)
            self.tz = np.ascontiguousarray(oz.ravel(), np.int32)
            self.tw = np.ascontiguousarray(w.ravel(), np.float64)
            # sense of motion per axis, for the readout and the adjoint seed
            self.cx = np.ascontiguousarray(np.sign(lx), np.int32)
            self.cz = np.ascontiguousarray(np.sign(lz), np.int32)
        else:
            raise ValueError(f"unknown streaming scheme {scheme!r}")
        shp = (self.nz, self.nx)
        own = lambda a, dt: np.array(np.broadcast_to(a, shp), dt, order="C", copy=True)
        self.tau = own(tau, np.float64)
        self.albedo = own(albedo, np.float64)
        self.emission = None if emission is None else own(emission, np.float64)
        self.cls = None if cls is None else own(cls, np.int32)
        Z = np.array(Z, np.float64, copy=True)
        if Z.ndim == 2:
            Z = Z[None]
        self.Z = np.ascontiguousarray(Z)
        assert self.Z.shape[1:] == (4 * self.n, 4 * self.n)
        self.surv_mode, self.abs_mode = int(surv_mode), int(abs_mode)
        self.bc = np.ascontiguousarray(bc, np.int32)
        if (self.bc[SIDE_TOP] == BC_PERIODIC) != (self.bc[SIDE_BOTTOM] == BC_PERIODIC) or \
           (self.bc[SIDE_LEFT] == BC_PERIODIC) != (self.bc[SIDE_RIGHT] == BC_PERIODIC):
            raise ValueError("periodic boundaries must be set on both sides of an axis")
        self.inflow = np.zeros((4, self.n, 4)) if inflow is None else np.array(inflow, np.float64)
        self.inflow = np.ascontiguousarray(self.inflow.reshape(4, self.n, 4))

    def _args(self):
        e = self.emission.ctypes.data if self.emission is not None else None
        c = self.cls.ctypes.data if self.cls is not None else None
        return (self.nx, self.nz, self.n, self.ntap, self.tx, self.tz, self.tw, self.tau, self.albedo, e, c,
                self.Z, self.surv_mode, self.abs_mode, self.bc, self.inflow)

    def zero_state(self) -> np.ndarray:
        return np.zeros((self.nz, self.nx, self.n, 4))

    def step(self, S: np.ndarray) -> np.ndarray:
        S = np.ascontiguousarray(S, np.float64)
        out = np.empty_like(S)
        lib().orc_step(*self._args(), S, out)
        return out

    def step_fp8(self, S: np.ndarray) -> np.ndarray:
        """One step in the FP8 block-scaled form of the contraction (see
        orc_step_fp8); S must hold float32 values."""
        S = np.ascontiguousarray(S, np.float64)
        out = np.empty_like(S)
        a = self._args()
        lib().orc_step_fp8(*a[:12], int(self.Z.shape[0]), *a[12:], S, out)
        return out

    def step_fp8x(self, S: np.ndarray) -> np.ndarray:
        """One step in the split FP8 form of the contraction (see
        orc_step_fp8x: an emulation of that form); S must hold float32
        values."""
        S = np.ascontiguousarray(S, np.float64)
        out = np.empty_like(S)
        a = self._args()
        lib().orc_step_fp8x(*a[:12], int(self.Z.shape[0]), *a[12:], S, out)
        return out

    def run(self, S: np.ndarray, nsteps: int) -> np.ndarray:
        S = np.array(S, np.float64, order="C", copy=True)
        lib().orc_run(*self._args(), S, int(nsteps))
        return S

    def run_to_steady(self, S, tol, max_steps):
        S = np.array(S, np.float64, order="C", copy=True)
        r = C.c_double()
        t = lib().orc_run_to_steady(*self._args(), S, float(tol), int(max_steps), C.byref(r))
        return S, t, r.value

    def adjoint(self, S0, nsteps, dL_dout, want_S0=False):
        """Gradients of L = <dL_dout, radiance_out(top, S^N)> (S^N after
        nsteps steps from S0) w.r.t. tau [nz][nx], albedo [nz][nx], the phase
        tables [n_phase][4n][4n] and (optionally) S0."""
        S0 = np.ascontiguousarray(S0, np.float64)
        dl = np.ascontiguousarray(dL_dout, np.float64).reshape(self.nx, self.n, 4)
        gt = np.zeros((self.nz, self.nx))
        ga = np.zeros((self.nz, self.nx))
        gZ = np.zeros_like(self.Z)
        gS = np.zeros_like(S0) if want_S0 else None
        e = self.emission.ctypes.data if self.emission is not None else None
        c = self.cls.ctypes.data if self.cls is not None else None
        lib().orc_adjoint(self.nx, self.nz, self.n, self.ntap, self.tx, self.tz, self.tw, self.cz,
                          self.tau, self.albedo, e, c,
                          self.Z, self.Z.shape[0], self.surv_mode, self.abs_mode, self.bc, self.inflow,
                          S0, int(nsteps), dl, gt, ga, gZ, gS.ctypes.data if want_S0 else None)
        return (gt, ga, gZ, gS) if want_S0 else (gt, ga, gZ)

    def radiance_out(self, S, side=SIDE_TOP) -> np.ndarray:
        S = np.ascontiguousarray(S, np.float64)
        ln = self.nx if side in (SIDE_TOP, SIDE_BOTTOM) else self.nz
        out = np.zeros((ln, self.n, 4))
        lib().orc_radiance_out(self.nx, self.nz, self.n, self.cx, self.cz, int(side), S, out)
        return out


def e4m3(x: float) -> float:
    """Nearest e4m3 value (ties to even, saturating at +-448)."""
    return float(lib().orc_e4m3(float(x)))


def fp8_exponent(amax: float, fp32_floor: bool = False) -> int:
    """UE8M0 block exponent: smallest e with amax / 2^e <= 448, in [-127, 127]."""
    return int(lib().orc_fp8_exponent(float(amax), int(bool(fp32_floor))))


def residual(S_old, S_new) -> float:
    a = np.ascontiguousarray(S_old, np.float64).ravel()
    b = np.ascontiguousarray(S_new, np.float64).ravel()
    return lib().orc_residual(a.size, a, b)


def dop(stokes) -> np.ndarray:
    """Degree of polarization of (..., 4) Stokes arrays (vectorised for tests)."""
    s = np.asarray(stokes, np.float64)
    if s.ndim == 1:
        return lib().orc_dop(np.ascontiguousarray(s))
    p = np.sqrt(s[..., 1] ** 2 + s[..., 2] ** 2 + s[..., 3] ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(s[..., 0] != 0, p / s[..., 0], 0.0)
