"""Shared test helpers: build oracle problems from seeded workloads and
compare Stokes fields."""
import numpy as np


def oracle_problem(orc, w, offsets=None):
    """FP64 oracle problem for a Workload (tables built by the oracle itself)."""
    mu, phi = orc.direction_grid(w.n_zen, w.n_az)
    Z = np.stack([orc.phase_table_spec(mu, phi, s) for s in w.phase_specs])
    cls = None if w.phase_index is None else w.phase_index.astype(np.int32)
    return orc.Problem(w.nx, w.nz, mu, phi, w.tau, w.albedo, w.emission, cls, Z,
                       surv_mode=w.surv_mode, abs_mode=w.abs_mode, bc=w.bc,
                       inflow=w.inflow, offsets=offsets, scheme=w.scheme,
                       plane={"xz": orc.PLANE_XZ, "xy": orc.PLANE_XY}[w.plane])


def rel_err_I(S, R, floor_frac=1e-6):
    """Elementwise relative error of the I component against the reference R,
    with entries below floor_frac * max|I_ref| compared against that floor."""
    I, Ir = S[..., 0], R[..., 0]
    floor = floor_frac * np.abs(Ir).max() + 1e-300
    return float(np.max(np.abs(I - Ir) / np.maximum(np.abs(Ir), floor)))


def dop(S):
    p = np.sqrt(S[..., 1] ** 2 + S[..., 2] ** 2 + S[..., 3] ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(S[..., 0] > 0, p / np.where(S[..., 0] > 0, S[..., 0], 1), 0.0)


def abs_err_dop(S, R, floor_frac=1e-6):
    """Max absolute DOP error over entries whose reference I is above the floor."""
    mask = R[..., 0] > floor_frac * np.abs(R[..., 0]).max()
    return float(np.max(np.abs(dop(S) - dop(R))[mask])) if mask.any() else 0.0
