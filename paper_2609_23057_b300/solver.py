"""Python face of librtlb: a thin wrapper that hands torch / numpy buffers to
the C ABI.  torch is used for device memory and streams only; every step of
the solver runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import Directions, Grid, Options, check, lib

PRECISIONS = {"fp32": 0, "bf16": 1, "bf16x3": 2, "bf16x2": 3, "fp8": 4, "tf32x3": 5, "fp8x": 6}
SURVIVAL = {"linear": 0, "exp": 1}
ABSORPTION = {"beer_lambert": 0, "taylor": 1}
SIDES = {"top": 0, "bottom": 1, "left": 2, "right": 3}
BCS = {"vacuum": 0, "periodic": 1, "inflow": 2}
STREAMING = {"nearest": 0, "bilinear": 1}
PLANES = {"xz": 0, "xy": 1}


def _dirs(n_zen: int, n_az: int, mu=None, phi=None):
    d = Directions(n_zen, n_az, None, None)
    keep = None
    if mu is not None:
        mu = np.ascontiguousarray(mu, np.float64)
        phi = np.ascontiguousarray(phi, np.float64)
        d.mu = mu.ctypes.data_as(C.POINTER(C.c_double))
        d.phi = phi.ctypes.data_as(C.POINTER(C.c_double))
        keep = (mu, phi)
    return d, keep


def stream_offsets(n_zen: int, n_az: int, mu=None, phi=None):
    """(cx, cz) int32 arrays of the library's D2Q9 streaming offsets."""
    n = n_zen * n_az
    d, keep = _dirs(n_zen, n_az, mu, phi)
    cx, cz = np.zeros(n, np.int32), np.zeros(n, np.int32)
    check(lib().rtlb_stream_offsets(C.byref(d), cx.ctypes.data, cz.ctypes.data))
    return cx, cz


def stream_taps(n_zen: int, n_az: int, streaming: str = "bilinear", plane: str = "xz", mu=None, phi=None):
    """(ox, oz, w) [n][4] of the library's streaming taps (rtlb_stream_taps)."""
    n = n_zen * n_az
    d, keep = _dirs(n_zen, n_az, mu, phi)
    ox, oz, w = np.zeros((n, 4), np.int32), np.zeros((n, 4), np.int32), np.zeros((n, 4))
    check(lib().rtlb_stream_taps(C.byref(d), STREAMING[streaming], PLANES[plane], ox.ctypes.data, oz.ctypes.data,
                                 w.ctypes.data))
    return ox, oz, w


def phase_rayleigh(n_zen: int, n_az: int, mu=None, phi=None, depol: float = 0.0) -> np.ndarray:
    n = n_zen * n_az
    d, keep = _dirs(n_zen, n_az, mu, phi)
    Z = np.zeros((4 * n, 4 * n))
    check(lib().rtlb_phase_rayleigh(C.byref(d), float(depol), Z.ctypes.data))
    return Z


def conserve_intensity(Z) -> np.ndarray:
    """Intensity-conserving copy of a normalized table (rtlb_phase_conserve_intensity)."""
    Z = np.array(Z, np.float64, order="C", copy=True)
    check(lib().rtlb_phase_conserve_intensity(Z.shape[0] // 4, Z.ctypes.data))
    return Z


def phase_hg(n_zen: int, n_az: int, g: float, pol_amp: float, mu=None, phi=None, with_dg=False):
    n = n_zen * n_az
    d, keep = _dirs(n_zen, n_az, mu, phi)
    Z = np.zeros((4 * n, 4 * n))
    dZ = np.zeros((4 * n, 4 * n)) if with_dg else None
    check(lib().rtlb_phase_hg(C.byref(d), float(g), float(pol_amp), Z.ctypes.data,
                              dZ.ctypes.data if with_dg else None))
    return (Z, dZ) if with_dg else Z


def phase_hg_grad(n_zen: int, n_az: int, g: float, pol_amp: float, grad_Z, mu=None, phi=None) -> float:
    """dL/dg from dL/dZ of an HG table (rtlb_phase_hg_grad)."""
    d, keep = _dirs(n_zen, n_az, mu, phi)
    gZ = np.ascontiguousarray(grad_Z, np.float64)
    out = C.c_double()
    check(lib().rtlb_phase_hg_grad(C.byref(d), float(g), float(pol_amp), gZ.ctypes.data, C.byref(out)))
    return out.value


def phase_mix(n_zen: int, n_az: int, m: float, g: float, pol_amp: float, mu=None, phi=None):
    n = n_zen * n_az
    d, keep = _dirs(n_zen, n_az, mu, phi)
    Z = np.zeros((4 * n, 4 * n))
    check(lib().rtlb_phase_mix(C.byref(d), float(m), float(g), float(pol_amp), Z.ctypes.data))
    return Z


def phase_table_spec(n_zen: int, n_az: int, spec, mu=None, phi=None) -> np.ndarray:
    """Library table for a phase-class spec: ("rayleigh",), ("rayleigh", rho),
    ("hg", g, pol_amp), ("mix", m, g, pol_amp)."""
    if spec[0] == "rayleigh":
        return phase_rayleigh(n_zen, n_az, mu, phi, depol=spec[1] if len(spec) > 1 else 0.0)
    if spec[0] == "hg":
        return phase_hg(n_zen, n_az, spec[1], spec[2], mu, phi)
    if spec[0] == "mix":
        return phase_mix(n_zen, n_az, spec[1], spec[2], spec[3], mu, phi)
    raise ValueError(f"unknown phase spec {spec!r}")


def _ptr(a):
    """Raw pointer of a torch tensor (device or host) or numpy array; the
    caller keeps the object alive for the duration of the call."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Solver:
    """One lattice, one medium, one state, on the current CUDA device."""

    def __init__(self, nx: int, nz: int, n_zen: int, n_az: int, precision: str = "fp32",
                 survival: str = "linear", absorption: str = "beer_lambert", mu=None, phi=None,
                 streaming: str = "nearest", plane: str = "xz"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("librtlb needs a CUDA device")
        self.nx, self.nz, self.n_zen, self.n_az = nx, nz, n_zen, n_az
        self.n = n_zen * n_az
        self.precision = precision
        self.streaming, self.plane = streaming, plane
        d, self._keep = _dirs(n_zen, n_az, mu, phi)
        opts = Options(PRECISIONS[precision], SURVIVAL[survival], ABSORPTION[absorption], STREAMING[streaming],
                       PLANES[plane])
        ctx = C.c_void_p()
        check(lib().rtlb_create(C.byref(Grid(nx, nz)), C.byref(d), C.byref(opts), C.byref(ctx)))
        self._ctx = ctx

    # -- lifecycle
    def close(self):
        if getattr(self, "_ctx", None):
            lib().rtlb_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        check(st, self._ctx)

    # -- configuration
    def set_medium(self, tau, albedo, phase_tables, emission=None, phase_index=None, stream=None):
        """tau, albedo, emission: [nz][nx] float32 (torch cuda/cpu or numpy);
        phase_tables: float64 numpy [n_phase][4n][4n]; phase_index [nz][nx] uint8."""
        tabs = np.ascontiguousarray(phase_tables, np.float64)
        if tabs.ndim == 2:
            tabs = tabs[None]
        args = [tau, albedo, emission, phase_index]
        conv = []
        for a, dt in zip(args, [np.float32, np.float32, np.float32, np.uint8]):
            if a is None or hasattr(a, "data_ptr"):
                conv.append(a if a is None or a.is_contiguous() else a.contiguous())
            else:
                conv.append(np.ascontiguousarray(a, dt))
        self._check(lib().rtlb_set_medium(self._ctx, _ptr(conv[0]), _ptr(conv[1]), _ptr(conv[2]),
                                          tabs.shape[0], tabs.ctypes.data, _ptr(conv[3]),
                                          _stream(stream)))
        self._n_phase = tabs.shape[0]

    def set_boundary(self, side, kind, inflow=None):
        side = SIDES[side] if isinstance(side, str) else int(side)
        kind = BCS[kind] if isinstance(kind, str) else int(kind)
        buf = None if inflow is None else np.ascontiguousarray(inflow, np.float32).reshape(self.n, 4)
        self._check(lib().rtlb_set_boundary(self._ctx, side, kind, _ptr(buf)))

    # -- state
    def set_state(self, S, stream=None):
        """S: [nz][nx][n][4] float32, a torch tensor (device or pinned host) or numpy."""
        if not hasattr(S, "data_ptr"):
            S = np.ascontiguousarray(S, np.float32)
        self._check(lib().rtlb_set_state(self._ctx, _ptr(S), _stream(stream)))

    def get_state(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.nz, self.nx, self.n, 4), dtype=torch.float32, device="cuda")
        self._check(lib().rtlb_get_state(self._ctx, _ptr(out), _stream(stream)))
        return out

    # -- stepping
    def step(self, nsteps: int = 1, stream=None):
        self._check(lib().rtlb_step(self._ctx, int(nsteps), _stream(stream)))

    def run_to_steady(self, tol: float, max_steps: int, check_every: int = 10, stream=None):
        steps = C.c_int32()
        res = C.c_double()
        st = lib().rtlb_run_to_steady(self._ctx, float(tol), int(max_steps), int(check_every),
                                      C.byref(steps), C.byref(res), _stream(stream))
        if st not in (0, 9):
            self._check(st)
        return steps.value, res.value, st == 0

    def last_residual(self, stream=None) -> float:
        r = C.c_double()
        self._check(lib().rtlb_last_residual(self._ctx, C.byref(r), _stream(stream)))
        return r.value

    def dop_out(self, side="top", out=None, stream=None):
        """Degree of polarization [len][n] of the radiance leaving through a
        side (rtlb_dop_out)."""
        import torch
        side = SIDES[side] if isinstance(side, str) else int(side)
        ln = self.nx if side in (0, 1) else self.nz
        if out is None:
            out = torch.empty((ln, self.n), dtype=torch.float32, device="cuda")
        self._check(lib().rtlb_dop_out(self._ctx, side, _ptr(out), _stream(stream)))
        return out

    def stall_next_step(self):
        """Arm the bounded-wait test hook (rtlb_test_stall_next_step)."""
        self._check(lib().rtlb_test_stall_next_step(self._ctx))

    def total_intensity(self, stream=None) -> float:
        r = C.c_double()
        self._check(lib().rtlb_total_intensity(self._ctx, C.byref(r), _stream(stream)))
        return r.value

    def radiance_out(self, side="top", out=None, stream=None):
        import torch
        side = SIDES[side] if isinstance(side, str) else int(side)
        ln = self.nx if side in (0, 1) else self.nz
        if out is None:
            out = torch.empty((ln, self.n, 4), dtype=torch.float32, device="cuda")
        self._check(lib().rtlb_radiance_out(self._ctx, side, _ptr(out), _stream(stream)))
        return out

    def adjoint(self, nsteps: int, dL_dout, checkpoint_every: int = 50, want_S0: bool = False,
                want_Z: bool = True, stream=None):
        """Run nsteps float32 steps from the current state and return the
        gradients of a loss whose gradient w.r.t. the final top radiance is
        dL_dout [nx][n][4]: (grad_tau, grad_albedo) as cuda tensors [nz][nx],
        grad_Z (numpy [n_phase][4n][4n] or None) and grad_S0 (cuda tensor or
        None)."""
        import torch
        dl = dL_dout if hasattr(dL_dout, "data_ptr") else torch.as_tensor(np.asarray(dL_dout, np.float32))
        dl = dl.to(device="cuda", dtype=torch.float32).contiguous()
        gt = torch.empty((self.nz, self.nx), dtype=torch.float32, device="cuda")
        ga = torch.empty_like(gt)
        n_phase = self._n_phase
        gZ = np.zeros((n_phase, 4 * self.n, 4 * self.n)) if want_Z else None
        gS = torch.empty((self.nz, self.nx, self.n, 4), dtype=torch.float32, device="cuda") if want_S0 else None
        self._check(lib().rtlb_adjoint(self._ctx, int(nsteps), int(checkpoint_every), _ptr(dl), _ptr(gt), _ptr(ga),
                                       _ptr(gZ), _ptr(gS), _stream(stream)))
        return gt, ga, gZ, gS

    def release_workspace(self):
        """Free the device workspace adjoint() keeps between calls (its
        checkpoints and adjoint states); the next adjoint() allocates again."""
        self._check(lib().rtlb_release_workspace(self._ctx))

    @property
    def steps_done(self) -> int:
        return int(lib().rtlb_steps_done(self._ctx))

    def form(self) -> dict:
        """How the steps run (rtlb_get_form): tensor_core, cta_pair,
        gather_form, mixed_tiles, stages."""
        f = _lib.Form()
        self._check(lib().rtlb_get_form(self._ctx, C.byref(f)))
        return {k: int(getattr(f, k)) for k, _ in f._fields_}

    @property
    def gather_form(self) -> bool:
        return bool(self.form()["gather_form"])

    @property
    def mixed_tiles(self) -> int:
        return self.form()["mixed_tiles"]


def solver_for(w, precision: str = "fp32") -> Solver:
    """Solver set up for a workloads.Workload (medium, tables, boundaries)."""
    surv = "exp" if w.surv_mode == 1 else "linear"
    absm = "taylor" if w.abs_mode == 1 else "beer_lambert"
    s = Solver(w.nx, w.nz, w.n_zen, w.n_az, precision=precision, survival=surv, absorption=absm,
               streaming=getattr(w, "scheme", "nearest"), plane=getattr(w, "plane", "xz"))
    tabs = np.stack([phase_table_spec(w.n_zen, w.n_az, sp) for sp in w.phase_specs])
    s.set_medium(w.tau.astype(np.float32), w.albedo.astype(np.float32), tabs,
                 emission=None if w.emission is None else w.emission.astype(np.float32),
                 phase_index=w.phase_index)
    for side in range(4):
        inflow = None if w.inflow is None else w.inflow[side]
        s.set_boundary(side, w.bc[side], inflow if w.bc[side] == 2 else None)
    return s


def _tables_for(solver: Solver, specs, g_value=None, hg_index=None):
    tabs = []
    for k, sp in enumerate(specs):
        if k == hg_index:
            tabs.append(phase_hg(solver.n_zen, solver.n_az, float(g_value), sp[2]))
        else:
            tabs.append(phase_table_spec(solver.n_zen, solver.n_az, sp))
    return np.stack(tabs)


def _make_top_radiance_fn():
    import torch

    class TopRadiance(torch.autograd.Function):
        """top radiance [nx][n][4] after `nsteps` steps from a zero state, as a
        differentiable function of per-cell extinction tau [nz][nx], albedo
        [nz][nx] and the asymmetry g of the HG class `hg_index`.  Forward:
        rtlb_set_medium + rtlb_step + rtlb_radiance_out.  Backward:
        rtlb_adjoint (float32 forward replayed from checkpoints every
        `checkpoint_every` steps) and rtlb_phase_hg_grad for dL/dg."""

        @staticmethod
        def forward(ctx, tau, albedo, g, solver, specs, hg_index, phase_index, nsteps, checkpoint_every):
            tabs = _tables_for(solver, specs, g.item(), hg_index)
            solver.set_medium(tau.detach().float().contiguous(), albedo.detach().float().contiguous(), tabs,
                              phase_index=phase_index)
            zero = torch.zeros((solver.nz, solver.nx, solver.n, 4), dtype=torch.float32, device="cuda")
            solver.set_state(zero)
            solver.step(nsteps)
            out = solver.radiance_out("top").clone()
            ctx.solver, ctx.nsteps, ctx.K, ctx.hg_index = solver, nsteps, checkpoint_every, hg_index
            ctx.g, ctx.pol_amp = float(g.item()), (specs[hg_index][2] if hg_index is not None else 0.0)
            ctx.zero = zero
            return out

        @staticmethod
        def backward(ctx, grad_out):
            s = ctx.solver
            s.set_state(ctx.zero)
            gt, ga, gZ, _ = s.adjoint(ctx.nsteps, grad_out.contiguous(), checkpoint_every=ctx.K)
            gg = None
            if ctx.hg_index is not None:
                dg = phase_hg_grad(s.n_zen, s.n_az, ctx.g, ctx.pol_amp, gZ[ctx.hg_index])
                gg = torch.tensor(dg, dtype=torch.float64, device="cuda")
            return gt, ga, gg, None, None, None, None, None, None

    return TopRadiance


_TOP_RADIANCE = None


def top_radiance(tau, albedo, g, solver: Solver, specs, hg_index=None, phase_index=None, nsteps=100,
                 checkpoint_every=50):
    """Differentiable top radiance (see TopRadiance); g is a scalar tensor."""
    global _TOP_RADIANCE
    if _TOP_RADIANCE is None:
        _TOP_RADIANCE = _make_top_radiance_fn()
    return _TOP_RADIANCE.apply(tau, albedo, g, solver, specs, hg_index, phase_index, nsteps, checkpoint_every)


class Batch:
    """Several Solvers (same tensor-core precision, n <= 32) advanced by one
    persistent launch per step (rtlb_batch_*)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s._ctx for s in self.solvers])
        b = C.c_void_p()
        check(lib().rtlb_batch_create(len(self.solvers), arr, C.byref(b)))
        self._b = b
        self.stages = 4
        self.tile_cost = 4

    def _check(self, st):
        if st != _lib.RTLB_OK:
            raw = lib().rtlb_batch_last_error(self._b)
            raise _lib.RtlbError(st, raw.decode() if raw else "")

    def configure(self, stages: int):
        self._check(lib().rtlb_batch_configure(self._b, int(stages)))
        self.stages = int(stages)

    def balance(self, tile_cost: int):
        """Work estimate of a tile in the CTAs' item ranges: n + tile_cost
        directions' worth (rtlb_batch_balance)."""
        self._check(lib().rtlb_batch_balance(self._b, int(tile_cost)))
        self.tile_cost = int(tile_cost)

    def step(self, nsteps: int = 1, stream=None):
        self._check(lib().rtlb_batch_step(self._b, int(nsteps), _stream(stream)))

    def check(self, stream=None):
        self._check(lib().rtlb_batch_check(self._b, _stream(stream)))

    @property
    def site_direction_updates_per_step(self) -> int:
        return sum(s.nx * s.nz * s.n for s in self.solvers)

    def close(self):
        if getattr(self, "_b", None):
            lib().rtlb_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tune_cache_path():
    import os
    return os.environ.get("RTLB_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "rtlb_tune.json")


def autotune_batch(batch: Batch, candidates=(2, 4, 6, 8), costs=(4, 0, 8, 16), trial_steps: int = 4,
                   cache_path=None) -> int:
    """Tune the batch kernel on its own workload: every pipeline depth in
    `candidates` crossed with every work-balance tile cost in `costs`
    (rtlb_batch_configure, rtlb_batch_balance), each timed over `trial_steps`
    real steps (every setting computes the same result, so the channels simply
    advance; on a tie the setting tried first, the default cost 4, stays).
    The fastest pair is applied and remembered in a JSON cache
    keyed by device, precision and workload shape; a cached choice is applied
    without timing.  Returns the chosen depth (the cost is batch.tile_cost)."""
    import json
    import os

    import torch
    path = cache_path or _tune_cache_path()
    sig = {"device": torch.cuda.get_device_name(), "precision": batch.solvers[0].precision,
           "n": sorted({s.n for s in batch.solvers}), "channels": len(batch.solvers),
           "sdu_per_step_log2": int(np.log2(max(1, batch.site_direction_updates_per_step)))}
    key = json.dumps(sig, sort_keys=True)
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    if key in cache:
        batch.configure(cache[key]["stages"])
        batch.balance(cache[key].get("tile_cost", 4))
        return cache[key]["stages"]
    best, best_ms = None, float("inf")
    for cost in costs:
        try:
            batch.balance(cost)
        except _lib.RtlbError:
            continue
        for st in candidates:
            try:
                batch.configure(st)
            except _lib.RtlbError:
                continue
            batch.step(2)                          # capture + warm
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            batch.step(trial_steps)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / trial_steps
            if ms < best_ms:
                best, best_ms = (st, cost), ms
    batch.configure(best[0])
    batch.balance(best[1])
    cache[key] = {"stages": best[0], "tile_cost": best[1], "ms_per_step": best_ms}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return best[0]
