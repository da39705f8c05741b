"""ctypes binding of librtlb.so (the in-tree CUDA library).

Argument marshalling only.  The library must have been built
(``python -m paper_2609_23057_b300.build``); there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# RTLB_LIBRARY may point at another build of the same library (e.g. a variant
# compiled with different tuning macros); the default is the in-tree build.
LIB_PATH = os.environ.get("RTLB_LIBRARY") or os.path.join(_HERE, "librtlb.so")

RTLB_OK = 0
STATUS_NAMES = {
    0: "RTLB_OK", 1: "RTLB_E_ARG", 2: "RTLB_E_SHAPE", 3: "RTLB_E_RANGE",
    4: "RTLB_E_AMBIGUOUS_STREAM", 5: "RTLB_E_STATE", 6: "RTLB_E_OOM", 7: "RTLB_E_CUDA",
    8: "RTLB_E_NONFINITE", 9: "RTLB_E_NOT_CONVERGED", 10: "RTLB_E_TIMEOUT",
    11: "RTLB_E_UNSUPPORTED",
}

# Every symbol include/rtlb.h declares (checked by the CPU test suite).
EXPORTS = [
    "rtlb_create", "rtlb_set_medium", "rtlb_set_boundary", "rtlb_set_state", "rtlb_get_state",
    "rtlb_step", "rtlb_run_to_steady", "rtlb_last_residual", "rtlb_radiance_out",
    "rtlb_total_intensity", "rtlb_steps_done", "rtlb_last_error", "rtlb_destroy",
    "rtlb_stream_offsets", "rtlb_phase_rayleigh", "rtlb_phase_hg", "rtlb_phase_mix",
    "rtlb_residual_noalloc", "rtlb_adjoint", "rtlb_phase_conserve_intensity",
    "rtlb_batch_create", "rtlb_batch_configure", "rtlb_batch_balance", "rtlb_batch_step", "rtlb_batch_check",
    "rtlb_batch_last_error", "rtlb_batch_destroy", "rtlb_stream_taps", "rtlb_release_workspace",
    "rtlb_dop_out", "rtlb_phase_hg_grad", "rtlb_test_stall_next_step", "rtlb_get_form",
]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nz", C.c_int32)]


class Directions(C.Structure):
    _fields_ = [("n_zen", C.c_int32), ("n_az", C.c_int32),
                ("mu", C.POINTER(C.c_double)), ("phi", C.POINTER(C.c_double))]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("survival", C.c_int32), ("absorption", C.c_int32),
                ("streaming", C.c_int32), ("plane", C.c_int32)]


class Form(C.Structure):
    _fields_ = [("tensor_core", C.c_int32), ("cta_pair", C.c_int32), ("gather_form", C.c_int32),
                ("mixed_tiles", C.c_int32), ("stages", C.c_int32)]


class RtlbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


_lib = None


def lib() -> C.CDLL:
    """Load librtlb.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_23057_b300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i32, dp = C.c_void_p, C.c_int32, C.POINTER(C.c_double)
    L.rtlb_create.argtypes = [C.POINTER(Grid), C.POINTER(Directions), C.POINTER(Options), C.POINTER(vp)]
    L.rtlb_set_medium.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp]
    L.rtlb_set_boundary.argtypes = [vp, i32, i32, vp]
    L.rtlb_set_state.argtypes = [vp, vp, vp]
    L.rtlb_get_state.argtypes = [vp, vp, vp]
    L.rtlb_step.argtypes = [vp, i32, vp]
    L.rtlb_run_to_steady.argtypes = [vp, C.c_double, i32, i32, C.POINTER(i32), dp, vp]
    L.rtlb_last_residual.argtypes = [vp, dp, vp]
    L.rtlb_radiance_out.argtypes = [vp, i32, vp, vp]
    L.rtlb_total_intensity.argtypes = [vp, dp, vp]
    L.rtlb_steps_done.argtypes = [vp]
    L.rtlb_steps_done.restype = C.c_int64
    L.rtlb_last_error.argtypes = [vp]
    L.rtlb_last_error.restype = C.c_char_p
    L.rtlb_destroy.argtypes = [vp]
    L.rtlb_destroy.restype = None
    L.rtlb_stream_offsets.argtypes = [C.POINTER(Directions), vp, vp]
    L.rtlb_stream_taps.argtypes = [C.POINTER(Directions), i32, i32, vp, vp, vp]
    L.rtlb_phase_rayleigh.argtypes = [C.POINTER(Directions), C.c_double, vp]
    L.rtlb_phase_conserve_intensity.argtypes = [i32, vp]
    L.rtlb_phase_hg.argtypes = [C.POINTER(Directions), C.c_double, C.c_double, vp, vp]
    L.rtlb_phase_mix.argtypes = [C.POINTER(Directions), C.c_double, C.c_double, C.c_double, vp]
    L.rtlb_residual_noalloc.argtypes = [vp, vp, C.c_size_t, vp, vp]
    L.rtlb_adjoint.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp]
    L.rtlb_release_workspace.argtypes = [vp]
    L.rtlb_batch_create.argtypes = [i32, C.POINTER(vp), C.POINTER(vp)]
    L.rtlb_batch_configure.argtypes = [vp, i32]
    L.rtlb_batch_balance.argtypes = [vp, i32]
    L.rtlb_batch_step.argtypes = [vp, i32, vp]
    L.rtlb_batch_check.argtypes = [vp, vp]
    L.rtlb_batch_last_error.argtypes = [vp]
    L.rtlb_batch_last_error.restype = C.c_char_p
    L.rtlb_batch_destroy.argtypes = [vp]
    L.rtlb_batch_destroy.restype = None
    L.rtlb_dop_out.argtypes = [vp, i32, vp, vp]
    L.rtlb_phase_hg_grad.argtypes = [C.POINTER(Directions), C.c_double, C.c_double, vp, dp]
    L.rtlb_test_stall_next_step.argtypes = [vp]
    L.rtlb_get_form.argtypes = [vp, C.POINTER(Form)]
    for name in EXPORTS:
        f = getattr(L, name)
        if f.restype is C.c_int:     # ctypes default: status codes are int32
            f.restype = C.c_int32
    _lib = L
    return L


def check(status: int, ctx=None) -> None:
    if status != RTLB_OK:
        msg = ""
        if ctx:
            raw = lib().rtlb_last_error(ctx)
            msg = raw.decode() if raw else ""
        raise RtlbError(status, msg)
