"""B300-native polarized lattice-Boltzmann radiative-transfer step.

The solver itself is the CUDA library ``librtlb.so`` (C ABI in
``include/rtlb.h``); :mod:`.solver` wraps it for Python callers and
:mod:`.workloads` draws seeded synthetic inputs.  Importing this package does
not load the library; the first solver call does, and fails loudly when the
library has not been built.
"""
__all__ = ["solver", "workloads"]


def __getattr__(name):
    if name in ("Solver", "solver_for", "phase_rayleigh", "phase_hg", "phase_mix",
                "phase_table_spec", "stream_offsets"):
        from . import solver as _s
        return getattr(_s, name)
    raise AttributeError(name)
