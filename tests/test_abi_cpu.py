"""CPU-only checks of the C-ABI library: it loads, exports every symbol that
include/rtlb.h declares, and its host-side (float64) helpers -- streaming
offsets and phase tables, written independently of the oracle -- agree with
the oracle.  No GPU call is made here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2609_23057_b300 import _lib
from paper_2609_23057_b300 import solver as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rtlb_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    declared = _declared_symbols()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    assert set(_lib.EXPORTS) <= declared


def _header_struct_fields(name):
    """int32 fields of `typedef struct { ... } name;` in include/rtlb.h, in order."""
    text = open(os.path.join(ROOT, "include", "rtlb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", text, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, names = decl.split(None, 1)
        assert typ == "int32_t", decl
        fields += [n.strip() for n in names.split(",")]
    return fields


def test_binding_structs_match_the_header():
    """The ctypes mirrors of the ABI's all-int32 structs list the header's
    fields in the header's order."""
    for struct, cls in (("rtlb_options", _lib.Options), ("rtlb_form", _lib.Form), ("rtlb_grid", _lib.Grid)):
        assert [f for f, _ in cls._fields_] == _header_struct_fields(struct), struct
        assert all(t is C.c_int32 for _, t in cls._fields_), struct


@pytest.mark.parametrize("nzen,naz", [(2, 4), (4, 8), (8, 8), (3, 6), (1, 4), (5, 7)])
def test_offsets_match_oracle(orc, nzen, naz):
    mu, phi = orc.direction_grid(nzen, naz)
    cx, cz = S.stream_offsets(nzen, naz)
    ox, oz = orc.stream_offsets(mu, phi)
    assert np.array_equal(cx, ox) and np.array_equal(cz, oz)


def test_tie_is_rejected():
    mu = np.array([np.sin(np.radians(22.5))])
    with pytest.raises(_lib.RtlbError) as ei:
        S.stream_offsets(1, 1, mu, np.array([0.0]))
    assert ei.value.status == 4


@pytest.mark.parametrize("nzen,naz", [(2, 4), (4, 8), (8, 8), (3, 6)])
@pytest.mark.parametrize("spec", [("rayleigh",), ("rayleigh", 0.0279), ("hg", 0.85, -0.1), ("mix", 0.4, 0.6, -0.1)])
def test_tables_match_oracle(orc, nzen, naz, spec):
    mu, phi = orc.direction_grid(nzen, naz)
    Zl = S.phase_table_spec(nzen, naz, spec)
    Zo = orc.phase_table_spec(mu, phi, spec)
    assert np.abs(Zl - Zo).max() <= 1e-14 * max(1.0, np.abs(Zo).max())


def test_explicit_direction_lists(orc):
    """Tables 1-2 use explicit azimuth / zenith sets (e.g. {0,120,240} deg)."""
    mu = np.array([-0.5, -0.5, -0.5, 0.5, 0.5, 0.5])
    phi = np.radians([0.0, 120.0, 240.0, 0.0, 120.0, 240.0])
    Zl = S.phase_rayleigh(2, 3, mu, phi)
    Zo = orc.phase_table(mu, phi)
    assert np.abs(Zl - Zo).max() < 1e-15
    cx, cz = S.stream_offsets(2, 3, mu, phi)
    ox, oz = orc.stream_offsets(mu, phi)
    assert np.array_equal(cx, ox) and np.array_equal(cz, oz)


def test_hg_derivative_matches_central_difference():
    """dZ/dg of the normalized HG table (used by the adjoint) against a
    central difference of the table itself."""
    Z, dZ = S.phase_hg(4, 8, 0.7, -0.1, with_dg=True)
    h = 1e-5
    fd = (S.phase_hg(4, 8, 0.7 + h, -0.1) - S.phase_hg(4, 8, 0.7 - h, -0.1)) / (2 * h)
    assert np.abs(dZ - fd).max() < 1e-6 * max(1.0, np.abs(fd).max())


@pytest.mark.parametrize("nzen,naz,g", [(2, 4, 0.85), (4, 8, 0.85), (8, 8, 0.3)])
def test_hg_gradient_contraction_matches_oracle_table(orc, nzen, naz, g):
    """rtlb_phase_hg_grad (dL/dg = <dZ/dg, dL/dZ>) against the same
    contraction with a central difference of the oracle's own HG table, for a
    random dL/dZ."""
    rng = np.random.default_rng(nzen * naz)
    n = nzen * naz
    gZ = rng.standard_normal((4 * n, 4 * n))
    got = S.phase_hg_grad(nzen, naz, g, -0.1, gZ)
    mu, phi = orc.direction_grid(nzen, naz)
    h = 1e-6
    dZ = (orc.phase_table_spec(mu, phi, ("hg", g + h, -0.1)) - orc.phase_table_spec(mu, phi, ("hg", g - h, -0.1))) / (2 * h)
    ref = float(np.sum(dZ * gZ))
    assert got == pytest.approx(ref, rel=1e-6, abs=1e-8 * np.abs(dZ).sum())
    L = _lib.lib()
    d = _lib.Directions(nzen, naz, None, None)
    out = C.c_double()
    assert L.rtlb_phase_hg_grad(C.byref(d), 1.2, -0.1, gZ.ctypes.data, C.byref(out)) == 3   # RTLB_E_RANGE
    assert L.rtlb_phase_hg_grad(C.byref(d), g, -0.1, None, C.byref(out)) == 1               # RTLB_E_ARG


def test_host_helper_argument_errors():
    L = _lib.lib()
    d = _lib.Directions(0, 4, None, None)
    Z = np.zeros(16)
    assert L.rtlb_phase_rayleigh(C.byref(d), 0.0, Z.ctypes.data) == 2      # RTLB_E_SHAPE
    d = _lib.Directions(2, 4, None, None)
    assert L.rtlb_phase_hg(C.byref(d), 1.5, -0.1, Z.ctypes.data, None) == 3  # RTLB_E_RANGE
    assert L.rtlb_phase_rayleigh(C.byref(d), 0.0, None) == 1                # RTLB_E_ARG
    assert L.rtlb_phase_rayleigh(C.byref(d), 0.7, Z.ctypes.data) == 3       # RTLB_E_RANGE
    big = _lib.Directions(32, 16, None, None)
    assert L.rtlb_stream_offsets(C.byref(big), Z.ctypes.data, Z.ctypes.data) == 2


def test_conserve_intensity_matches_oracle(orc):
    mu, phi = orc.direction_grid(4, 8)
    for spec in [("rayleigh",), ("hg", 0.85, -0.1)]:
        Zl = S.conserve_intensity(S.phase_table_spec(4, 8, spec))
        Zo = orc.conserve_intensity(orc.phase_table_spec(mu, phi, spec))
        assert np.abs(Zl - Zo).max() <= 1e-14 * max(1.0, np.abs(Zo).max())


@pytest.mark.parametrize("plane", ["xz", "xy"])
@pytest.mark.parametrize("nzen,naz", [(2, 4), (4, 8), (8, 8), (3, 6), (1, 4), (5, 7)])
def test_bilinear_taps_match_oracle(orc, nzen, naz, plane):
    mu, phi = orc.direction_grid(nzen, naz)
    pl = {"xz": orc.PLANE_XZ, "xy": orc.PLANE_XY}[plane]
    ox, oz, w = S.stream_taps(nzen, naz, "bilinear", plane)
    rx, rz, rw, _, _ = orc.bilinear_taps(mu, phi, pl)
    assert np.array_equal(ox, rx) and np.array_equal(oz, rz)
    assert np.abs(w - rw).max() < 1e-15


def test_nearest_taps_and_xy_offsets_match_oracle(orc):
    for nzen, naz in [(2, 4), (4, 8), (3, 6)]:
        mu, phi = orc.direction_grid(nzen, naz)
        for plane, pl in (("xz", orc.PLANE_XZ), ("xy", orc.PLANE_XY)):
            ox, oz, w = S.stream_taps(nzen, naz, "nearest", plane)
            cx, cz = orc.stream_offsets(mu, phi, pl)
            assert np.array_equal(ox[:, 0], cx) and np.array_equal(oz[:, 0], cz)
            assert (w[:, 0] == 1).all() and not w[:, 1:].any()


def test_offset_azimuths_need_bilinear_streaming(orc):
    """Table 1's azimuths offset by 22.5 deg on the horizontal lattice lie
    between two D2Q9 offsets: the nearest scheme rejects them, the bilinear
    one streams them."""
    mu = np.array([-0.5] * 4 + [0.5] * 4)
    phi = np.radians([22.5, 112.5, 202.5, 292.5] * 2)
    with pytest.raises(_lib.RtlbError) as ei:
        S.stream_taps(2, 4, "nearest", "xy", mu, phi)
    assert ei.value.status == 4
    ox, oz, w = S.stream_taps(2, 4, "bilinear", "xy", mu, phi)
    rx, rz, rw, _, _ = orc.bilinear_taps(mu, phi, orc.PLANE_XY)
    assert np.array_equal(ox, rx) and np.array_equal(oz, rz) and np.abs(w - rw).max() < 1e-15


def test_stream_taps_argument_errors():
    L = _lib.lib()
    d = _lib.Directions(2, 4, None, None)
    o = np.zeros(32, np.int32)
    w = np.zeros(32)
    assert L.rtlb_stream_taps(C.byref(d), 2, 0, o.ctypes.data, o.ctypes.data, w.ctypes.data) == 1
    assert L.rtlb_stream_taps(C.byref(d), 1, 5, o.ctypes.data, o.ctypes.data, w.ctypes.data) == 1
    assert L.rtlb_stream_taps(C.byref(d), 1, 0, None, o.ctypes.data, w.ctypes.data) == 1
