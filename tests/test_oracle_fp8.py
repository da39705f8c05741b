"""Pins of the oracle's FP8 block-scaled form (orc_e4m3, orc_fp8_exponent,
orc_step_fp8) to things other than itself.

- e4m3 rounding: every finite e4m3 value is built from its bit fields (OCP
  8-bit floating point, E4M3: exponent bias 7, 3 mantissa bits, exponent
  field 0 subnormal, the all-ones pattern NaN) and must round to itself; the
  midpoint of two neighbours must go to the one with the even mantissa; values
  beyond 448 saturate.
- block exponent: the defining inequalities (amax / 2^e <= 448 < amax / 2^(e-1)).
- the step: with every quantized quantity exactly representable the FP8 form
  must equal the plain FP64 step; with realistic values its error must stay
  within the e4m3 error bound of each product.
"""
import numpy as np
import pytest

import oracle as orc


def _e4m3_values():
    """All non-negative finite e4m3 values, from the bit fields."""
    vals = []
    for E in range(16):
        for M in range(8):
            if E == 15 and M == 7:
                continue                                  # NaN
            vals.append(M * 2.0 ** -9 if E == 0 else (1 + M / 8) * 2.0 ** (E - 7))
    return np.array(vals)


def _mantissa_bits(v):
    """Mantissa field of a positive finite e4m3 value."""
    if v < 2.0 ** -6:
        return int(round(v / 2.0 ** -9))
    e = int(np.floor(np.log2(v)))
    return int(round((v / 2.0 ** e - 1) * 8))


def test_e4m3_values_are_fixed_points():
    vals = _e4m3_values()
    assert vals.max() == 448.0 and vals[1] == 2.0 ** -9 and len(vals) == 127
    for v in vals:
        assert orc.e4m3(v) == v
        assert orc.e4m3(-v) == -v


def test_e4m3_ties_to_even_and_rounding():
    vals = np.unique(_e4m3_values())
    for a, b in zip(vals[:-1], vals[1:]):
        mid = 0.5 * (a + b)
        even = a if _mantissa_bits(a) % 2 == 0 else b
        assert orc.e4m3(mid) == even, (a, b)
        # just off the midpoint goes to the nearer neighbour
        assert orc.e4m3(mid - (b - a) * 1e-6) == a
        assert orc.e4m3(mid + (b - a) * 1e-6) == b


def test_e4m3_saturation_and_tiny():
    assert orc.e4m3(448.0) == 448.0
    assert orc.e4m3(463.9) == 448.0
    assert orc.e4m3(1e30) == 448.0
    assert orc.e4m3(-1e30) == -448.0
    assert orc.e4m3(2.0 ** -10) == 0.0                   # tie between 0 and 2^-9: even is 0
    assert orc.e4m3(3 * 2.0 ** -10) == 2.0 ** -8         # tie between 2^-9 and 2^-8: even is 2^-8
    assert orc.e4m3(0.0) == 0.0


@pytest.mark.parametrize("amax", [1e-30, 3.1e-7, 0.4375, 0.44, 1.0, 1.75, 1.7500001, 447.0, 448.0, 449.0,
                                  3.0e5, 2.0 ** 100])
def test_block_exponent_inequalities(amax):
    for floor in (False, True):
        e = orc.fp8_exponent(amax, floor)
        if floor and amax < 2.0 ** -126:
            assert e == -127
            continue
        assert amax / 2.0 ** e <= 448.0
        if e > -127:
            assert amax / 2.0 ** (e - 1) > 448.0


def test_block_exponent_clamps():
    assert orc.fp8_exponent(0.0) == -127
    assert orc.fp8_exponent(1e-300) == -127
    assert orc.fp8_exponent(1e-40, True) == -127
    assert orc.fp8_exponent(1e300) == 127


def _single_site(n, Z, S, tau, albedo, surv, emission=0.0):
    """A 1x1 periodic lattice: every direction streams back into the site, so
    one step is the collision alone."""
    mu, phi = np.zeros(n), np.zeros(n)         # unused: the offsets are given
    P = orc.Problem(1, 1, mu, phi, tau, albedo, emission if emission else None, None, Z,
                    surv_mode=surv, bc=(orc.BC_PERIODIC,) * 4, offsets=(np.zeros(n), np.zeros(n)))
    return P


def _exact_table(rng, K, diag_blocks, k_lo):
    """Entries m 2^k with 3-bit mantissas, k in [k_lo, k_lo + 5] (every 32-entry
    block spans less than 2^8, so its e4m3 block quantization is exact; with
    k_lo far outside e4m3's range only a correct block scale keeps it so)."""
    m = 1 + rng.integers(0, 8, size=(K, K)) / 8.0
    Z = m * 2.0 ** rng.integers(k_lo, k_lo + 6, size=(K, K)) * rng.choice([-1.0, 1.0], size=(K, K))
    Z[rng.random((K, K)) < 0.2] = 0.0
    if diag_blocks:
        n = K // 4
        for i in range(n):
            Z[4 * i:4 * i + 4, 4 * i:4 * i + 4] = np.eye(4) * (0.5 + i / 64.0)   # float32-exact c_i
    return Z


@pytest.mark.parametrize("n", [8, 16, 32])
@pytest.mark.parametrize("diag_blocks", [False, True])
@pytest.mark.parametrize("z_lo,s_lo", [(-6, -3), (-16, -20), (10, 6)])
def test_fp8_step_exact_when_representable(n, diag_blocks, z_lo, s_lo):
    """tau = 0.25, albedo = 1, linear survival: A = 1, beta = 0.25, alpha =
    0.75 exactly; the state m 2^k (3-bit m, k in [s_lo, s_lo + 3]) makes beta
    S~ exact in e4m3 after the block scale, so the FP8 form equals the FP64
    step.  The table and state magnitudes include ones below e4m3's smallest
    value and above its largest, which need the block scales."""
    rng = np.random.default_rng([n, int(diag_blocks), z_lo + 100])
    K = 4 * n
    Z = _exact_table(rng, K, diag_blocks, z_lo)
    S = ((1 + rng.integers(0, 4, size=K) / 4.0) * 2.0 ** rng.integers(s_lo, s_lo + 4, size=K)).reshape(1, 1, n, 4)
    P = _single_site(n, Z, S, 0.25, 1.0, orc.SURV_LINEAR)
    ref = P.step(S)
    got = P.step_fp8(S)
    scat = 0.25 * Z @ S.ravel()
    assert np.abs(got.ravel() - ref.ravel()).max() <= 1e-14 * np.abs(scat).max()
    # and the plain step is alpha S + beta Z S
    assert np.allclose(ref.ravel(), 0.75 * S.ravel() + scat, rtol=1e-14, atol=0)


@pytest.mark.parametrize("n", [8, 32, 64])
def test_fp8_step_within_e4m3_bound(n):
    """Realistic table (HG + polarization) and state: each product of two
    e4m3-rounded factors is within (2 u + u^2) of the exact one, u = 2^-4, so
    |P_fp8 - P| <= (2u + u^2) beta sum_k |Z_rk| |S~_k| (+ float32 rounding of
    S~ and beta), and a deliberately dropped block scale would break it."""
    nzen, naz = {8: (2, 4), 32: (4, 8), 64: (8, 8)}[n]
    mu, phi = orc.direction_grid(nzen, naz)
    Z = orc.phase_table(mu, phi, orc.PHASE_HG, 0.85, -0.1)
    rng = np.random.default_rng(n)
    S = rng.random((1, 1, n, 4)).astype(np.float32).astype(np.float64)
    S[..., 1:] *= 0.3
    tau, w = 0.6, 0.95
    P = _single_site(n, Z, S, tau, w, orc.SURV_EXP)
    ref = P.step(S)
    got = P.step_fp8(S)
    A = np.exp(-(1 - w) * tau)
    beta = A * (1 - np.exp(-w * tau))
    u = 2.0 ** -4
    bound = (2 * u + u * u) * beta * (np.abs(Z) @ np.abs(S.ravel())) + 1e-6 * np.abs(ref).max()
    err = np.abs(got.ravel() - ref.ravel())
    assert np.all(err <= bound)
    assert err.max() > 0          # the form does round


# ---- the split form (orc_step_fp8x): state in two e4m3 terms, table in three


def _bits_table(rng, K, mant_bits, k_lo):
    """Entries (1 + j / 2^mant_bits) 2^k with one exponent k per 32-entry block
    (k in [k_lo, k_lo + 5]), random signs, 20 % zeros: a block's terms then
    carry 4 significant bits each, so 4 mantissa bits fit one e4m3 term, 8 two
    and 11 three."""
    m = 1 + rng.integers(0, 2 ** mant_bits, size=(K, K)) / 2.0 ** mant_bits
    k = np.repeat(rng.integers(k_lo, k_lo + 6, size=(K, K // 32)), 32, axis=1)
    Z = m * 2.0 ** k * rng.choice([-1.0, 1.0], size=(K, K))
    Z[rng.random((K, K)) < 0.2] = 0.0
    return Z


@pytest.mark.parametrize("n", [8, 32])
@pytest.mark.parametrize("z_lo,s_lo", [(-6, -3), (-16, -20), (10, 6)])
@pytest.mark.parametrize("state_bits,table_bits", [(7, 7), (3, 11)])
def test_fp8x_step_exact_when_representable(n, z_lo, s_lo, state_bits, table_bits):
    """beta = 0.25, alpha = 0.75 exactly (as above).  A state with 7-bit
    mantissas needs both state terms and a table with 7-bit mantissas two of
    its three terms: every product the form keeps is exact and the one it
    drops (state lo x table term 3) is zero, so the form equals the FP64
    step; likewise a 3-bit state (one term) with an 11-bit table (all three
    terms).  Dropping any kept product, or a wrong scale for a lo term, breaks
    the equality."""
    rng = np.random.default_rng([n, z_lo + 100, state_bits])
    K = 4 * n
    Z = _bits_table(rng, K, table_bits, z_lo)
    mant = 1 + rng.integers(0, 2 ** state_bits, size=K) / 2.0 ** state_bits
    kexp = np.repeat(rng.integers(s_lo, s_lo + 2, size=K // 32), 32)   # one exponent range per block
    S = (mant * 2.0 ** kexp).reshape(1, 1, n, 4)
    P = _single_site(n, Z, S, 0.25, 1.0, orc.SURV_LINEAR)
    ref = P.step(S)
    got = P.step_fp8x(S)
    scat = 0.25 * Z @ S.ravel()
    assert np.abs(got.ravel() - ref.ravel()).max() <= 1e-14 * np.abs(scat).max()
    # the single-term form does not represent these operands
    if state_bits > 3 or table_bits > 3:
        assert np.abs(P.step_fp8(S).ravel() - ref.ravel()).max() > 1e-6 * np.abs(scat).max()


@pytest.mark.parametrize("n", [8, 32, 64])
def test_fp8x_step_within_split_bound(n):
    """Realistic table (HG + polarization) and state.  The two state terms
    leave at most u^2 |x| of each value (u = 2^-4), the three table terms
    u^3 |w|, and the dropped product (state lo x table term 3) is below
    u^3 (1 + u)^2 |x| |w|, so |P_fp8x - P| <= (u^2 + 2.3 u^3) beta
    sum_k |Z_rk| |S~_k| plus an absolute floor for entries far below their
    block's largest (subnormal spacing of the lo terms).  The split form is
    also far closer than the single-term form."""
    nzen, naz = {8: (2, 4), 32: (4, 8), 64: (8, 8)}[n]
    mu, phi = orc.direction_grid(nzen, naz)
    Z = orc.phase_table(mu, phi, orc.PHASE_HG, 0.85, -0.1)
    rng = np.random.default_rng(n + 7)
    S = rng.random((1, 1, n, 4)).astype(np.float32).astype(np.float64)
    S[..., 1:] *= 0.3
    tau, w = 0.6, 0.95
    P = _single_site(n, Z, S, tau, w, orc.SURV_EXP)
    ref = P.step(S)
    got = P.step_fp8x(S)
    A = np.exp(-(1 - w) * tau)
    beta = A * (1 - np.exp(-w * tau))
    u = 2.0 ** -4
    mag = beta * (np.abs(Z) @ np.abs(S.ravel()))
    bound = (u * u + 2.3 * u ** 3) * mag + 2.0 ** -20 * beta * np.abs(S).max() * np.abs(Z).sum(axis=1) \
        + 1e-6 * np.abs(ref).max() * 2.0 ** -10
    err = np.abs(got.ravel() - ref.ravel())
    assert np.all(err <= bound)
    assert err.max() > 0
    err1 = np.abs(P.step_fp8(S).ravel() - ref.ravel())
    assert err.max() < 0.1 * err1.max()


@pytest.mark.parametrize("n", [8, 32])
def test_fp8x_lo_term_has_its_own_scale(n):
    """Each 32-value block of the state holds one large value that e4m3 holds
    exactly (so it leaves no remainder) and small values with 7-bit mantissas
    2^12 below it.  The hi term's scale is set by the large value; the small
    values' remainders lie below e4m3's smallest subnormal at that scale, so
    only a lo term scaled from the remainders' own maximum keeps them, and
    then the form is exact (table exact in one term)."""
    rng = np.random.default_rng(n + 11)
    K = 4 * n
    Z = _bits_table(rng, K, 3, -4)
    S = (1 + rng.integers(0, 128, size=K) / 128.0) * 2.0 ** -12
    S[::32] = 1.5                                  # one e4m3-exact value per block
    S = S.reshape(1, 1, n, 4)
    P = _single_site(n, Z, S, 0.25, 1.0, orc.SURV_LINEAR)
    ref = P.step(S)
    scat = 0.25 * Z @ S.ravel()
    assert np.abs(P.step_fp8x(S).ravel() - ref.ravel()).max() <= 1e-14 * np.abs(scat).max()
