"""Pins of the reduced-precision spinor codecs (Sec. 6.5, Table sloppy).  No
GPU.  What fixes them: the IEEE bit patterns of the truncation; the 8-bit
round-trip bound; exact zeros; and an HDCG solve with the codec applied to
the M_IRS input converging in about as many outer iterations as without
(Table sloppy: no change for 16 bits)."""
import numpy as np
import pytest

import synthetic as sy
from oracle.codec import bytes_i8_per_site, decode_i8, encode_i8, truncate16
from oracle.solvers import DeflationSpace, adef2, mirs


def test_truncate16_bit_pattern():
    x = np.array([1.0, -1.0, 3.14159265, 1e-3, 65504.0, 0.0, 1.0 + 2 ** -8])
    t = truncate16(x)
    for a, b in zip(x, t):
        fa = np.float32(a).view(np.uint32)
        assert np.float32(b).view(np.uint32) == (fa & 0xFFFF0000)
    # 7 mantissa bits: relative error below 2^-7, never rounded up in magnitude
    y = sy.complex_normal(1960, (100,))
    ty = truncate16(y)
    for a, b in [(y.real, ty.real), (y.imag, ty.imag)]:
        assert np.all(np.abs(a - b) <= 2.0 ** -7 * np.abs(a) * 1.0000001)
        assert np.all(np.abs(b) <= np.abs(a) * (1 + 1e-7))


def test_i8_round_trip_bound():
    psi = sy.complex_normal(1961, (50, 4, 4, 3)) * np.geomspace(1e-3, 1e3, 4)[None, :, None, None]
    scale, q = encode_i8(psi)
    assert scale.dtype == np.float16 and q.dtype == np.int8 and q.shape == (50, 4, 24)
    out = decode_i8(scale, q)
    v = psi.view(np.float64).reshape(50, 4, 24)
    w = out.view(np.float64).reshape(50, 4, 24)
    s = np.abs(v).max(axis=-1)
    sh = scale.astype(np.float64)
    # half a quantum of the prefactor, plus the prefactor's own FP16 rounding
    bound = sh / 254.0 + np.abs(s - sh) + 1e-15 * s
    assert np.all(np.abs(v - w) <= bound[..., None])
    assert np.all(np.abs(q) <= 127)
    assert bytes_i8_per_site() == 26


def test_i8_zero_and_exact_values():
    z = np.zeros((3, 2, 4, 3), dtype=np.complex128)
    sc, q = encode_i8(z)
    assert np.all(decode_i8(sc, q) == 0)
    k = np.zeros((1, 1, 4, 3), dtype=np.complex128)
    k[0, 0, 0, 0] = 2.0
    k[0, 0, 1, 1] = -1.0j
    sc, q = encode_i8(k)
    out = decode_i8(sc, q)
    assert out[0, 0, 0, 0] == 2.0 and abs(out[0, 0, 1, 1] + 1.0j) < 2.0 / 254


@pytest.fixture(scope="module")
def two_level(two_level_8x8x4x4):
    d, bl, phi, A, b, xs, it8 = two_level_8x8x4x4
    ref = adef2(d.mdagm, b, DeflationSpace(phi, bl, A, coarse_tol=0.04), 1e-8)
    return d, bl, phi, A, b, ref


@pytest.mark.parametrize("codec", ["truncate16", "i8"])
def test_hdcg_with_compressed_smoother_input(two_level, codec):
    """M_IRS applied to the codec's image of its input (as if that input had
    crossed a compressed halo): the outer A-DEF2 still meets the tolerance,
    within a few iterations of the unrounded solve.  (Without the unit-RMS
    scaling the 8-bit format's FP16 prefactors underflow once the residual
    has fallen by about 1e-5 per site, and the solve breaks down.)"""
    d, bl, phi, A, b, ref = two_level

    def squeeze(r):
        if codec == "truncate16":
            return truncate16(r)
        # the FP16 prefactor needs values inside its range: the residual is
        # scaled to unit RMS per real first and back afterwards, as the
        # library does before any 16-bit storage of the smoother's input
        rms = np.sqrt(np.vdot(r, r).real / (2 * r.size))
        return rms * decode_i8(*encode_i8(r / rms))

    res = adef2(d.mdagm, b, DeflationSpace(phi, bl, A, coarse_tol=0.04), 1e-8,
                M=lambda r: mirs(d.mdagm, squeeze(r), 7, 1.0))
    assert res.true_residual < 2e-8
    assert res.iterations <= ref.iterations + 3


def _half_by_enumeration(x):
    """The binary16 value nearest to x >= 0 (ties to the even bit pattern), by
    search over every finite non-negative half; +inf at or beyond 65520."""
    bits = np.arange(0, 0x7C00, dtype=np.uint16)
    vals = bits.view(np.float16).astype(np.float64)
    if x >= 65520.0:
        return np.uint16(0x7C00)
    d = np.abs(vals - x)
    cand = np.flatnonzero(d == d.min())
    even = [c for c in cand if bits[c] % 2 == 0]
    return bits[even[0] if len(cand) > 1 else cand[0]]


def test_i8_prefactor_is_the_correctly_rounded_half():
    """The prefactor rounds max |v| from double to binary16 directly (one
    rounding): a value just above a midpoint that a float32 step would move
    onto the midpoint, subnormal ties, and the overflow edge."""
    xs = [1 + 2.0 ** -11 + 2.0 ** -40, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 2.0 ** -25, 3 * 2.0 ** -25,
          2.0 ** -25 * (1 + 2.0 ** -30), 6.1e-5, 65519.0, 65504.0, 65519.99, 0.3, 1e-7]
    for x in xs:
        psi = np.zeros((1, 4, 3), dtype=np.complex128)
        psi[0, 0, 0] = x
        scale, _ = encode_i8(psi)
        assert scale.view(np.uint16)[0] == _half_by_enumeration(x), x
