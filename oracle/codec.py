"""FP64 oracle: reduced-precision spinor codecs of Sec. 6.5 ("Reduced precision
in preconditioner communication", Table sloppy).

TEST INFRASTRUCTURE (see ``oracle/__init__``): never imported by the library.

* ``truncate16``  each FP32 word cut to its top 16 bits (8-bit exponent,
               7-bit mantissa: the BF16 layout, by truncation), the format of
               Table sloppy's last row.
* ``encode_i8`` / ``decode_i8``  a four-spinor of one 5D site (24 reals) as
               a half-precision prefactor and 24 signed 8-bit integers (the
               proposal of Sec. 6.5: scale by the largest magnitude and round
               to bytes).  Reading:
               the prefactor is the largest |real| of the site rounded to
               FP16, the integers are round(127 v / prefactor) clipped to
               [-127, 127], and decoding multiplies back by prefactor / 127.
               26 bytes per site against 48 (FP16) or 96 (FP32).  The FP16
               prefactor limits the range: sites whose largest |real| is at
               most 2^-25 (about 3e-8) encode as zero, those below 2^-14 keep
               fewer prefactor bits, and 65520 or more gives an infinite
               prefactor (NaN once decoded), so data must be normalised first
               (as the library scales the smoother's input to unit RMS).

Parity: pinned by tests/test_oracle_codec.py (the truncation against the bit
pattern, the 8-bit round-trip bound of half a quantum plus the prefactor's
rounding, the prefactor against the nearest binary16 found by enumerating
every half (one rounding from double, ties to even, subnormals, overflow),
exact zeros, the byte count, and an HDCG solve whose M_IRS input passes
through either codec converging like the unrounded one).
"""
from __future__ import annotations

import numpy as np


def truncate16(x):
    """Each real of the FP32 rounding of x cut to its top 16 bits (as float64)."""
    a = np.ascontiguousarray(x)
    re = np.ascontiguousarray(a.view(np.float64) if np.iscomplexobj(a) else a, dtype=np.float64)
    f = re.astype(np.float32)
    bits = f.view(np.uint32) & np.uint32(0xFFFF0000)
    out = bits.view(np.float32).astype(np.float64)
    return out.view(np.complex128).reshape(a.shape) if np.iscomplexobj(a) else out.reshape(a.shape)


def encode_i8(psi):
    """psi (..., Ls, 4, 3) complex -> (scale (..., Ls) float16, q (..., Ls, 24) int8)."""
    v = np.ascontiguousarray(psi).view(np.float64).reshape(psi.shape[:-2] + (24,))
    s = np.abs(v).max(axis=-1)
    scale = s.astype(np.float16)
    sf = scale.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(sf[..., None] > 0, np.rint(127.0 * v / sf[..., None]), 0.0)
    return scale, np.clip(q, -127, 127).astype(np.int8)


def decode_i8(scale, q):
    """Inverse of encode_i8: (..., Ls, 4, 3) complex."""
    v = q.astype(np.float64) * (scale.astype(np.float64)[..., None] / 127.0)
    return np.ascontiguousarray(v).view(np.complex128).reshape(q.shape[:-1] + (4, 3))


def bytes_i8_per_site() -> int:
    return 2 + 24
