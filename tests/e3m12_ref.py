"""The E3M12 16-bit storage format written out from its definition (test
infrastructure): 1 sign, 3 exponent and 12 mantissa bits, value
2^(e-11) (1 + m/4096) for exponent field e = 1..7 and m * 2^-22 for e = 0.
Rounding to nearest picks the nearest representable magnitude by search
over all of them, ties to the even code, and saturates at the largest."""
import numpy as np


def decode(code):
    """float64 value of each 16-bit code."""
    code = np.asarray(code, dtype=np.int64)
    e = (code >> 12) & 7
    m = code & 0xFFF
    mag = np.where(e == 0, m * 2.0 ** -22, (1.0 + m / 4096.0) * np.exp2(e - 11.0))
    return np.where(code & 0x8000, -mag, mag)


_MAGS = decode(np.arange(0x8000))  # increasing with the code


def encode_rn(x):
    """Code of each float32 value, rounded to the nearest magnitude (ties to
    the even code), saturating at the largest; NaN saturates too."""
    x = np.asarray(x, dtype=np.float32)
    a = np.abs(x.astype(np.float64))
    a = np.where(np.isnan(a), np.inf, a)
    hi = np.clip(np.searchsorted(_MAGS, a, side="left"), 0, 0x7FFF)
    lo = np.clip(hi - 1, 0, 0x7FFF)
    dlo = np.abs(a - _MAGS[lo])
    dhi = np.abs(_MAGS[hi] - a)
    code = np.where(dlo < dhi, lo, hi)
    tie = (dlo == dhi) & (lo != hi)
    code = np.where(tie, np.where(lo % 2 == 0, lo, hi), code)
    code = np.where(a > _MAGS[-1], 0x7FFF, code)
    sign = np.signbit(x)
    return (code | np.where(sign, 0x8000, 0)).astype(np.uint16)
