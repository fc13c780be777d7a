"""Independent numpy model of the low-precision storage formats (BF16, FP16, E4M3).

Used by the tests to check the library's stored codes bit for bit and to build
the dequantized matrix the FP64 oracle then solves.  Rounding is written from
the formats' definitions (sign, exponent with bias, mantissa bits, subnormals):
round to nearest, ties to even, with saturation at the largest finite value.
"""
import numpy as np

# (mantissa bits, smallest normal exponent, largest finite value, per-column target max)
FORMATS = {
    "bf16": (7, -126, float(np.finfo(np.float32).max) * (1 - 2.0 ** -8), 1.0),
    "f16": (10, -14, 65504.0, 32768.0),
    "e4m3": (3, -6, 448.0, 448.0),
}


def round_to_format(x, fmt):
    """Nearest representable value of the format (ties to even), saturating."""
    mbits, emin, vmax, _ = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    ax = np.abs(x[nz])
    e = np.floor(np.log2(ax))
    # guard against log2 rounding at exact powers of two
    e = np.where(2.0 ** e > ax, e - 1, e)
    e = np.where(2.0 ** (e + 1) <= ax, e + 1, e)
    e = np.maximum(e, emin)
    step = 2.0 ** (e - mbits)
    q = np.rint(ax / step) * step           # np.rint rounds half to even
    q = np.minimum(q, vmax)
    out[nz] = np.sign(x[nz]) * q
    return out


def quantize(Z, fmt):
    """(dequantized values, per-column scale) as the library defines them."""
    Z = np.asarray(Z, dtype=np.float64)
    amax = np.abs(Z).max(axis=0)
    s = np.where(amax > 0, amax / FORMATS[fmt][3], 1.0)
    q = round_to_format(Z / s[None, :], fmt)
    return q, s


def e4m3_table():
    """Value of each of the 256 E4M3 codes (NaN for 0x7F / 0xFF)."""
    vals = np.zeros(256)
    for c in range(256):
        sgn = -1.0 if c & 0x80 else 1.0
        ex = (c >> 3) & 0xF
        m = c & 7
        if ex == 0xF and m == 7:
            vals[c] = np.nan
        elif ex == 0:
            vals[c] = sgn * (m / 8.0) * 2.0 ** -6
        else:
            vals[c] = sgn * (1 + m / 8.0) * 2.0 ** (ex - 7)
    return vals


def decode(codes, fmt):
    """Values of raw stored codes (BF16 uint16 bits, FP16, E4M3 uint8 bits)."""
    if fmt == "bf16":
        return (codes.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if fmt == "f16":
        return codes.astype(np.float64)
    return e4m3_table()[codes.astype(np.int64)]
