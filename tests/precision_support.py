"""Reference encoders/decoders of the storage formats, written from their definitions
(test code; independent of CUDA's conversion intrinsics).

  bfloat16: the upper 16 bits of an IEEE binary32; rounding to nearest even of the
            dropped 16 bits.
  float16:  IEEE binary16 (numpy's float32 -> float16 conversion rounds to nearest even).
  E4M3:     1 sign, 4 exponent (bias 7), 3 mantissa bits; exponent 0 is subnormal
            (m / 8 * 2^-6); S.1111.111 is NaN, so the largest finite magnitude is
            1.75 * 2^8 = 448; no infinities.  Saturating conversion clamps to +-448.
"""
import numpy as np

BF16, F16, FP8 = 1, 2, 3


def e4m3_values() -> np.ndarray:
    """Magnitude of each code 0x00..0x7E (0x7F is NaN)."""
    vals = np.zeros(127)
    for code in range(127):
        e, m = code >> 3, code & 7
        vals[code] = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return vals


_E4M3 = e4m3_values()


def decode_e4m3(b: np.ndarray) -> np.ndarray:
    b = np.asarray(b, np.uint8)
    mag = b & 0x7F
    out = np.where(mag == 0x7F, np.nan, _E4M3[np.minimum(mag, 126)])
    return np.where(b & 0x80, -out, out).astype(np.float32)


def encode_e4m3_satfinite(y: np.ndarray) -> np.ndarray:
    """Round to the nearest E4M3 value, ties to the even code, saturating at 448."""
    y = np.asarray(y, np.float64)
    a = np.minimum(np.abs(y), 448.0)
    hi = np.searchsorted(_E4M3, a, side="left")           # first value >= a
    hi = np.minimum(hi, 126)
    lo = np.maximum(hi - 1, 0)
    dlo, dhi = a - _E4M3[lo], _E4M3[hi] - a
    pick = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(lo % 2 == 0, lo, hi)))
    pick = np.where(_E4M3[hi] == a, hi, pick)
    return (pick | np.where(np.signbit(y), 0x80, 0)).astype(np.uint8)


def encode_bf16_rne(y: np.ndarray) -> np.ndarray:
    u = np.asarray(y, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def decode_bf16(u16: np.ndarray) -> np.ndarray:
    return (np.asarray(u16, np.uint16).astype(np.uint32) << 16).view(np.float32)


def to_numpy_bits(t):
    """Raw storage of a quantised torch tensor as numpy (uint16 bits or uint8 codes)."""
    import torch
    if t.dtype == torch.bfloat16 or t.dtype == torch.float16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy().astype(np.uint8)


def dequantize(t, scale, dtype) -> np.ndarray:
    """Values the solver uses: stored value x per-channel scale, in FP32."""
    bits = to_numpy_bits(t)
    if dtype == BF16:
        v = decode_bf16(bits)
    elif dtype == F16:
        v = bits.view(np.float16).astype(np.float32)
    else:
        v = decode_e4m3(bits)
    if scale is None:                 # stored without scales: the values are used as stored
        return v.astype(np.float32)
    return (v * scale.cpu().numpy().astype(np.float32)).astype(np.float32)
