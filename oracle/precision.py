"""Host-side round-to-nearest-even into the solver's low-precision formats.

Test infrastructure (part of the CPU oracle).  Each routine rounds float64
values to the nearest value representable in the target format, ties to
even, and returns them as float64 so that the oracle's float64 arithmetic can
use them.  The formats are the IEEE/OCP definitions:

* fp32:  IEEE binary32 (8-bit exponent, 23-bit fraction)
* tf32:  binary32 exponent with a 10-bit fraction
* bf16:  binary32 exponent with a 7-bit fraction
* fp16:  IEEE binary16 (5-bit exponent, 10-bit fraction)
* e4m3:  OCP FP8 E4M3 (bias 7, no infinities, max 448), saturating
"""
from __future__ import annotations

import numpy as np


def to_fp32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _round_f32_mantissa(x, drop_bits: int):
    """Round binary32 values to a fraction of 23 - drop_bits bits (RNE)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    half = np.uint64(1 << (drop_bits - 1))
    lsb = (u >> np.uint64(drop_bits)) & np.uint64(1)
    u = (u + half - np.uint64(1) + lsb) >> np.uint64(drop_bits) << np.uint64(drop_bits)
    out = (u & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    # NaN / Inf pass through unchanged
    out = np.where(np.isfinite(f), out, f)
    return out.astype(np.float64)


def to_tf32(x):
    """Two roundings (float64 -> binary32 -> tf32) are what the GPU path does."""
    return _round_f32_mantissa(x, 13)


def to_bf16(x):
    return _round_f32_mantissa(x, 16)


def to_fp16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def _e4m3_grid():
    vals = [0.0]
    for e in range(16):
        for mnt in range(8):
            if e == 15 and mnt == 7:
                continue  # NaN encoding
            if e == 0:
                v = (mnt / 8.0) * 2.0 ** (1 - 7)
            else:
                v = (1.0 + mnt / 8.0) * 2.0 ** (e - 7)
            vals.append(v)
    g = np.unique(np.array(vals))
    return g


_E4M3 = _e4m3_grid()


def to_e4m3(x):
    """Nearest E4M3 value (ties to the even code), saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), 448.0)
    idx = np.searchsorted(_E4M3, a)
    idx = np.clip(idx, 1, len(_E4M3) - 1)
    lo, hi = _E4M3[idx - 1], _E4M3[idx]
    dlo, dhi = a - lo, hi - a
    # code parity: the grid index equals the magnitude code, so even index = even code
    pick_hi = (dhi < dlo) | ((dhi == dlo) & ((idx % 2) == 0))
    r = np.where(pick_hi, hi, lo)
    return np.copysign(r, x)


ROUND = {
    "fp64": lambda x: np.asarray(x, dtype=np.float64),
    "fp32": to_fp32,
    "tf32": to_tf32,
    "bf16": to_bf16,
    "fp16": to_fp16,
    "fp8": to_e4m3,
}

UNIT_ROUNDOFF = {
    "fp64": 2.0 ** -53,
    "fp32": 2.0 ** -24,
    "tf32": 2.0 ** -11,
    "fp16": 2.0 ** -11,
    "bf16": 2.0 ** -8,
    "fp8": 2.0 ** -4,
}
