"""Low-precision codec of Sec. 3.2 (Eq. 1, Table 1) -- TEST INFRASTRUCTURE ONLY.

Eq. 1, per group i of a real tensor T (complex tensors as their interleaved
real and imaginary parts):

    Q([T]_i) = [T]_i^exp * scale + zero,
    scale = (q_max - q_min) / (max [T]_i - min [T]_i),
    zero  = (q_min max [T]_i - q_max min [T]_i) / (max [T]_i - min [T]_i).

Table 1 kinds: "half" (exp 1, one group = the whole tensor, no rounding,
stored as FP16), "int8" (-128..127, exp 0.2, whole tensor, rounded),
"int4" (0..15, exp 1, groups, rounded; two codes per byte).  Readings
where the paper is silent, ambiguous or garbled:

* the half range printed as +-6.65e4 lies above FP16's largest finite value
  (65504, i.e. 6.55e4); +-65504 is used;
* x^exp of a negative x is sign(x) |x|^exp, and max / min in scale and zero
  are taken over the transformed values, so a group's transformed range
  maps exactly onto [q_min, q_max];
* rounding is to nearest, ties to even, then clamped to [q_min, q_max];
  a group whose values are all equal gets scale 1 and zero q_min - value;
* decoding inverts Eq. 1: y = (q - zero) / scale, x = sign(y) |y|^(1/exp).

The decisions that produce integer codes are taken in FP32 here, in the
order the formulas are written, as the GPU kernels take them (the paper
fixes no precision); values and error bounds are checked in FP64.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

KINDS: Dict[str, Tuple[float, float, float, bool]] = {
    # q_min, q_max, exp, rounded
    "half": (-65504.0, 65504.0, 1.0, False),
    "int8": (-128.0, 127.0, 0.2, True),
    "int4": (0.0, 15.0, 1.0, True),
}


def transform(x: np.ndarray, exp: float) -> np.ndarray:
    """sign(x) |x|^exp in FP32."""
    x = np.asarray(x, dtype=np.float32)
    if exp == 1.0:
        return x
    return (np.sign(x) * np.power(np.abs(x), np.float32(exp))).astype(np.float32)


def encode(x: np.ndarray, kind: str, group: int = 0):
    """Quantize the real array x (flattened) in groups of ``group`` values
    (0: one group).  Returns (codes, scale, zero): codes int32 (or float16
    for "half"), one scale and zero (float32) per group."""
    q_min, q_max, exp, rounded = KINDS[kind]
    x = np.asarray(x, dtype=np.float32).ravel()
    g = x.size if group <= 0 else group
    if x.size % g:
        raise ValueError("the tensor must hold a whole number of groups")
    y = transform(x, exp).reshape(-1, g)
    lo = y.min(axis=1)
    hi = y.max(axis=1)
    span = (hi - lo).astype(np.float32)
    flat = span == 0
    safe = np.where(flat, np.float32(1), span).astype(np.float32)
    scale = np.where(flat, np.float32(1), np.float32(q_max - q_min) / safe).astype(np.float32)
    zero = np.where(flat, np.float32(q_min) - lo,
                    (np.float32(q_min) * hi - np.float32(q_max) * lo) / safe).astype(np.float32)
    v = (y * scale[:, None] + zero[:, None]).astype(np.float32)
    if rounded:
        codes = np.clip(np.rint(v), q_min, q_max).astype(np.int32)
    else:
        codes = v.astype(np.float16)
    return codes.reshape(-1), scale, zero


def decode(codes: np.ndarray, scale: np.ndarray, zero: np.ndarray, kind: str, group: int = 0) -> np.ndarray:
    """Invert Eq. 1 (FP64): x = sign(y) |y|^(1/exp), y = (q - zero) / scale."""
    q_min, q_max, exp, _ = KINDS[kind]
    q = np.asarray(codes, dtype=np.float64)
    g = q.size if group <= 0 else group
    q = q.reshape(-1, g)
    y = (q - np.asarray(zero, dtype=np.float64)[:, None]) / np.asarray(scale, dtype=np.float64)[:, None]
    if exp != 1.0:
        y = np.sign(y) * np.power(np.abs(y), 1.0 / exp)
    return y.reshape(-1)


def pack_int4(codes: np.ndarray) -> np.ndarray:
    """Two 4-bit codes per byte, the even-indexed one in the low nibble."""
    c = np.asarray(codes, dtype=np.uint8).reshape(-1, 2)
    return (c[:, 0] | (c[:, 1] << 4)).astype(np.uint8)


def unpack_int4(packed: np.ndarray) -> np.ndarray:
    p = np.asarray(packed, dtype=np.uint8)
    return np.stack([p & 15, p >> 4], axis=1).reshape(-1).astype(np.int32)
