"""Gaussian stage Y2 = Omega Y1 (Sec. 1.2.1) and the precision modes' operand
rounding.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

The paper's Gaussian ID sketches with an L x I matrix of iid N(0,1) entries.
Here the Gaussian matrix Omega (m2 x m1) is applied to the CountSketch output
Y1 (m1 x R).  With m2 = 0 the stage is skipped (Y2 = Y1), which is the paper's
Algorithm 2 exactly.

Precision modes (the operands each mode multiplies; the product itself is
formed here in float64):
  FP64   : Omega (float64)            times Y1
  FP32   : fl32(Omega)                times Y1      (fp32 working copy of Omega)
  BF16X3 : fl32(Omega)                times Y1      (same definition; the device
                                                     forms it from bf16 splits)
  BF16   : bf16(fl32(Omega))          times bf16(fl32(Y1))
  TF32X3 : fl32(Omega)                times Y1      (same definition; the device
                                                     forms it from two-term TF32
                                                     splits, three products)

FP8 (e4m3) operands are not a mode of the library; ``round_e4m3`` and
``fp8_operand`` state what such a mode would multiply (per-tensor scaling to the
format's largest finite value, 448), so that its error can be measured against
the FP64 oracle.
"""
from __future__ import annotations

import numpy as np

FP64, FP32, BF16X3, BF16, TF32X3 = 0, 1, 2, 3, 4


def round_bf16(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float32.  bfloat16 keeps the top 16 bits of the IEEE binary32 pattern."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32)


def gaussian_operand(Omega64: np.ndarray, precision: int) -> np.ndarray:
    """The Gaussian matrix as the given precision mode multiplies it (float64 array)."""
    if precision == FP64:
        return np.asarray(Omega64, dtype=np.float64)
    o32 = np.asarray(Omega64, dtype=np.float64).astype(np.float32)
    if precision == BF16:
        return round_bf16(o32).astype(np.float64)
    return o32.astype(np.float64)


def gaussian_stage(Omega64: np.ndarray, Y1: np.ndarray, precision: int = FP64) -> np.ndarray:
    """Y2 = Omega Y1 in float64 (plain matrix product of the mode's operands)."""
    Om = gaussian_operand(Omega64, precision)
    Y = np.asarray(Y1, dtype=np.float64)
    if precision == BF16:
        Y = round_bf16(Y.astype(np.float32)).astype(np.float64)
    return Om @ Y


def round_e4m3(x) -> np.ndarray:
    """Round to the nearest FP8 e4m3 value (1 sign, 4 exponent bits with bias 7, 3
    mantissa bits; subnormals down to 2^-9; largest finite 448), ties to even,
    saturating at 448; returned as float64."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.clip(np.floor(np.log2(np.maximum(a, 2.0 ** -9))), -6, 8)
    q = 2.0 ** (e - 3)                       # spacing of the binade (subnormal spacing 2^-9)
    r = np.minimum(np.round(a / q) * q, 448.0)
    return np.sign(x) * r


def fp8_operand(X) -> np.ndarray:
    """X scaled so that its largest magnitude is 448, rounded to e4m3, scaled back."""
    X = np.asarray(X, dtype=np.float64)
    m = np.abs(X).max()
    if m == 0:
        return X.copy()
    s = 448.0 / m
    return round_e4m3(X * s) / s
