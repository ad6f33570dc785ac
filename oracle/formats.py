"""Rounding of FP64 values to the leaf operand formats: TEST INFRASTRUCTURE ONLY.

Written from the format definitions: a binary floating-point format with p significant
bits and minimum normal exponent emin represents x as a multiple of the quantum
2^(max(E, emin) - p + 1), E = floor(log2 |x|); round to nearest, ties to even (IEEE 754).
  BF16: p = 8,  emin = -126    FP16: p = 11, emin = -14    TF32: p = 11, emin = -126
Overflow is not handled (the workloads stay far inside every range). The split pair of
a value in a format is hi = fmt(x), lo = fmt(x - hi) (x - hi is exact in FP64: both are
multiples of the unit in the last place of x).
"""
import numpy as np

FORMATS = {"bf16": (8, -126), "fp16": (11, -14), "tf32": (11, -126)}


def round_to(x: np.ndarray, fmt: str) -> np.ndarray:
    p, emin = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    _, ex = np.frexp(x)                      # x = m 2^ex, 0.5 <= |m| < 1
    E = np.maximum(ex.astype(np.int64) - 1, emin)
    q = np.ldexp(1.0, (E - (p - 1)).astype(np.int32))
    return np.rint(x / q) * q                # rint: round half to even


def split(x: np.ndarray, fmt: str):
    hi = round_to(x, fmt)
    lo = round_to(np.asarray(x, dtype=np.float64) - hi, fmt)
    return hi, lo


def split_bf16(x: np.ndarray):
    return split(x, "bf16")
