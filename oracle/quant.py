"""Rounding to IEEE binary16 and to OCP FP8 E4M3, written from the format
definitions (not from any library): a finite value is rounded to the nearest
multiple of its binade's quantum, ties to even.

binary16 (IEEE 754-2008): 1 sign, 5 exponent bits (bias 15), 10 fraction bits;
normal binades 2^-14 .. 2^15 with quantum 2^(e - 10), subnormal quantum 2^-24;
largest finite 65504; results at or beyond 65520 overflow to infinity.

E4M3 (OCP 8-bit floating point specification, "FP8 E4M3"): 1 sign, 4 exponent
bits (bias 7), 3 fraction bits, no infinities; normal binades 2^-6 .. 2^8 with
quantum 2^(e - 3), subnormal quantum 2^-9; largest finite 448.  The kernels use
the saturating conversion: anything beyond 448 in magnitude becomes +-448.

Used by the quantisation emulator (the precision forms: weights and
activations in FP16 or FP8 E4M3 with FP32 accumulation, outputs in FP16).
"""
from __future__ import annotations

import numpy as np


def _round_to_quantum(x: np.ndarray, min_exp: int, frac_bits: int) -> np.ndarray:
    """Nearest multiple (ties to even) of the quantum 2^(e - frac_bits) of x's
    binade 2^e <= |x| < 2^(e+1), with e clamped below at min_exp (subnormals)."""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)  # x = m 2^e with 1/2 <= |m| < 1: the binade exponent is e - 1 (exact)
    q = np.ldexp(1.0, np.maximum(e - 1, min_exp) - frac_bits)
    return np.rint(x / q) * q  # x / q and the product are exact (powers of two); rint ties to even


def round_fp16(x) -> np.ndarray:
    """Nearest binary16 value (ties to even) as FP64; overflow gives +-inf."""
    r = _round_to_quantum(x, -14, 10)
    return np.where(np.abs(r) >= 65536.0, np.copysign(np.inf, r), r)


def round_e4m3_satfinite(x) -> np.ndarray:
    """Nearest E4M3 value (ties to even), saturated to +-448, as FP64."""
    r = _round_to_quantum(x, -6, 3)
    return np.clip(r, -448.0, 448.0)


def fp16_value(bits) -> np.ndarray:
    """Value of binary16 bit patterns (uint16) -> FP64."""
    b = np.asarray(bits, dtype=np.int64)
    s = np.where(b >> 15, -1.0, 1.0)
    e = (b >> 10) & 31
    f = b & 1023
    val = np.where(e == 0, np.ldexp(f.astype(np.float64), -24),
                   np.ldexp((1024 + f).astype(np.float64), (e - 25).astype(np.int64)))
    val = np.where(e == 31, np.where(f == 0, np.inf, np.nan), val)
    return s * val


def e4m3_value(bits) -> np.ndarray:
    """Value of E4M3 bit patterns (uint8) -> FP64 (S.1111.111 is NaN)."""
    b = np.asarray(bits, dtype=np.int64)
    s = np.where(b >> 7, -1.0, 1.0)
    e = (b >> 3) & 15
    f = b & 7
    val = np.where(e == 0, np.ldexp(f.astype(np.float64), -9),
                   np.ldexp((8 + f).astype(np.float64), (e - 10).astype(np.int64)))
    val = np.where((e == 15) & (f == 7), np.nan, val)
    return s * val


def pow2_ceil(x) -> np.ndarray:
    """Smallest power of two >= x (x > 0), FP64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m 2^e, m in [0.5, 1)
    return np.where(m == 0.5, x, np.ldexp(1.0, e))
