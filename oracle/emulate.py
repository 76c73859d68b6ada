"""Quantisation emulator for the precision forms of the decode.

The precision forms run the MLP layers with FP16 (or FP8 E4M3) weights and
activations, accumulate in FP32 and write FP16 outputs.  This emulator rounds
exactly the same operands the kernels round -- the 12 input features, every
weight, every hidden activation after ReLU, and the final output -- with the
conversions of `quant` (written from the format definitions), but accumulates
each dot product exactly (FP64; products of FP16 / E4M3 values are exact in
FP64 and the sums carry at most a 2^-53 relative error).

Bias: the FP16 form feeds the bias to the tensor core like a weight (a column
of ones in A, the bias in B), so the bias is an FP16 operand too and is rounded
here; the FP8 form adds the FP32 bias in its FP32 epilogue, added here in FP64.

It therefore separates the error that the precision itself costs (emulator vs
FP64 oracle) from the error of the kernel's arithmetic (kernel vs emulator:
FP32 accumulation order and, rarely, a rounding decision that an FP32
intermediate flips).

FP8 scales (the paper names no scheme; fixed here): per layer l a weight scale
sw_l and an input-activation scale sa_l, both powers of two so that scaling is
exact on every side:
  sw_l = pow2_ceil(absmax(W_l) / 448),
  sa_l = pow2_ceil(absmax of layer l's input over a calibration set / 448),
where the calibration set is the FP32/FP64 decode of a sub-grid (every 16th
texel in x and y) of the same material.  A layer computes
  q(x) = E4M3(x / sa_l),  Wq = E4M3(W_l / sw_l),
  z = (Wq q) * sw_l * sa_l + b_l,  next input = ReLU(z).
"""
from __future__ import annotations

import numpy as np

from . import quant


def forward_fp16(x: np.ndarray, weights: list, biases: list, round_output: bool = True) -> np.ndarray:
    h = quant.round_fp16(np.asarray(x, dtype=np.float64))
    n = len(weights)
    for l, (w, b) in enumerate(zip(weights, biases)):
        w16 = quant.round_fp16(np.asarray(w, dtype=np.float64))
        z = h @ w16.T + quant.round_fp16(np.asarray(b, dtype=np.float64))
        if l < n - 1:
            h = quant.round_fp16(np.maximum(z, 0.0))
        else:
            h = quant.round_fp16(z) if round_output else z
    return h


def fp8_scales(weights: list, calib_inputs: list):
    """(sw, sa) per layer from the weights and the calibration-set layer inputs."""
    sw = [float(quant.pow2_ceil(np.max(np.abs(np.asarray(w, dtype=np.float64))) / 448.0)) for w in weights]
    sa = [float(quant.pow2_ceil(max(np.max(np.abs(a)), 2.0 ** -126) / 448.0)) for a in calib_inputs]
    return sw, sa


def forward_fp8(x: np.ndarray, weights: list, biases: list, sw: list, sa: list,
                round_output: bool = True) -> np.ndarray:
    h = np.asarray(x, dtype=np.float64)
    n = len(weights)
    for l, (w, b) in enumerate(zip(weights, biases)):
        q = quant.round_e4m3_satfinite(h / sa[l])
        wq = quant.round_e4m3_satfinite(np.asarray(w, dtype=np.float64) / sw[l])
        z = (q @ wq.T) * (sw[l] * sa[l]) + np.asarray(b, dtype=np.float64)
        if l < n - 1:
            h = np.maximum(z, 0.0)
        else:
            h = quant.round_fp16(z) if round_output else z
    return h
