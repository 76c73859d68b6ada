"""Quantisation emulator for the precision forms of the decode -- TEST
INFRASTRUCTURE (part of the oracle).

The precision forms run the MLP layers with FP16 (or FP8 E4M3) weights and
activations, accumulate in FP32 and write FP16 outputs; the split forms carry
every operand as a hi + lo pair of the narrow format (below).  This emulator rounds
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


# --------------------------------------------------------------------------- split operands
#
# The split forms carry every operand as a pair of narrow numbers, hi + lo, and
# run three products per layer -- hi(A) hi(W) + lo(A) hi(W) + hi(A) lo(W) --
# into one FP32 accumulator; lo(A) lo(W) is dropped (it lies below the
# accumulator's own rounding).  Every multiply still reads the narrow format
# (Sec. 4 runs the MLP on matrix units); the pair restores most of the
# precision a single rounding loses.
#
# FP16 split:  hi = RN16(v), lo = RN16(v - hi) (v - hi is exact); the bias
#              enters the products as an hi and a lo operand too.
# FP8 split:   the scaled value is first narrowed to FP16, v16 = RN16(v / s),
#              then hi = E4M3(v16), lo = E4M3(v16 - hi) (v16 - hi is exact in
#              FP16), both saturating; layer scales, FP32 bias and epilogue are
#              those of the FP8 form.


def split_fp16(v):
    """(hi, lo) FP16 pair of v: hi = RN16(v), lo = RN16(v - hi)."""
    v = np.asarray(v, dtype=np.float64)
    hi = quant.round_fp16(v)
    return hi, quant.round_fp16(v - hi)


def split_e4m3(v):
    """(hi, lo) E4M3 pair of an already scaled v: v16 = RN16(v), hi = E4M3(v16),
    lo = E4M3(v16 - hi)."""
    v16 = quant.round_fp16(np.asarray(v, dtype=np.float64))
    hi = quant.round_e4m3_satfinite(v16)
    return hi, quant.round_e4m3_satfinite(v16 - hi)


def forward_fp16_split(x: np.ndarray, weights: list, biases: list, round_output: bool = True) -> np.ndarray:
    ah, al = split_fp16(x)
    n = len(weights)
    for l, (w, b) in enumerate(zip(weights, biases)):
        wh, wl = split_fp16(w)
        bh, bl = split_fp16(b)
        z = ah @ wh.T + al @ wh.T + ah @ wl.T + bh + bl
        if l < n - 1:
            ah, al = split_fp16(np.maximum(z, 0.0))
    return quant.round_fp16(z) if round_output else z


def forward_fp8_split(x: np.ndarray, weights: list, biases: list, sw: list, sa: list,
                      round_output: bool = True) -> np.ndarray:
    qh, ql = split_e4m3(np.asarray(x, dtype=np.float64) / sa[0])
    n = len(weights)
    for l, (w, b) in enumerate(zip(weights, biases)):
        wh, wl = split_e4m3(np.asarray(w, dtype=np.float64) / sw[l])
        z = (qh @ wh.T + ql @ wh.T + qh @ wl.T) * (sw[l] * sa[l]) + np.asarray(b, dtype=np.float64)
        if l < n - 1:
            qh, ql = split_e4m3(np.maximum(z, 0.0) / sa[l + 1])
    return quant.round_fp16(z) if round_output else z


# --------------------------------------------------------------------------- admissible outputs
#
# A kernel takes the same roundings as the emulator but forms the values it
# rounds -- features, accumulated dot products, scaled epilogue values -- in
# FP32.  Where such a value lies near a rounding boundary of the narrow format
# the kernel may land on the other side and carry another, equally correct,
# narrow operand into the rest of the network (several results are correct
# there).  `output_interval` gives, per output, the interval of FP16 values a
# kernel may produce; it is the emulator's single value (up to the output's own
# rounding) wherever no rounding decision is in doubt.
#
# Error model (its parameters are arguments):
#  - FP32 noise: the kernel's feature deviates from the exact one by noise of
#    standard deviation sigma_x; an FP32 sum of n exact products and a bias by
#    noise of standard deviation 2^-24 sqrt(n) sqrt(sum of squared terms)
#    (independent roundings of at most half an FP32 unit of the partial sums;
#    times acc_scale for a tensor-core kind whose accumulator is coarser);
#    noise passes a near-identity operand representation (the FP16 split, whose
#    own lo rounding adds as noise too) and adds in quadrature through a dot
#    product.  A value is in doubt within k standard deviations.
#  - Flips: a representation that is constant between rounding boundaries
#    (FP16, E4M3, and the FP8 split, constant on FP16 cells) carries a value
#    that may jump wherever a boundary lies within the value's doubt; the jump
#    is the representation's largest change over that range, and jumps reach
#    the next layer through |W| (each in its worst direction) and add to its
#    doubt.
#  - The FP16 split's lo(W) multiplies hi(A) alone, so a hi that flips (lo
#    taking up the rest) moves the sum by that hi's change times |lo(W)|.

FORMS = ("fp16", "fp16s", "fp8", "fp8s")


def _rep(form: str, v):
    """Value a rounding site carries into the next products (scaled units for FP8)."""
    if form == "fp16":
        return quant.round_fp16(v)
    if form == "fp8":
        return quant.round_e4m3_satfinite(v)
    hi, lo = split_fp16(v) if form == "fp16s" else split_e4m3(v)
    return hi + lo


def _parts(form: str, v):
    """Operands of the products: (hi, lo) for the split forms, (value, 0) otherwise."""
    if form == "fp16s":
        return split_fp16(v)
    if form == "fp8s":
        return split_e4m3(v)
    r = _rep(form, v)
    return r, np.zeros_like(r)


def _change(f, v, p):
    """Largest change of the monotone function f over [v - p, v + p]."""
    r = f(v)
    return np.maximum(np.abs(f(v + p) - r), np.abs(f(v - p) - r))


def output_interval(form: str, x: np.ndarray, weights: list, biases: list, scales=None,
                    sigma_x: float = 2.0 ** -24, k: float = 6.0, acc_scale=None):
    """(y, y_min, y_max): the emulated FP16 output of `form` and the interval of
    FP16 outputs admissible for a kernel under the error model above.
    scales = (sw, sa) for the FP8 forms; acc_scale = accumulation noise in units
    of FP32 round-to-nearest (default: 1 for the FP16 forms, 4 for the E4M3 forms,
    whose tensor-core accumulation measures about two bits coarser)."""
    assert form in FORMS
    fp8 = form in ("fp8", "fp8s")
    if acc_scale is None:
        acc_scale = 4.0 if fp8 else 1.0
    split = form in ("fp16s", "fp8s")
    dense = form == "fp16s"            # representation ~ identity: noise passes through
    n = len(weights)
    sw, sa = scales if fp8 else ([1.0] * n, [1.0] * (n + 1))
    v = np.asarray(x, dtype=np.float64) / sa[0]
    sig = np.full_like(v, sigma_x / sa[0])   # noise of the value a site rounds
    jmp = np.zeros_like(v)                   # flips reaching it from upstream
    for l, (w, b) in enumerate(zip(weights, biases)):
        ah, al = _parts(form, v)
        doubt = jmp + k * sig
        if dense:
            # the carried value follows the kernel's own value: noise and jumps
            # pass on; the split's own rounding (lo, at most 2^-22 |v| + 2^-25)
            # differs between nearby values and adds as noise
            carried_sig = np.sqrt(sig ** 2 + (2.0 ** -22 * np.abs(v) + 2.0 ** -25) ** 2)
            carried_jmp = jmp
        else:
            carried_sig = 0.0 * sig
            carried_jmp = _change(lambda t: _rep(form, t), v, doubt)
        dhi = _change(lambda t: _parts(form, t)[0], v, doubt) if split else 0.0 * v
        w = np.asarray(w, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        wh, wl = _parts(form, w / sw[l])
        if fp8:
            bh, bl, bias = 0.0, 0.0, b
        else:
            bh, bl = _parts(form, b)
            bias = 0.0
        s = sw[l] * sa[l]
        z = (ah @ wh.T + al @ wh.T + ah @ wl.T + bh + bl) * s + bias
        sq = (ah ** 2 @ (wh ** 2).T + al ** 2 @ (wh ** 2).T + ah ** 2 @ (wl ** 2).T + bh ** 2 + bl ** 2) * s * s
        nterms = (3 if split else 1) * w.shape[1] + (0 if fp8 else (2 if split else 1))
        sig_z = np.sqrt(carried_sig ** 2 @ ((wh + wl) ** 2).T * s * s + nterms * (acc_scale * 2.0 ** -24) ** 2 * sq)
        if fp8:   # the FP32 scale-and-bias FMA of the epilogue
            sig_z = np.sqrt(sig_z ** 2 + (2.0 ** -24 * (np.abs(z) + np.abs(b))) ** 2)
        jmp_z = (carried_jmp @ np.abs(wh + wl).T + dhi @ np.abs(wl).T) * s
        if l < n - 1:
            v = np.maximum(z, 0.0) / sa[l + 1]    # ReLU is monotone and 1-Lipschitz
            sig, jmp = sig_z / sa[l + 1], jmp_z / sa[l + 1]
    p = jmp_z + k * sig_z
    return quant.round_fp16(z), quant.round_fp16(z - p), quant.round_fp16(z + p)
