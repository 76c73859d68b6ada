"""Whole decode of a material at given uv or on its texel-centre grid (Sec. 3.1):
BC1 decode of every latent level, bilinear sampling with the per-level shift,
concatenation, MLP.  Precision "fp64" is the plain definition; "fp16", "fp8"
and the split-operand "fp16s", "fp8s" are the quantisation emulator of the
precision forms."""
from __future__ import annotations

import numpy as np

from . import bc1, emulate, mlp, sample


def level_rgb(level, mip: int = 0) -> np.ndarray:
    w, h = level.width, level.height
    for _ in range(mip):
        w, h = max(4, w // 2), max(4, h // 2)
    return bc1.decode_level(level.blocks[mip], w, h).astype(np.float64) / 255.0


def features_at(material, u, v, tex=None) -> np.ndarray:
    tex = tex if tex is not None else [level_rgb(lv) for lv in material.levels]
    return sample.features(tex, [lv.shift for lv in material.levels], u, v, material.address)


def run_mlp(material, x, precision: str = "fp64", fp8=None):
    m = material.mlp
    if precision == "fp64":
        return mlp.forward(x, m.weights, m.biases)
    if precision == "fp16":
        return emulate.forward_fp16(x, m.weights, m.biases)
    if precision == "fp8":
        sw, sa = fp8
        return emulate.forward_fp8(x, m.weights, m.biases, sw, sa)
    if precision == "fp16s":
        return emulate.forward_fp16_split(x, m.weights, m.biases)
    if precision == "fp8s":
        sw, sa = fp8
        return emulate.forward_fp8_split(x, m.weights, m.biases, sw, sa)
    raise ValueError(precision)


def mlp_interval(material, x, precision: str, fp8=None, **error_model):
    """(y, y_min, y_max) of a precision form: emulated FP16 output and the outputs
    admissible under the FP32 error model of `emulate.output_interval`."""
    m = material.mlp
    return emulate.output_interval(precision, x, m.weights, m.biases, fp8, **error_model)


def decode_uv(material, uv: np.ndarray, precision: str = "fp64", fp8=None, tex=None) -> np.ndarray:
    x = features_at(material, uv[:, 0].astype(np.float64), uv[:, 1].astype(np.float64), tex)
    return run_mlp(material, x, precision, fp8)


def decode_grid(material, width: int, height: int, idx=None, precision: str = "fp64",
                fp8=None, tex=None) -> np.ndarray:
    """Decode texel-centre outputs; idx = linear texel indices (row-major) or all."""
    if idx is None:
        idx = np.arange(width * height)
    idx = np.asarray(idx, dtype=np.int64)
    u = sample.grid_coord(idx % width, width).astype(np.float64)
    v = sample.grid_coord(idx // width, height).astype(np.float64)
    x = features_at(material, u, v, tex)
    return run_mlp(material, x, precision, fp8)


def fp8_calibration(material, width: int, height: int, step: int = 16, tex=None):
    """(sw, sa) power-of-two FP8 scales from the sub-grid of every `step`-th texel."""
    j, i = np.meshgrid(np.arange(0, height, step), np.arange(0, width, step), indexing="ij")
    idx = (j * width + i).reshape(-1)
    u = sample.grid_coord(idx % width, width).astype(np.float64)
    v = sample.grid_coord(idx // width, height).astype(np.float64)
    x = features_at(material, u, v, tex)
    acts = mlp.hidden_activations(x, material.mlp.weights, material.mlp.biases)
    return emulate.fp8_scales(material.mlp.weights, acts)
