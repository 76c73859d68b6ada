"""Latent sampling T_k(uv) and feature concatenation, FP64.

Paper Sec. 3.1: a texel at uv is decoded by sampling each latent texture
c_k = T_k(uv) and concatenating x = [c_0 ... c_K]; Sec. 3.2 samples latents the
way a texture unit does (bilinear within a level, trilinear across mips);
Sec. 3.1 ("Variants") shifts the 2nd and 4th latent textures by half a texel.

Conventions fixed here (the paper is silent): u runs along x (columns), v along
y (rows), origin at the top-left corner; texel centres sit at half-integers, so
the continuous texel coordinate is x = u * W - 0.5 + s (s = per-level shift in
texels, both axes); neighbours x0 = floor(x), x0 + 1 are clamped to [0, W - 1]
(clamp) or taken modulo W (wrap).

Coordinate precision (a reading: the decode samples at FP32 texture
coordinates, the uv a shader hands its texture fetch): the texel coordinate x is
the exact value of u * W - 0.5 + s rounded once to FP32, and a grid's texel-
centre coordinate is (i + 1/2) / W correctly rounded to FP32.  Which texels are
read and with which weights is then decided in the same precision as on the
GPU; the blend and everything after it are FP64.  With power-of-two sizes both
roundings are exact.
"""
from __future__ import annotations

import numpy as np


def _wrap_or_clamp(i: np.ndarray, n: int, address: str) -> np.ndarray:
    if address == "clamp":
        return np.clip(i, 0, n - 1)
    if address == "wrap":
        return np.mod(i, n)
    raise ValueError(address)


def texel_coord(u, n: int, shift: float) -> np.ndarray:
    """u * n - 0.5 + shift (exact in FP64 for an FP32 u and n < 2^24) rounded once to FP32."""
    return (np.asarray(u, dtype=np.float64) * n - 0.5 + shift).astype(np.float32).astype(np.float64)


def axis_taps(u, n: int, shift: float, address: str):
    """Neighbour indices (i0, i1) and weight f of i1 along one axis.  u is taken
    as FP32; wrap first drops its whole periods (u - floor(u), an FP32
    subtraction), so tiled coordinates keep their fraction; then the texel
    coordinate is rounded once to FP32 (texel_coord) and split into floor and
    fraction (exact); indices are clamped or wrapped as integers."""
    u = np.asarray(u, dtype=np.float64).astype(np.float32)
    if address == "wrap":
        u = u - np.floor(u)
    x = texel_coord(u.astype(np.float64), n, shift)
    x0 = np.floor(x)
    f = x - x0
    x0 = x0.astype(np.int64)
    return _wrap_or_clamp(x0, n, address), _wrap_or_clamp(x0 + 1, n, address), f


def grid_coord(i, n: int) -> np.ndarray:
    """Texel-centre coordinate (i + 1/2) / n correctly rounded to FP32 (IEEE FP32 division)."""
    return (np.asarray(i, dtype=np.float32) + np.float32(0.5)) / np.float32(n)


def bilinear(tex: np.ndarray, u, v, shift: float = 0.0, address: str = "clamp") -> np.ndarray:
    """Bilinear sample of tex [H, W, C] (FP64 values) at (u, v); returns [n, C]."""
    tex = np.asarray(tex, dtype=np.float64)
    h, w = tex.shape[:2]
    xa, xb, fx = axis_taps(u, w, shift, address)
    ya, yb, fy = axis_taps(v, h, shift, address)
    fx, fy = fx[..., None], fy[..., None]
    return ((1 - fx) * (1 - fy) * tex[ya, xa] + fx * (1 - fy) * tex[ya, xb]
            + (1 - fx) * fy * tex[yb, xa] + fx * fy * tex[yb, xb])


def trilinear(mips: list, u, v, lod, shift: float = 0.0, address: str = "wrap") -> np.ndarray:
    """Mip-mapped sample: lod clamped to [0, len(mips) - 1]; the bilinear samples of
    mips floor(lod) and floor(lod) + 1 (capped at the last mip) are blended by
    frac(lod).  The shift is in texels of each mip."""
    lod = np.clip(np.asarray(lod, dtype=np.float64), 0.0, len(mips) - 1)
    m0 = np.floor(lod).astype(np.int64)
    m1 = np.minimum(m0 + 1, len(mips) - 1)
    t = (lod - m0)[..., None]
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros(u.shape + (mips[0].shape[2],))
    for m in np.unique(np.concatenate([m0, m1])):
        s = bilinear(mips[m], u, v, shift, address)
        out += np.where((m0 == m)[..., None], 1 - t, 0.0) * s + np.where((m1 == m)[..., None], t, 0.0) * s
    return out


def grid_uv(width: int, height: int):
    """Texel-centre uv of a width x height output, row-major: u = (i + .5)/W, v = (j + .5)/H
    (each rounded to FP32, see grid_coord)."""
    j, i = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    return grid_coord(i, width).astype(np.float64).reshape(-1), grid_coord(j, height).astype(np.float64).reshape(-1)


def features(level_tex: list, shifts, u, v, address: str = "clamp") -> np.ndarray:
    """x = [T_0(uv), ..., T_{L-1}(uv)] -> [n, 3L] FP64 (Sec. 3.1)."""
    return np.concatenate([bilinear(t, u, v, s, address) for t, s in zip(level_tex, shifts)], axis=-1)
