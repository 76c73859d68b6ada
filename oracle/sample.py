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
"""
from __future__ import annotations

import numpy as np


def _wrap_or_clamp(i: np.ndarray, n: int, address: str) -> np.ndarray:
    if address == "clamp":
        return np.clip(i, 0, n - 1)
    if address == "wrap":
        return np.mod(i, n)
    raise ValueError(address)


def bilinear(tex: np.ndarray, u, v, shift: float = 0.0, address: str = "clamp") -> np.ndarray:
    """Bilinear sample of tex [H, W, C] (FP64 values) at (u, v); returns [n, C]."""
    tex = np.asarray(tex, dtype=np.float64)
    h, w = tex.shape[:2]
    x = np.asarray(u, dtype=np.float64) * w - 0.5 + shift
    y = np.asarray(v, dtype=np.float64) * h - 0.5 + shift
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = (x - x0)[..., None], (y - y0)[..., None]
    x0, y0 = x0.astype(np.int64), y0.astype(np.int64)
    xa, xb = _wrap_or_clamp(x0, w, address), _wrap_or_clamp(x0 + 1, w, address)
    ya, yb = _wrap_or_clamp(y0, h, address), _wrap_or_clamp(y0 + 1, h, address)
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
    """Texel-centre uv of a width x height output, row-major: u = (i + .5)/W, v = (j + .5)/H."""
    j, i = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    return ((i + 0.5) / width).reshape(-1), ((j + 0.5) / height).reshape(-1)


def features(level_tex: list, shifts, u, v, address: str = "clamp") -> np.ndarray:
    """x = [T_0(uv), ..., T_{L-1}(uv)] -> [n, 3L] FP64 (Sec. 3.1)."""
    return np.concatenate([bilinear(t, u, v, s, address) for t, s in zip(level_tex, shifts)], axis=-1)
