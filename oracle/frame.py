"""Multi-material frame: tile classification, binning and per-pixel decode.

Paper Sec. 4 ("Tile-based classification") and Algorithm 1: the screen is cut
into tiles; pass A marks each tile as having no neural pixel, one network for
all its valid pixels and more than half of them valid ("uniform"), or anything
else ("mixed"); pass B gives every valid pixel of a mixed tile a slot in a
per-network packed list, so that networks run on tiles whose pixels share one
MLP.  The slot offsets per network are an exclusive prefix sum of the
per-network counts (Algorithm 1 reads them but does not say how they are
made).  Here a tile is 128 pixels (tile_w x tile_h) and each network's packed
list starts on a multiple of 128 slots, so every packed tile holds one network.

The per-pixel decode follows Sec. 3.1 with the texture unit's mip-mapped
filter of Sec. 3.2 / Sec. 3.3: per latent level k, lod_k = lod + log2(W_k)
(lod = log2 of the uv footprint of one pixel, plus the mip bias), clamped to
the level's mip range, trilinear with wrap addressing; the MLP runs in the
FP16 form (see `emulate`).
"""
from __future__ import annotations

import numpy as np

from . import bc1, emulate
from . import sample
from .sample import trilinear

EMPTY, UNIFORM, MIXED = 0, 1, 2


def classify(mat_id: np.ndarray, tile_w: int, tile_h: int):
    """Per tile (row-major over tiles): (kind, material of a uniform tile or -1)."""
    h, w = mat_id.shape
    assert h % tile_h == 0 and w % tile_w == 0
    t = mat_id.reshape(h // tile_h, tile_h, w // tile_w, tile_w).transpose(0, 2, 1, 3)
    t = t.reshape(-1, tile_w * tile_h).astype(np.int64)
    valid = t >= 0
    count = valid.sum(axis=1)
    big = np.iinfo(np.int64).max
    mn = np.where(valid, t, big).min(axis=1)
    mx = np.where(valid, t, -1).max(axis=1)
    kind = np.where(count == 0, EMPTY, np.where((mn == mx) & (count * 2 > tile_w * tile_h), UNIFORM, MIXED))
    mat = np.where(kind == UNIFORM, mn, -1)
    return kind, mat


def tile_pixels(tile: int, w: int, tile_w: int, tile_h: int) -> np.ndarray:
    """Linear pixel indices of a tile, row-major inside the tile."""
    tiles_x = w // tile_w
    ty, tx = divmod(tile, tiles_x)
    yy, xx = np.meshgrid(np.arange(tile_h), np.arange(tile_w), indexing="ij")
    return ((ty * tile_h + yy) * w + tx * tile_w + xx).reshape(-1)


def mixed_counts(mat_id: np.ndarray, kind: np.ndarray, tile_w: int, tile_h: int, m: int):
    """Per-material count of valid pixels lying in mixed tiles, and the exclusive
    scan of those counts rounded up to whole 128-slot tiles (slot offsets)."""
    h, w = mat_id.shape
    flat = mat_id.reshape(-1)
    counts = np.zeros(m, dtype=np.int64)
    for tile in np.nonzero(kind == MIXED)[0]:
        ids = flat[tile_pixels(tile, w, tile_w, tile_h)]
        ids = ids[ids >= 0]
        counts += np.bincount(ids, minlength=m)
    per = tile_w * tile_h
    padded = (counts + per - 1) // per * per
    offsets = np.concatenate([[0], np.cumsum(padded)[:-1]])
    return counts, offsets


def decode_pixels(material, levels_mips_rgb: list, uv: np.ndarray, lod: np.ndarray,
                  precision: str = "fp16") -> np.ndarray:
    """Decode the given pixels of one material: uv [n, 2], lod [n] -> [n, N]."""
    u, v = uv[:, 0].astype(np.float64), uv[:, 1].astype(np.float64)
    feats = []
    for lv, mips in zip(material.levels, levels_mips_rgb):
        lam = lod.astype(np.float64) + np.log2(float(lv.width))
        feats.append(trilinear(mips, u, v, lam, lv.shift, material.address))
    x = np.concatenate(feats, axis=-1)
    mlp = material.mlp
    if precision == "fp16":
        return emulate.forward_fp16(x, mlp.weights, mlp.biases)
    from . import mlp as mlp_mod
    return mlp_mod.forward(x, mlp.weights, mlp.biases)


def level_mips_rgb(level) -> list:
    """Decoded mips of a BC1 latent level as FP64 [h, w, 3] in [0, 1]."""
    out = []
    w, h = level.width, level.height
    for blocks in level.blocks:
        out.append(bc1.decode_level(blocks, w, h).astype(np.float64) / 255.0)
        w, h = max(4, w // 2), max(4, h // 2)
    return out


def _bilinear_bc1(level_blocks, w, h, u, v, shift, address):
    """Bilinear sample of one BC1 mip (w x h) at (u, v), fetching only the four
    texels each sample needs (same filter as sample.bilinear)."""
    xa, xb, fx = sample.axis_taps(u, w, shift, address)
    ya, yb, fy = sample.axis_taps(v, h, shift, address)
    fx, fy = fx[..., None], fy[..., None]
    t = lambda xx, yy: bc1.texel_rgb8(level_blocks, w, xx, yy).astype(np.float64) / 255.0
    return ((1 - fx) * (1 - fy) * t(xa, ya) + fx * (1 - fy) * t(xb, ya)
            + (1 - fx) * fy * t(xa, yb) + fx * fy * t(xb, yb))


def pixel_features_direct(material, uv: np.ndarray, lod: np.ndarray) -> np.ndarray:
    """[n, 12] trilinear features of the given pixels, each tap's BC1 texel
    decoded on demand (for spot checks of large frames)."""
    u, v = uv[:, 0].astype(np.float64), uv[:, 1].astype(np.float64)
    feats = []
    for lv in material.levels:
        mips = lv.num_mips
        lam = np.clip(lod.astype(np.float64) + np.log2(float(lv.width)), 0.0, mips - 1)
        m0 = np.floor(lam).astype(np.int64)
        m1 = np.minimum(m0 + 1, mips - 1)
        t = (lam - m0)[:, None]
        acc = np.zeros((len(u), 3))
        w, h = lv.width, lv.height
        for m in range(mips):
            sel0, sel1 = m0 == m, m1 == m
            sel = sel0 | sel1
            if np.any(sel):
                smp = _bilinear_bc1(lv.blocks[m], w, h, u[sel], v[sel], lv.shift, material.address)
                wt = np.where(sel0[sel][:, None], 1 - t[sel], 0.0) + np.where(sel1[sel][:, None], t[sel], 0.0)
                acc[sel] += wt * smp
            w, h = max(4, w // 2), max(4, h // 2)
        feats.append(acc)
    return np.concatenate(feats, axis=-1)


def decode_pixels_direct(material, uv: np.ndarray, lod: np.ndarray, precision: str = "fp16") -> np.ndarray:
    """decode_pixels without decoding whole mips (see pixel_features_direct)."""
    x = pixel_features_direct(material, uv, lod)
    mlp = material.mlp
    if precision == "fp16":
        return emulate.forward_fp16(x, mlp.weights, mlp.biases)
    from . import mlp as mlp_mod
    return mlp_mod.forward(x, mlp.weights, mlp.biases)


def aniso_count(duv: np.ndarray, max_aniso: int):
    """Anisotropic filter of the latents (Sec. 3.2, "Anisotropic Filtering"): the
    paper uses the texture unit's anisotropic filter on the latents unchanged;
    this restates the reference formulas of the anisotropic-filtering extension
    (EXT_texture_filter_anisotropic): with Px = |d(u,v)/dx|, Py = |d(u,v)/dy|,
    Pmax = max, Pmin = min, N = min(ceil(Pmax / Pmin), max_aniso) probes along the
    major axis, lod = log2(Pmax / N).  Computed in texture-coordinate units (the
    square latents make the ratio the same for every level).  N is an integer
    decided by floating point, so it is decided here in FP32 with the kernel's
    operation order (products, sum, square root, quotient, ceil -- all correctly
    rounded).  Returns (N [n], along_x [n] bool, Pmax [n] FP32)."""
    d = np.asarray(duv, dtype=np.float32)
    px = np.sqrt(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1])
    py = np.sqrt(d[..., 2] * d[..., 2] + d[..., 3] * d[..., 3])
    along_x = px >= py
    pmax = np.where(along_x, px, py)
    pmin = np.where(along_x, py, px)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.ceil(pmax / pmin)
    n = np.where(pmax > 0, np.where(pmin > 0, np.minimum(ratio, np.float32(max_aniso)), max_aniso), 1)
    return n.astype(np.int64), along_x, pmax


def aniso_features(material, levels_mips_rgb: list, uv: np.ndarray, duv: np.ndarray, bias: np.ndarray,
                   max_aniso: int) -> np.ndarray:
    """[n, 12] features: the mean of N trilinear probes at uv + (i / (N + 1) - 1/2)
    times the major-axis derivative, i = 1..N, each level at lod
    bias + log2(Pmax W_k / N).  FP64 apart from the decision of N and the probe
    coordinates: a probe samples the latents at a texture coordinate, which is
    an FP32 value (Sec. 3.1 samples T_k at the FP32 uv a shader passes), formed
    as RN32(u + o d) with the offset o = RN32(RN32(i / (N + 1)) - 1/2) -- one
    rounding of the exact product and sum, as an FMA takes it."""
    n, along_x, pmax = aniso_count(duv, max_aniso)
    d = np.asarray(duv, dtype=np.float64)
    au = np.where(along_x, d[:, 0], d[:, 2])
    av = np.where(along_x, d[:, 1], d[:, 3])
    u, v = uv[:, 0].astype(np.float64), uv[:, 1].astype(np.float64)
    base = np.asarray(bias, dtype=np.float64)
    with np.errstate(divide="ignore"):
        base = base + np.log2(pmax.astype(np.float64) / n)
    feats = np.zeros((len(u), 12))
    for i in range(1, int(n.max()) + 1):
        sel = n >= i
        off = ((np.float32(i) / (n[sel] + 1).astype(np.float32)) - np.float32(0.5)).astype(np.float64)
        # off * a is exact in FP64 (two 24-bit significands); the sum is rounded
        # once more in FP64 before the FP32 rounding, which changes the FP32 result
        # only when the FP64 sum lands exactly on an FP32 midpoint
        uu = (u[sel] + off * au[sel]).astype(np.float32).astype(np.float64)
        vv = (v[sel] + off * av[sel]).astype(np.float32).astype(np.float64)
        for k, (lv, mips) in enumerate(zip(material.levels, levels_mips_rgb)):
            lam = base[sel] + np.log2(float(lv.width))
            feats[sel, 3 * k:3 * k + 3] += trilinear(mips, uu, vv, lam, lv.shift, material.address)
    return feats / n[:, None]


def decode_pixels_aniso(material, levels_mips_rgb: list, uv: np.ndarray, duv: np.ndarray, bias: np.ndarray,
                        max_aniso: int, precision: str = "fp16") -> np.ndarray:
    """decode_pixels with the anisotropic latent filter instead of trilinear."""
    x = aniso_features(material, levels_mips_rgb, uv, duv, bias, max_aniso)
    mlp = material.mlp
    if precision == "fp16":
        return emulate.forward_fp16(x, mlp.weights, mlp.biases)
    from . import mlp as mlp_mod
    return mlp_mod.forward(x, mlp.weights, mlp.biases)
