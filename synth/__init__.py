"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no BC1 decode, no filtering, no MLP).  Every array it
returns is plain host memory (numpy); the same bytes are handed to both sides.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream s under seed k is mix(base(k, s) + (i + 1) * gamma).
Uniforms take the top 53 bits; normals use the Box-Muller transform.

The five workloads follow the method's shapes: 4 BC1 RGB latent levels at
1/4, 1/8, 1/16, 1/32 of the output side (the paper's "variant B" ratios, Sec. 3.1),
half-texel shifts on the 2nd and 4th latent (Sec. 3.1), 9 output channels and
ReLU MLPs with He-initialised weights.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _base(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        a = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)]))[0]
        s = np.array([np.uint64(stream & 0xFFFFFFFFFFFFFFFF)]) * GAMMA
        return _mix(np.array([a]) ^ s)[0]


class Rng:
    """Counter-based SplitMix64 stream.  `Rng(seed, stream)` is reproducible and
    independent of the order in which other streams are drawn."""

    def __init__(self, seed: int, stream: int = 0):
        self.base = _base(seed, stream)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
            out = _mix(self.base + idx * GAMMA)
        self.counter += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, std: float = 1.0) -> np.ndarray:
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)  # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])[:n]
        return std * z


# --------------------------------------------------------------------------- data

@dataclass
class Level:
    """One BC1 latent texture.  `blocks[m]` holds mip m as uint64 blocks in
    row-major block order (block (bx, by) at by * (w_m / 4) + bx)."""
    width: int
    height: int
    shift: float
    blocks: list  # list of np.ndarray(uint64), one per mip

    @property
    def num_mips(self) -> int:
        return len(self.blocks)

    def packed(self) -> np.ndarray:
        """All mips back to back (mip 0 first), as one uint64 array."""
        return np.concatenate(self.blocks)


@dataclass
class Mlp:
    """ReLU MLP; layer l weight is [dims[l+1], dims[l]] (out x in), FP32."""
    dims: list
    weights: list
    biases: list

    def packed_weights(self) -> np.ndarray:
        return np.concatenate([w.reshape(-1) for w in self.weights]).astype(np.float32)

    def packed_biases(self) -> np.ndarray:
        return np.concatenate([b.reshape(-1) for b in self.biases]).astype(np.float32)


@dataclass
class Material:
    levels: list
    mlp: Mlp
    address: str = "clamp"  # "clamp" or "wrap"


SHIFTS = (0.0, 0.5, 0.0, 0.5)  # half-texel shift of the 2nd and 4th latent (Sec. 3.1)
CHANNELS = ("albedo_r", "albedo_g", "albedo_b", "normal_x", "normal_y",
            "roughness", "metalness", "ao", "displacement")


def random_blocks(rng: Rng, n: int) -> np.ndarray:
    """n BC1 blocks of 64 uniform random bits (both c0 > c1 and c0 <= c1 modes occur)."""
    return rng.u64(n)


def bc1_level(rng: Rng, width: int, height: int, shift: float, mips: int = 1) -> Level:
    assert width % 4 == 0 and height % 4 == 0
    blocks = []
    w, h = width, height
    for _ in range(mips):
        blocks.append(random_blocks(rng, (w // 4) * (h // 4)))
        w, h = max(4, w // 2), max(4, h // 2)
    return Level(width, height, shift, blocks)


def he_mlp(rng: Rng, dims) -> Mlp:
    ws, bs = [], []
    for i in range(len(dims) - 1):
        fan_in, fan_out = dims[i], dims[i + 1]
        ws.append(rng.normal(fan_out * fan_in, math.sqrt(2.0 / fan_in)).reshape(fan_out, fan_in).astype(np.float32))
        bs.append((0.01 * rng.normal(fan_out)).astype(np.float32))
    return Mlp(list(dims), ws, bs)


def full_mips(side: int) -> int:
    """Mips of a square BC1 texture: halve while the side stays a multiple of 4
    (every mip then tiles into whole 4x4 blocks; a power-of-two side ends at 4x4)."""
    m = 1
    while (side >> m) >= 4 and (side >> m) % 4 == 0 and (side >> (m - 1)) % 2 == 0:
        m += 1
    return m


def latent_pyramid(rng: Rng, side: int, mips: bool = False) -> list:
    """4 BC1 levels at side/4, /8, /16, /32 with shifts (0, 1/2, 0, 1/2)."""
    levels = []
    for k in range(4):
        w = side >> (k + 2)
        levels.append(bc1_level(rng, w, w, SHIFTS[k], full_mips(w) if mips else 1))
    return levels


def has_both_modes(blocks: np.ndarray) -> bool:
    c0 = blocks & np.uint64(0xFFFF)
    c1 = (blocks >> np.uint64(16)) & np.uint64(0xFFFF)
    return bool(np.any(c0 > c1)) and bool(np.any(c0 <= c1))


# --------------------------------------------------------------------------- workloads

@dataclass
class DecodeWorkload:
    name: str
    out_w: int
    out_h: int
    material: Material
    seed: int


def decode_workload(k: int) -> DecodeWorkload:
    """Decode workloads: k = 0 (256^2, 12-32-32-9), 1 (4096^2, 12-64-64-9),
    2 (4096^2, 12-64-64-64-9, run in FP16 / FP8 on tensor cores)."""
    seed = 1000 + k
    side = {0: 256, 1: 4096, 2: 4096}[k]
    dims = {0: [12, 32, 32, 9], 1: [12, 64, 64, 9], 2: [12, 64, 64, 64, 9]}[k]
    rng_lat = Rng(seed, 1)
    rng_mlp = Rng(seed, 2)
    levels = latent_pyramid(rng_lat, side)
    for lv in levels:
        assert has_both_modes(lv.blocks[0])
    mlp = he_mlp(rng_mlp, dims)
    name = {0: "decode-256sq-mlp12-32-32-9-fp32", 1: "decode-4096sq-mlp12-64-64-9-fp32",
            2: "decode-4096sq-mlp12-64-64-64-9-fp16out"}[k]
    return DecodeWorkload(name, side, side, Material(levels, mlp, "clamp"), seed)


def small_decode_workload(side: int, dims, seed: int, shifts=SHIFTS, address="clamp",
                          level_sides=None) -> DecodeWorkload:
    """Reduced workload of the same recipe (test sizes)."""
    rng_lat, rng_mlp = Rng(seed, 1), Rng(seed, 2)
    if level_sides is None:
        level_sides = [side >> (k + 2) for k in range(4)]
    levels = [bc1_level(rng_lat, s, s, shifts[i % len(shifts)]) for i, s in enumerate(level_sides)]
    return DecodeWorkload(f"decode-{side}sq-test", side, side,
                          Material(levels, he_mlp(rng_mlp, dims), address), seed)


def random_uv(seed: int, n: int, stream: int = 7, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n uv pairs uniform in [lo, hi)^2, FP32, shape [n, 2]."""
    r = Rng(seed, stream)
    return r.uniform(2 * n, lo, hi).astype(np.float32).reshape(n, 2)


# --------------------------------------------------------------------------- training

@dataclass
class TrainWorkload:
    name: str
    latent_sides: list
    shifts: tuple
    latents: list          # list of [h, w, 3] FP32 arrays (continuous latents)
    mlp: Mlp
    target: np.ndarray     # [th, tw, 9] FP32
    batch: int
    seed: int
    lr_mlp: float = 1e-3
    lr_latent: float = 1e-2

    def uv(self, step: int) -> np.ndarray:
        return random_uv(self.seed, self.batch, stream=1000 + step)


def sinusoid_target(rng: Rng, side: int, channels: int = 9, terms: int = 16,
                    noise: float = 0.02) -> np.ndarray:
    """Each channel: 0.5 + sum_j (0.5/terms) sin(2 pi f_j (cos t_j x + sin t_j y) + p_j) + N(0, noise),
    x = (i + 0.5) / side, f_j ~ U[1, 64] cycles per texture, t_j, p_j ~ U[0, 2 pi).
    Evaluated per term as an outer product of x and y factors (sin(a+b) expansion)."""
    coord = (np.arange(side, dtype=np.float64) + 0.5) / side
    out = np.empty((side, side, channels), dtype=np.float32)
    for c in range(channels):
        f = rng.uniform(terms, 1.0, 64.0)
        th = rng.uniform(terms, 0.0, 2 * np.pi)
        ph = rng.uniform(terms, 0.0, 2 * np.pi)
        acc = np.full((side, side), 0.5)
        for j in range(terms):
            ax = 2 * np.pi * f[j] * np.cos(th[j]) * coord
            by = 2 * np.pi * f[j] * np.sin(th[j]) * coord + ph[j]
            acc += (0.5 / terms) * (np.outer(np.cos(by), np.sin(ax)) + np.outer(np.sin(by), np.cos(ax)))
        acc += rng.normal(side * side, noise).reshape(side, side)
        out[:, :, c] = acc.astype(np.float32)
    return out


def train_workload(full: bool = True, seed: int = 1003) -> TrainWorkload:
    """Full: latents 1024^2..128^2 (the 4096^2 pyramid before BC1 quantisation),
    target 2048^2 x 9, batch 2^20, MLP 12-64-64-9.  Reduced (finite differences):
    target 64^2, latents 16^2..2^2, batch 512."""
    if full:
        sides, tside, batch = [1024, 512, 256, 128], 2048, 1 << 20
    else:
        sides, tside, batch = [16, 8, 4, 2], 64, 512
    rng_lat, rng_mlp, rng_t = Rng(seed, 1), Rng(seed, 2), Rng(seed, 3)
    lat = [rng_lat.normal(s * s * 3, 0.1).reshape(s, s, 3).astype(np.float32) for s in sides]
    mlp = he_mlp(rng_mlp, [12, 64, 64, 9])
    target = sinusoid_target(rng_t, tside)
    name = "train-latents1024-mlp12-64-64-9-batch2^20" if full else "train-64sq-fd"
    return TrainWorkload(name, sides, SHIFTS, lat, mlp, target, batch, seed)


# --------------------------------------------------------------------------- batching

@dataclass
class BatchWorkload:
    name: str
    materials: list   # list of Material (wrap addressing, BC1 mip chains)
    sizes: list       # output side per material
    frame_w: int
    frame_h: int
    mat_id: np.ndarray    # [frame_h, frame_w] int32, material per pixel (-1 = none)
    uv: np.ndarray        # [frame_h, frame_w, 2] FP32
    lod_bias: np.ndarray  # [frame_h, frame_w] FP32
    seed: int
    lod: np.ndarray = None  # [frame_h, frame_w] FP32: log2(uv footprint of a pixel) + bias
    duv: np.ndarray = None  # [frame_h, frame_w, 4] FP32 anisotropic footprint: du/dx, dv/dx, du/dy, dv/dy


def voronoi_ids(rng: Rng, w: int, h: int, m: int):
    """Material id per pixel: nearest of m uniform seed points (Euclidean, ties to the lower id)."""
    sx = rng.uniform(m, 0.0, w)
    sy = rng.uniform(m, 0.0, h)
    ids = np.zeros((h, w), dtype=np.int32)
    best = np.full((h, w), np.inf)
    px = np.arange(w, dtype=np.float64) + 0.5
    for row0 in range(0, h, 256):
        py = np.arange(row0, min(h, row0 + 256), dtype=np.float64) + 0.5
        d_best = best[row0:row0 + len(py)]
        i_best = ids[row0:row0 + len(py)]
        for k in range(m):
            d = (py[:, None] - sy[k]) ** 2 + (px[None, :] - sx[k]) ** 2
            better = d < d_best
            d_best[better] = d[better]
            i_best[better] = k
    return ids, sx, sy


def batch_workload(num_materials: int = 64, frame_w: int = 3840, frame_h: int = 2160,
                   smin: int = 256, smax: int = 4096, seed: int = 1004) -> BatchWorkload:
    rng_s, rng_f = Rng(seed, 1), Rng(seed, 2)
    lo, hi = math.log(smin), math.log(smax)
    sizes = []
    for x in rng_s.uniform(num_materials, lo, hi):
        s = int(round(math.exp(x) / 128.0)) * 128
        sizes.append(min(smax, max(smin, s)))
    mats = []
    for i, s in enumerate(sizes):
        r_lat, r_mlp = Rng(seed, 100 + 2 * i), Rng(seed, 101 + 2 * i)
        mats.append(Material(latent_pyramid(r_lat, s, mips=True), he_mlp(r_mlp, [12, 64, 64, 9]), "wrap"))
    ids, _, _ = voronoi_ids(rng_f, frame_w, frame_h, num_materials)
    scale = rng_f.uniform(num_materials, 1.0, 8.0)
    py, px = np.meshgrid(np.arange(frame_h) + 0.5, np.arange(frame_w) + 0.5, indexing="ij")
    s_pix = scale[ids]
    uv = np.stack([s_pix * px / frame_h, s_pix * py / frame_h], axis=-1).astype(np.float32)
    bias = rng_f.uniform(frame_w * frame_h, 0.0, 3.0).reshape(frame_h, frame_w).astype(np.float32)
    # a pixel spans s_m / frame_h in uv (tiled uv of scale s_m over the frame height)
    lod = (bias.astype(np.float64) + np.log2(s_pix / frame_h)).astype(np.float32)
    duv = aniso_footprints(Rng(seed, 3), ids, s_pix / frame_h, num_materials)
    return BatchWorkload(f"batch-{num_materials}mat-{frame_w}x{frame_h}", mats, sizes, frame_w, frame_h,
                         ids, uv, bias, seed, lod, duv)


def aniso_footprints(rng: Rng, ids: np.ndarray, f: np.ndarray, num_materials: int) -> np.ndarray:
    """Screen-space uv derivatives [h, w, 4] = (du/dx, dv/dx, du/dy, dv/dy) of an
    anisotropic footprint: the isotropic footprint f (uv per pixel) stretched by
    r = 1 + 15 y / h (1 at the top row, 16 at the bottom, like a plane seen at a
    growing grazing angle) along a direction phi drawn per material."""
    h, w = ids.shape
    phi = rng.uniform(num_materials, 0.0, np.pi)[ids]
    r = 1.0 + 15.0 * (np.arange(h, dtype=np.float64) + 0.5)[:, None] / h
    c, s = np.cos(phi), np.sin(phi)
    # J = R(phi) diag(r, 1) f: screen x maps along the stretched direction
    dudx, dvdx = f * r * c, f * r * s
    dudy, dvdy = -f * s, f * c
    return np.stack([dudx, dvdx, dudy, dvdy], axis=-1).astype(np.float32)
