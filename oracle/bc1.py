"""BC1 block decode (integer, bit-exact reference).

Paper Sec. 3.1, "Latent BC1 compression": each latent texel is an interpolation
T = (1 - alpha) e0 + alpha e1 of two endpoints shared by a 4x4 block, with
alpha on 2 bits and the endpoints on a [5,6,5] bit pattern; the format itself is
the BC1 (S3TC DXT1) block of the Khronos Data Format Specification that the
paper cites.

Block layout (8 bytes, little endian): bits 0-15 colour c0, bits 16-31 colour
c1, each R5 (bits 15-11) G6 (10-5) B5 (4-0); bits 32-63 hold sixteen 2-bit
indices, texel (tx, ty) of the block at bits 2 * (4 * ty + tx).

Integer rounding (the paper and the format text give real-valued formulas
only; this reading is fixed here and used by both sides):
  * 5/6-bit channels expand to 8 bits by bit replication.
  * c0 > c1 (raw 16-bit compare): p2 = (2 c0 + c1 + 1) // 3, p3 = (c0 + 2 c1 + 1) // 3.
  * c0 <= c1: p2 = (c0 + c1 + 1) // 2, p3 = black (0, 0, 0).
  * Palette order: index 0 -> c0, 1 -> c1, 2 -> p2, 3 -> p3.
"""
from __future__ import annotations

import numpy as np


def split_block(blocks: np.ndarray):
    """uint64 blocks -> (c0, c1, index word) as int64 arrays."""
    b = np.asarray(blocks, dtype=np.uint64)
    c0 = (b & np.uint64(0xFFFF)).astype(np.int64)
    c1 = ((b >> np.uint64(16)) & np.uint64(0xFFFF)).astype(np.int64)
    idx = (b >> np.uint64(32)).astype(np.int64)
    return c0, c1, idx


def expand565(c: np.ndarray) -> np.ndarray:
    """RGB565 word -> [..., 3] RGB8 by bit replication."""
    c = np.asarray(c, dtype=np.int64)
    r5, g6, b5 = (c >> 11) & 31, (c >> 5) & 63, c & 31
    r8 = (r5 << 3) | (r5 >> 2)
    g8 = (g6 << 2) | (g6 >> 4)
    b8 = (b5 << 3) | (b5 >> 2)
    return np.stack([r8, g8, b8], axis=-1)


def palette(c0: np.ndarray, c1: np.ndarray) -> np.ndarray:
    """[..., 4, 3] RGB8 palette of blocks with endpoint words c0, c1."""
    e0, e1 = expand565(c0), expand565(c1)
    four = (np.asarray(c0) > np.asarray(c1))[..., None]
    p2 = np.where(four, (2 * e0 + e1 + 1) // 3, (e0 + e1 + 1) // 2)
    p3 = np.where(four, (e0 + 2 * e1 + 1) // 3, 0)
    return np.stack([e0, e1, p2, p3], axis=-2)


def texel_index(idx_word: np.ndarray, tx: np.ndarray, ty: np.ndarray) -> np.ndarray:
    """2-bit palette index of texel (tx, ty) inside its block."""
    return (np.asarray(idx_word) >> (2 * (4 * np.asarray(ty) + np.asarray(tx)))) & 3


def texel_rgb8(blocks: np.ndarray, width: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """RGB8 of texels (x, y) of a BC1 image of `width` texels (block row-major)."""
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    blk = np.asarray(blocks, dtype=np.uint64)[(y >> 2) * (width // 4) + (x >> 2)]
    c0, c1, iw = split_block(blk)
    pal = palette(c0, c1)
    i = texel_index(iw, x & 3, y & 3)
    return np.take_along_axis(pal, i[..., None, None].repeat(3, axis=-1), axis=-2)[..., 0, :]


def decode_level(blocks: np.ndarray, width: int, height: int) -> np.ndarray:
    """Whole BC1 image -> uint8 [height, width, 3]."""
    assert width % 4 == 0 and height % 4 == 0
    assert len(blocks) == (width // 4) * (height // 4)
    y, x = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    return texel_rgb8(blocks, width, x, y).astype(np.uint8)


def footprint_bytes(width: int, height: int, mips: bool = True) -> int:
    """Bytes of a BC1 texture (8 bytes per 4x4 block), with its mip chain down
    to one block when `mips`."""
    total = 0
    w, h = width, height
    while True:
        total += ((w + 3) // 4) * ((h + 3) // 4) * 8
        if not mips or (w <= 4 and h <= 4):
            return total
        w, h = max(1, w // 2), max(1, h // 2)
