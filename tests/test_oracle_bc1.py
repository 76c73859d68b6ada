"""Pins of the oracle's BC1 decode (Sec. 3.1 "Latent BC1 compression" and the
BC1 format definition the paper cites)."""
import os

import numpy as np
import pytest

from oracle import bc1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bc1_blocks.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        name, hexbytes, texels = [f.strip() for f in line.split("|")]
        raw = bytes(int(h, 16) for h in hexbytes.split())
        block = np.frombuffer(raw, dtype="<u8")
        rgb = np.array([[int(c) for c in t.split(",")] for t in texels.split()]).reshape(4, 4, 3)
        rows.append((name, block, rgb))
    return rows


@pytest.mark.parametrize("name,block,rgb", _golden(), ids=[g[0] for g in _golden()])
def test_hand_built_blocks(name, block, rgb):
    got = bc1.decode_level(block, 4, 4)
    np.testing.assert_array_equal(got, rgb)


def test_expansion_exhaustive_properties():
    c = np.arange(1 << 16)
    e = bc1.expand565(c)
    r5, g6, b5 = (c >> 11) & 31, (c >> 5) & 63, c & 31
    # within one 8-bit step of the real-valued scaling c * 255 / (2^b - 1)
    for ch, f, bits in ((0, r5, 5), (1, g6, 6), (2, b5, 5)):
        exact = f * 255.0 / ((1 << bits) - 1)
        assert np.all(np.abs(e[..., ch] - exact) < 1.0)
    # end points map to 0 and 255, and the map is strictly increasing
    assert bc1.expand565(0xFFFF).tolist() == [255, 255, 255]
    assert bc1.expand565(0).tolist() == [0, 0, 0]
    assert np.all(np.diff(bc1.expand565(np.arange(32) << 11)[:, 0]) > 0)
    assert np.all(np.diff(bc1.expand565(np.arange(64) << 5)[:, 1]) > 0)


def test_palette_matches_paper_interpolation_4colour():
    """T = (1 - a) e0 + a e1 with a in {0, 1, 1/3, 2/3} for indices 0..3, up to the
    8-bit rounding (<= 1/2 step)."""
    rng = np.random.default_rng(0)
    c = rng.integers(0, 1 << 16, size=(200000, 2))
    c0, c1 = c.max(axis=1), c.min(axis=1)
    keep = c0 > c1
    c0, c1 = c0[keep], c1[keep]
    pal = bc1.palette(c0, c1).astype(np.float64)
    e0, e1 = bc1.expand565(c0).astype(np.float64), bc1.expand565(c1).astype(np.float64)
    for i, a in enumerate((0.0, 1.0, 1.0 / 3.0, 2.0 / 3.0)):
        assert np.all(np.abs(pal[:, i] - ((1 - a) * e0 + a * e1)) <= 0.5 + 1e-12)


def test_palette_3colour_mode():
    rng = np.random.default_rng(1)
    c = rng.integers(0, 1 << 16, size=(100000, 2))
    c0, c1 = c.min(axis=1), c.max(axis=1)  # c0 <= c1, includes equal pairs
    pal = bc1.palette(c0, c1).astype(np.float64)
    e0, e1 = bc1.expand565(c0), bc1.expand565(c1)
    assert np.all(np.abs(pal[:, 2] - (e0 + e1) / 2.0) <= 0.5)
    assert np.all(pal[:, 3] == 0)
    assert np.all(pal[:, 0] == e0) and np.all(pal[:, 1] == e1)


def test_texel_and_block_addressing():
    """Block (bx, by) at by * (W/4) + bx, texel (tx, ty) at index bits 2 * (4 ty + tx)."""
    W, H = 16, 12
    blocks = []
    for by in range(H // 4):
        for bx in range(W // 4):
            c0 = (((bx + 1) << 11) | ((by + 1) << 5)) + 1   # distinct endpoint per block
            c1 = 0
            idx = 0
            for ty in range(4):
                for tx in range(4):
                    idx |= ((tx + ty) % 2) << (2 * (4 * ty + tx))  # index 0 or 1
            blocks.append(np.uint64(c0) | (np.uint64(c1) << np.uint64(16)) | (np.uint64(idx) << np.uint64(32)))
    img = bc1.decode_level(np.array(blocks, dtype=np.uint64), W, H)
    for y in range(H):
        for x in range(W):
            bx, by, tx, ty = x // 4, y // 4, x % 4, y % 4
            c0 = (((bx + 1) << 11) | ((by + 1) << 5)) + 1
            want = bc1.expand565(c0) if (tx + ty) % 2 == 0 else np.zeros(3, dtype=np.int64)
            np.testing.assert_array_equal(img[y, x], want)


def test_footprint_matches_paper_28mb():
    """Abstract: 28 MB of VRAM per 4K texture set.  Variant A (W, W, W/2, W/2) of
    BC1 latents (8 bytes per 4x4 block) with full mip chains."""
    total = 0
    for side in (4096, 4096, 2048, 2048):
        total += bc1.footprint_bytes(side, side, mips=True)
    assert round(total / 1e6) == 28
