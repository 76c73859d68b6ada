"""Pins of the oracle's frame classification / binning (Sec. 4, Algorithm 1)
and per-pixel mip-mapped decode."""
import numpy as np

import synth
from oracle import decode, frame


def test_classification_cases():
    tw, th = 16, 8
    ids = np.zeros((8, 64), dtype=np.int32)
    ids[:, 0:16] = 3                       # tile 0: one material, all valid -> uniform
    ids[:, 16:32] = 1; ids[0, 20] = 2      # tile 1: two materials -> mixed
    ids[:, 32:48] = -1; ids[:4, 32:48] = 5; ids[4, 32] = 5   # tile 2: 65 valid of 128 -> uniform
    ids[:, 48:64] = -1; ids[:4, 48:64] = 6  # tile 3: 64 valid of 128 (not more than half) -> mixed
    kind, mat = frame.classify(ids, tw, th)
    assert kind.tolist() == [frame.UNIFORM, frame.MIXED, frame.UNIFORM, frame.MIXED]
    assert mat.tolist() == [3, -1, 5, -1]
    kind, _ = frame.classify(np.full((8, 16), -1, dtype=np.int32), tw, th)
    assert kind.tolist() == [frame.EMPTY]


def test_binning_invariants():
    rng = synth.Rng(5, 0)
    ids, _, _ = synth.voronoi_ids(rng, 256, 128, 12)
    ids[rng.uniform(256 * 128).reshape(128, 256) < 0.05] = -1
    kind, mat = frame.classify(ids, 16, 8)
    counts, offsets = frame.mixed_counts(ids, kind, 16, 8, 12)
    assert np.all(offsets % 128 == 0)
    assert np.all(np.diff(np.concatenate([offsets, [offsets[-1] + counts[-1]]])) >= 0)
    # every valid pixel is either in a uniform tile of its own material or counted once
    covered = np.zeros(12, dtype=np.int64)
    for t in range(len(kind)):
        px = frame.tile_pixels(t, 256, 16, 8)
        v = ids.reshape(-1)[px]
        if kind[t] == frame.UNIFORM:
            assert np.all((v == mat[t]) | (v < 0))
            covered += np.bincount(v[v >= 0], minlength=12)
    assert np.array_equal(covered + counts, np.bincount(ids[ids >= 0], minlength=12))


def test_pixel_decode_at_mip0_equals_grid_decode():
    bw = synth.batch_workload(num_materials=2, frame_w=64, frame_h=32, smin=256, smax=256)
    mat = bw.materials[0]
    mips = [frame.level_mips_rgb(lv) for lv in mat.levels]
    n = 500
    idx = np.arange(n) * 97 % (256 * 256)
    uv = np.stack([(idx % 256 + 0.5) / 256, (idx // 256 + 0.5) / 256], -1)
    got = frame.decode_pixels(mat, mips, uv, np.full(n, -20.0), precision="fp64")
    want = decode.decode_grid(mat, 256, 256, idx)
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_direct_pixel_decode_equals_full_mip_decode():
    """Tap-on-demand BC1 sampling gives the same frame decode as sampling fully decoded mips."""
    bw = synth.batch_workload(num_materials=3, frame_w=64, frame_h=32, smin=256, smax=512)
    rng = np.random.default_rng(9)
    for mat in bw.materials:
        mips = [frame.level_mips_rgb(lv) for lv in mat.levels]
        n = 400
        uv = rng.uniform(-2, 6, size=(n, 2))
        lod = rng.uniform(-12, 2, size=n)
        for prec in ("fp64", "fp16"):
            a = frame.decode_pixels(mat, mips, uv, lod, precision=prec)
            b = frame.decode_pixels_direct(mat, uv, lod, precision=prec)
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
