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


def _small_mip_material(seed=21, side=256):
    rng_lat, rng_mlp = synth.Rng(seed, 1), synth.Rng(seed, 2)
    return synth.Material(synth.latent_pyramid(rng_lat, side, mips=True), synth.he_mlp(rng_mlp, [12, 64, 64, 9]),
                          "wrap")


def test_aniso_count_matches_the_extension_formula():
    rng = np.random.default_rng(3)
    duv = rng.normal(0, 1e-3, (20000, 4)).astype(np.float32)
    n, along_x, pmax = frame.aniso_count(duv, 16)
    d = duv.astype(np.float64)
    px, py = np.hypot(d[:, 0], d[:, 1]), np.hypot(d[:, 2], d[:, 3])
    ratio = np.maximum(px, py) / np.minimum(px, py)
    clear = np.abs(ratio - np.round(ratio)) > 1e-4          # away from integer ratios
    want = np.minimum(np.ceil(ratio), 16).astype(np.int64)
    assert np.array_equal(n[clear], want[clear])
    assert np.array_equal(along_x, px >= py) or np.mean(along_x == (px >= py)) > 0.9999
    assert n.min() >= 1 and n.max() == 16
    # no footprint (magnification): one probe
    n0, _, _ = frame.aniso_count(np.zeros((3, 4), np.float32), 16)
    assert n0.tolist() == [1, 1, 1]


def test_aniso_with_isotropic_footprint_is_trilinear():
    mat = _small_mip_material()
    mips = [frame.level_mips_rgb(lv) for lv in mat.levels]
    rng = np.random.default_rng(4)
    uv = rng.uniform(-2, 3, (500, 2)).astype(np.float32)
    f = (2.0 ** rng.uniform(-9, -2, 500)).astype(np.float32)
    bias = rng.uniform(0, 3, 500).astype(np.float32)
    duv = np.stack([f, 0 * f, 0 * f, f], axis=-1)
    lod = bias.astype(np.float64) + np.log2(f.astype(np.float64))
    got = frame.decode_pixels_aniso(mat, mips, uv, duv, bias, 16, precision="fp64")
    want = frame.decode_pixels(mat, mips, uv, lod, precision="fp64")
    assert np.max(np.abs(got - want)) < 1e-12


def test_aniso_symmetries_and_constant_texture():
    mat = _small_mip_material(seed=22)
    mips = [frame.level_mips_rgb(lv) for lv in mat.levels]
    rng = np.random.default_rng(5)
    uv = rng.uniform(0, 4, (400, 2)).astype(np.float32)
    duv = rng.normal(0, 4e-3, (400, 4)).astype(np.float32)
    bias = rng.uniform(0, 2, 400).astype(np.float32)
    x = frame.aniso_features(mat, mips, uv, duv, bias, 16)
    # the probes are symmetric about uv: negating the derivatives changes nothing
    # but the FP32 roundings of the probe coordinates (a shift of the offsets,
    # e.g. i / N - 1/2, breaks the symmetry by ~1e-3)
    assert np.max(np.abs(frame.aniso_features(mat, mips, uv, -duv, bias, 16) - x)) < 2.0 ** -14
    # which screen axis carries the major derivative does not matter
    sw = duv[:, [2, 3, 0, 1]]
    assert np.max(np.abs(frame.aniso_features(mat, mips, uv, sw, bias, 16) - x)) < 1e-12
    # a latent pyramid of constant colour filters to that colour for any footprint
    const = []
    for lv in mat.levels:
        blocks = [np.full(len(b), np.uint64(0x000052AA52AA), dtype=np.uint64) for b in lv.blocks]
        const.append(synth.Level(lv.width, lv.height, lv.shift, blocks))
    cm = synth.Material(const, mat.mlp, "wrap")
    cx = frame.aniso_features(cm, [frame.level_mips_rgb(lv) for lv in cm.levels], uv, duv, bias, 16)
    rgb = np.array([0x52AA >> 11, (0x52AA >> 5) & 63, 0x52AA & 31])
    want = np.array([(rgb[0] << 3 | rgb[0] >> 2), (rgb[1] << 2 | rgb[1] >> 4), (rgb[2] << 3 | rgb[2] >> 2)]) / 255
    assert np.max(np.abs(cx - np.tile(want, 4))) < 1e-12
