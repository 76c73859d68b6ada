"""Pins of the oracle's latent sampling (Sec. 3.1 T_k(uv), half-texel shifts;
Sec. 3.2 texture-unit filtering)."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import sample


def _scipy_bilinear(tex, u, v, shift, mode):
    h, w, c = tex.shape
    x = u * w - 0.5 + shift
    y = v * h - 0.5 + shift
    return np.stack([ndimage.map_coordinates(tex[:, :, k], [y, x], order=1, mode=mode) for k in range(c)], -1)


@pytest.mark.parametrize("shift", [0.0, 0.5, 0.25])
@pytest.mark.parametrize("address,mode", [("clamp", "nearest"), ("wrap", "grid-wrap")])
def test_bilinear_matches_scipy(shift, address, mode):
    rng = np.random.default_rng(3)
    tex = rng.random((8, 16, 3))
    # coordinates on a 2^-12 grid: exact in FP32, so dropping whole periods (wrap)
    # and forming the texel coordinate lose nothing and the FP64 interpolation
    # must match scipy's
    u = rng.integers(-1229, 5325, 4000) / 4096.0
    v = rng.integers(-1229, 5325, 4000) / 4096.0
    got = sample.bilinear(tex, u, v, shift, address)
    want = _scipy_bilinear(tex, u, v, shift, mode)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_texel_centres_exact():
    rng = np.random.default_rng(4)
    tex = rng.random((8, 8, 3))
    j, i = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    got = sample.bilinear(tex, (i.ravel() + 0.5) / 8, (j.ravel() + 0.5) / 8, 0.0, "clamp")
    np.testing.assert_array_equal(got, tex.reshape(-1, 3))


def test_half_texel_shift_gives_mean_of_four():
    rng = np.random.default_rng(5)
    tex = rng.random((8, 8, 3))
    i, j = 2, 5   # texel centre of (2, 5): shifted by +1/2 lands on the corner of 4 texels
    got = sample.bilinear(tex, np.array([(i + 0.5) / 8]), np.array([(j + 0.5) / 8]), 0.5, "clamp")[0]
    want = (tex[j, i] + tex[j, i + 1] + tex[j + 1, i] + tex[j + 1, i + 1]) / 4
    np.testing.assert_allclose(got, want, atol=1e-15)


def test_constant_and_ramp():
    tex = np.full((4, 4, 3), 0.37)
    u = np.linspace(-0.2, 1.2, 101)
    for addr in ("clamp", "wrap"):
        np.testing.assert_allclose(sample.bilinear(tex, u, u[::-1], 0.5, addr), 0.37, atol=1e-15)
    # a linear ramp in x is reproduced exactly between the first and last texel centres
    w = 16
    ramp = np.tile((np.arange(w) * 0.25 + 1.0)[None, :, None], (4, 1, 3))
    u = np.linspace(0.5 / w, (w - 0.5) / w, 57)
    got = sample.bilinear(ramp, u, np.full_like(u, 0.5), 0.0, "clamp")[:, 0]
    np.testing.assert_allclose(got, (u * w - 0.5) * 0.25 + 1.0, atol=1e-12)


def test_trilinear_integer_and_fractional_lod():
    rng = np.random.default_rng(6)
    mips = [rng.random((16, 16, 3)), rng.random((8, 8, 3)), rng.random((4, 4, 3))]
    u, v = rng.random(500), rng.random(500)
    for m in range(3):
        np.testing.assert_allclose(sample.trilinear(mips, u, v, np.full(500, float(m)), 0.5),
                                   sample.bilinear(mips[m], u, v, 0.5, "wrap"), atol=1e-14)
    lod = np.full(500, 0.25)
    want = 0.75 * sample.bilinear(mips[0], u, v, 0.5, "wrap") + 0.25 * sample.bilinear(mips[1], u, v, 0.5, "wrap")
    np.testing.assert_allclose(sample.trilinear(mips, u, v, lod, 0.5), want, atol=1e-14)
    # lod is clamped to the mip range
    np.testing.assert_allclose(sample.trilinear(mips, u, v, np.full(500, -3.0), 0.5),
                               sample.bilinear(mips[0], u, v, 0.5, "wrap"), atol=1e-14)
    np.testing.assert_allclose(sample.trilinear(mips, u, v, np.full(500, 7.5), 0.5),
                               sample.bilinear(mips[2], u, v, 0.5, "wrap"), atol=1e-14)


def test_feature_order():
    a = np.zeros((4, 4, 3)); a[..., :] = [1, 2, 3]
    b = np.zeros((2, 2, 3)); b[..., :] = [4, 5, 6]
    f = sample.features([a, b], [0.0, 0.5], np.array([0.3]), np.array([0.6]))
    np.testing.assert_allclose(f, [[1, 2, 3, 4, 5, 6]])


def test_grid_uv_row_major():
    u, v = sample.grid_uv(4, 2)
    np.testing.assert_allclose(u, [0.125, 0.375, 0.625, 0.875] * 2)
    np.testing.assert_allclose(v, [0.25] * 4 + [0.75] * 4)


def test_grid_coord_is_the_correctly_rounded_quotient():
    """grid_coord(i, n) is (2i + 1) / (2n) rounded to the nearest FP32 (ties to
    even), checked against exact rational arithmetic; exact for powers of two."""
    from fractions import Fraction
    rng = np.random.default_rng(11)
    for n in (200, 1000, 3840, 1731, 4096, 7):
        idx = rng.integers(0, n, 300)
        got = sample.grid_coord(idx, n)
        assert got.dtype == np.float32
        for i, g in zip(idx, got):
            exact = Fraction(2 * int(i) + 1, 2 * n)
            g_f = Fraction(float(g))
            lo = Fraction(float(np.nextafter(g, np.float32(-1))))
            hi = Fraction(float(np.nextafter(g, np.float32(2))))
            # no FP32 neighbour is closer to the exact value
            assert abs(g_f - exact) <= abs(lo - exact) and abs(g_f - exact) <= abs(hi - exact)
            if n & (n - 1) == 0:
                assert g_f == exact


def test_texel_coord_rounds_once_to_fp32():
    """texel_coord = u n - 1/2 + s rounded once: exact for power-of-two n and an
    FP32 u; for other n it is the FP32 value nearest the exact one."""
    from fractions import Fraction
    rng = np.random.default_rng(12)
    u = rng.uniform(0, 1, 500).astype(np.float32)
    for n, s in ((1024, 0.5), (384, 0.0), (1000, 0.5)):
        x = sample.texel_coord(u.astype(np.float64), n, s)
        for ui, xi in zip(u, x):
            exact = Fraction(float(ui)) * n - Fraction(1, 2) + Fraction(s)
            if n & (n - 1) == 0:
                assert Fraction(xi) == exact
            else:
                xf = np.float32(xi)
                assert abs(Fraction(xi) - exact) <= abs(Fraction(float(np.nextafter(xf, np.float32(-1e9)))) - exact)
                assert abs(Fraction(xi) - exact) <= abs(Fraction(float(np.nextafter(xf, np.float32(1e9)))) - exact)


def test_wrap_is_periodic():
    """Wrap addressing: shifting u, v by whole periods changes nothing (coordinates
    on a 2^-12 grid, periods up to 8 as in the tiled frame)."""
    rng = np.random.default_rng(13)
    tex = rng.random((16, 32, 3))
    u = rng.integers(0, 4096, 1000) / 4096.0
    v = rng.integers(0, 4096, 1000) / 4096.0
    base = sample.bilinear(tex, u, v, 0.5, "wrap")
    for k in (-3, 1, 7):
        np.testing.assert_array_equal(sample.bilinear(tex, u + k, v - k, 0.5, "wrap"), base)
