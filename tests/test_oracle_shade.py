"""Pins of the lighting-pass oracle (Sec. 4, "Rendering architecture") against
closed forms and invariants of the shading model: the GGX distribution's
normalisation (numerical integration), its value at alpha = 1, the visibility
term's closed form, BRDF reciprocity, the normal decoding, normal incidence and
a constant environment."""
import numpy as np

from oracle import shade


def test_ggx_distribution_is_normalised():
    th = np.linspace(0.0, np.pi / 2, 200001)
    for alpha in (0.05, 0.2, 0.5, 1.0):
        f = shade.ggx_d(np.cos(th), alpha) * np.cos(th) * np.sin(th)
        integral = 2.0 * np.pi * np.trapezoid(f, th)
        assert abs(integral - 1.0) < 2e-4, (alpha, integral)


def test_closed_forms_at_alpha_one():
    c = np.linspace(0.0, 1.0, 11)
    assert np.allclose(shade.ggx_d(c, 1.0), 1.0 / np.pi)
    l, v = np.linspace(0.1, 1.0, 10), np.linspace(1.0, 0.1, 10)
    assert np.allclose(shade.smith_visibility(l, v, 1.0), 0.5 / (l + v))
    assert np.all(shade.smith_visibility(np.zeros(3), np.zeros(3), 0.3) == 0.0)


def _gbuffer(n, seed):
    r = np.random.default_rng(seed)
    y = r.uniform(-0.2, 1.2, (n, 9))
    return y


def test_brdf_is_reciprocal():
    y = _gbuffer(500, 1)
    albedo, n, rough, metal, _ = shade.surface(y)
    r = np.random.default_rng(2)
    for _ in range(5):
        l = r.normal(size=3); l[2] = abs(l[2]); l /= np.linalg.norm(l)
        v = r.normal(size=3); v[2] = abs(v[2]); v /= np.linalg.norm(v)
        f1, _ = shade.brdf(albedo, n, rough, metal, l, v)
        f2, _ = shade.brdf(albedo, n, rough, metal, v, l)
        # n.v is floored at 1e-4 on one side only: compare where both dot products are clear of it
        ok = (n @ l > 1e-3) & (n @ v > 1e-3)
        assert np.allclose(f1[ok], f2[ok], rtol=1e-12, atol=0)


def test_normal_decoding():
    y = np.zeros((3, 9))
    y[0, 3:5] = 0.5                 # flat
    y[1, 3:5] = (1.0, 0.5)          # along +x
    y[2, 3:5] = (0.5, 0.0)          # along -y
    _, n, _, _, _ = shade.surface(y)
    assert np.allclose(n, [[0, 0, 1], [1, 0, 0], [0, -1, 0]])


def test_normal_incidence_specular():
    """l = v = n: D = 1 / (pi a^2), V = 1/4, F = F0; specular = F0 / (4 pi a^2)."""
    y = np.zeros((4, 9))
    y[:, 0:3] = [[0.2, 0.5, 0.9]] * 4
    y[:, 3:5] = 0.5
    y[:, 5] = [0.3, 0.5, 0.8, 1.0]
    y[:, 6] = [0.0, 1.0, 0.5, 0.25]
    albedo, n, rough, metal, _ = shade.surface(y)
    f, ndotl = shade.brdf(albedo, n, rough, metal, np.array([0, 0, 1.0]), np.array([0, 0, 1.0]))
    a = rough ** 2
    f0 = 0.04 * (1 - metal)[:, None] + albedo * metal[:, None]
    want = (1 - metal)[:, None] * albedo / np.pi + f0 / (4 * np.pi * a * a)[:, None]
    assert np.allclose(f, want, rtol=1e-12)
    assert np.allclose(ndotl, 1.0)


def test_constant_environment_and_no_light():
    y = _gbuffer(300, 3)
    c = np.array([0.3, 0.6, 0.9])
    out = shade.shade(y, [0, 0, 1.0], [0.0, 0.0, 0.0], [0.2, 0.1, 1.0], c, c)
    albedo, n, rough, metal, ao = shade.surface(y)
    v = np.array([0.2, 0.1, 1.0]) / np.linalg.norm([0.2, 0.1, 1.0])
    ndotv = np.maximum(n @ v, 1e-4)
    f0 = 0.04 * (1 - metal)[:, None] + albedo * metal[:, None]
    fr = f0 + (np.maximum((1 - rough)[:, None], f0) - f0) * ((1 - ndotv) ** 5)[:, None]
    want = ao[:, None] * ((1 - metal)[:, None] * albedo * c + fr * c)
    assert np.allclose(out, want, rtol=1e-12)
