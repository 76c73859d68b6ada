"""Lighting pass on the decoded G-buffer, FP64 -- TEST INFRASTRUCTURE ONLY.

Paper Sec. 4 ("Rendering architecture"): after the G-buffer pass decodes the
neural texture set, a lighting pass shades every pixel with a diffuse lobe and a
GGX lobe under a directional light plus prefiltered image-based lighting, after
the physically based model the paper cites (Lagarde and de Rousiers, "Moving
Frostbite to physically based rendering").

Readings fixed here (the paper gives no formulas):
  * channels: albedo RGB = y[0:3], tangent-space normal XY = y[3:5] encoded as
    (n + 1) / 2, roughness = y[5], metalness = y[6], ambient occlusion = y[7]
    (y[8], displacement, does not enter shading); each clamped to its range,
    perceptual roughness to [0.045, 1] and alpha = roughness^2;
  * n = normalize(2 x - 1, 2 y - 1, sqrt(max(0, 1 - nx^2 - ny^2))) with the
    components clamped to [-1, 1];
  * diffuse: Lambert, (1 - metalness) albedo / pi;
  * specular: GGX distribution D = a^2 / (pi ((n.h)^2 (a^2 - 1) + 1)^2), the
    height-correlated Smith visibility
    V = 0.5 / ((n.l) sqrt((n.v)^2 (1 - a^2) + a^2) + (n.v) sqrt((n.l)^2 (1 - a^2) + a^2)),
    Schlick Fresnel F = F0 + (1 - F0) (1 - l.h)^5 with F0 = 0.04 (1 - m) + albedo m;
  * image-based lighting has no environment maps here: a two-colour hemisphere
    E(d) = ground + (sky - ground) (1 + d_z) / 2 stands in for the prefiltered
    radiance, sampled at n for the diffuse part and at the reflection vector for
    the specular part, whose Fresnel is Schlick's at n.v with the
    roughness-aware limit max(1 - roughness, F0); both scaled by the occlusion;
  * n.v is floored at 1e-4; a zero denominator in V gives V = 0.
Output: linear HDR RGB radiance.
"""
from __future__ import annotations

import numpy as np


def _normalize(v):
    n = np.linalg.norm(v, axis=-1, keepdims=True)
    return v / np.where(n > 0, n, 1.0)


def ggx_d(ndoth, alpha):
    a2 = alpha * alpha
    d = ndoth * ndoth * (a2 - 1.0) + 1.0
    return a2 / (np.pi * d * d)


def smith_visibility(ndotl, ndotv, alpha):
    a2 = alpha * alpha
    den = ndotl * np.sqrt(ndotv * ndotv * (1.0 - a2) + a2) + ndotv * np.sqrt(ndotl * ndotl * (1.0 - a2) + a2)
    return np.where(den > 0, 0.5 / np.where(den > 0, den, 1.0), 0.0)


def surface(y: np.ndarray):
    """G-buffer channels [n, 9] -> (albedo, normal, roughness, metalness, ao)."""
    y = np.asarray(y, dtype=np.float64)
    albedo = np.clip(y[:, 0:3], 0.0, 1.0)
    nx = np.clip(2.0 * y[:, 3] - 1.0, -1.0, 1.0)
    ny = np.clip(2.0 * y[:, 4] - 1.0, -1.0, 1.0)
    nz = np.sqrt(np.maximum(0.0, 1.0 - nx * nx - ny * ny))
    n = np.stack([nx, ny, nz], axis=-1)
    n = np.where(np.linalg.norm(n, axis=-1, keepdims=True) > 0, _normalize(n), np.array([0.0, 0.0, 1.0]))
    rough = np.clip(y[:, 5], 0.045, 1.0)
    metal = np.clip(y[:, 6], 0.0, 1.0)
    ao = np.clip(y[:, 7], 0.0, 1.0)
    return albedo, n, rough, metal, ao


def brdf(albedo, n, rough, metal, l, v):
    """Diffuse + specular BRDF value [n, 3] for unit light / view directions [3]."""
    alpha = rough * rough
    h = _normalize(np.asarray(l, dtype=np.float64) + np.asarray(v, dtype=np.float64))[None, :]
    ndotl = np.maximum(n @ np.asarray(l, dtype=np.float64), 0.0)
    ndotv = np.maximum(n @ np.asarray(v, dtype=np.float64), 1e-4)
    ndoth = np.maximum(np.sum(n * h, axis=-1), 0.0)
    ldoth = max(float(np.dot(l, h[0])), 0.0)
    f0 = 0.04 * (1.0 - metal)[:, None] + albedo * metal[:, None]
    fr = f0 + (1.0 - f0) * (1.0 - ldoth) ** 5
    spec = (ggx_d(ndoth, alpha) * smith_visibility(ndotl, ndotv, alpha))[:, None] * fr
    diff = (1.0 - metal)[:, None] * albedo / np.pi
    return diff + spec, ndotl


def hemisphere(d, sky, ground):
    t = (1.0 + d[..., 2:3]) * 0.5
    return np.asarray(ground, dtype=np.float64) + (np.asarray(sky, dtype=np.float64) -
                                                   np.asarray(ground, dtype=np.float64)) * t


def shade(y: np.ndarray, light_dir, light_rgb, view_dir, sky, ground) -> np.ndarray:
    """Shaded linear RGB [n, 3] of G-buffer pixels y [n, 9] (tangent space)."""
    l = _normalize(np.asarray(light_dir, dtype=np.float64)[None, :])[0]
    v = _normalize(np.asarray(view_dir, dtype=np.float64)[None, :])[0]
    albedo, n, rough, metal, ao = surface(y)
    f, ndotl = brdf(albedo, n, rough, metal, l, v)
    direct = f * np.asarray(light_rgb, dtype=np.float64) * ndotl[:, None]
    ndotv = np.maximum(n @ v, 1e-4)
    r = 2.0 * ndotv[:, None] * n - v
    f0 = 0.04 * (1.0 - metal)[:, None] + albedo * metal[:, None]
    fmax = np.maximum((1.0 - rough)[:, None], f0)
    fr = f0 + (fmax - f0) * ((1.0 - ndotv) ** 5)[:, None]
    amb = ao[:, None] * ((1.0 - metal)[:, None] * albedo * hemisphere(n, sky, ground) + fr * hemisphere(r, sky, ground))
    return direct + amb
