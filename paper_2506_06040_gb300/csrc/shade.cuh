// Lighting pass fused into the frame decode's output epilogue (Sec. 4,
// "Rendering architecture": a diffuse lobe and a GGX lobe under a directional
// light and prefiltered image-based lighting, after the Frostbite model the
// paper cites).  The G-buffer channels of a pixel -- albedo RGB, tangent-space
// normal XY encoded as (n + 1) / 2, roughness, metalness, ambient occlusion --
// are shaded in FP32:
//   diffuse  Lambert, (1 - metalness) albedo / pi
//   specular GGX D = a^2 / (pi ((n.h)^2 (a^2 - 1) + 1)^2), a = roughness^2
//            (roughness clamped to [0.045, 1]), height-correlated Smith
//            visibility, Schlick Fresnel on l.h with F0 = lerp(0.04, albedo, m)
//   ambient  a two-colour hemisphere (ground -> sky along z) in place of
//            prefiltered environment maps: at n for the diffuse part, at the
//            reflection vector for the specular part (Schlick on n.v with the
//            roughness-aware limit max(1 - roughness, F0)), times the occlusion.
#pragma once

#include "../../include/nbtc.h"

namespace nbtc {

struct LightDev {
  float l[3];       // unit light direction (toward the light), tangent space
  float rgb[3];     // light radiance
  float v[3];       // unit view direction (toward the viewer)
  float h[3];       // normalize(l + v)
  float ldoth;      // max(l . h, 0)
  float sky[3], ground[3];
};

__device__ __forceinline__ float3 hemisphere_radiance(const LightDev& L, float dz) {
  const float t = 0.5f * (1.f + dz);
  return make_float3(fmaf(t, L.sky[0] - L.ground[0], L.ground[0]), fmaf(t, L.sky[1] - L.ground[1], L.ground[1]),
                     fmaf(t, L.sky[2] - L.ground[2], L.ground[2]));
}

// Lit linear RGB of one pixel from its G-buffer channels y[0..7].
__device__ __forceinline__ float3 shade_pixel(const float* y, const LightDev& L) {
  const float ar = fminf(fmaxf(y[0], 0.f), 1.f), ag = fminf(fmaxf(y[1], 0.f), 1.f), ab = fminf(fmaxf(y[2], 0.f), 1.f);
  float nx = fminf(fmaxf(2.f * y[3] - 1.f, -1.f), 1.f), ny = fminf(fmaxf(2.f * y[4] - 1.f, -1.f), 1.f);
  float nz = sqrtf(fmaxf(0.f, 1.f - nx * nx - ny * ny));
  const float len = sqrtf(nx * nx + ny * ny + nz * nz);
  if (len > 0.f) {
    nx /= len;
    ny /= len;
    nz /= len;
  } else {
    nz = 1.f;
  }
  const float rough = fminf(fmaxf(y[5], 0.045f), 1.f);
  const float metal = fminf(fmaxf(y[6], 0.f), 1.f);
  const float ao = fminf(fmaxf(y[7], 0.f), 1.f);
  const float alpha = rough * rough, a2 = alpha * alpha;
  const float ndotl = fmaxf(nx * L.l[0] + ny * L.l[1] + nz * L.l[2], 0.f);
  const float ndotv = fmaxf(nx * L.v[0] + ny * L.v[1] + nz * L.v[2], 1e-4f);
  const float ndoth = fmaxf(nx * L.h[0] + ny * L.h[1] + nz * L.h[2], 0.f);
  const float d = ndoth * ndoth * (a2 - 1.f) + 1.f;
  const float D = a2 / (3.14159265358979f * d * d);
  const float den = ndotl * sqrtf(ndotv * ndotv * (1.f - a2) + a2) + ndotv * sqrtf(ndotl * ndotl * (1.f - a2) + a2);
  const float vis = den > 0.f ? 0.5f / den : 0.f;
  const float dm = 1.f - metal;
  const float f0[3] = {0.04f * dm + ar * metal, 0.04f * dm + ag * metal, 0.04f * dm + ab * metal};
  const float alb[3] = {ar, ag, ab};
  const float s = 1.f - L.ldoth, s5 = s * s * s * s * s;
  const float c = 1.f - ndotv, c5 = c * c * c * c * c;
  // reflection vector r = 2 (n.v) n - v: only its z enters the hemisphere
  const float rz = 2.f * ndotv * nz - L.v[2];
  const float3 en = hemisphere_radiance(L, nz), er = hemisphere_radiance(L, rz);
  const float enc[3] = {en.x, en.y, en.z}, erc[3] = {er.x, er.y, er.z};
  float out[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float fr = f0[k] + (1.f - f0[k]) * s5;
    const float f = dm * alb[k] * (1.f / 3.14159265358979f) + D * vis * fr;
    const float fmx = fmaxf(1.f - rough, f0[k]);
    const float fa = f0[k] + (fmx - f0[k]) * c5;
    out[k] = f * L.rgb[k] * ndotl + ao * (dm * alb[k] * enc[k] + fa * erc[k]);
  }
  return make_float3(out[0], out[1], out[2]);
}

}  // namespace nbtc
