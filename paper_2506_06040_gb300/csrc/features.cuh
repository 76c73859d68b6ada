// Feature stage shared by the tiled decode kernels: the 12 latent features
// (4 levels x RGB, Sec. 3.1) of a tile of consecutive output texels, computed
// by a group of NT threads (thread t owns texel tile_start + t).
//
// Row-footprint mode (texel-centre grid, tile inside one output row, every
// latent level no wider than the output): the output row samples each level
// at one vertical position, so the group decodes only the latent columns the
// tile touches -- two BC1 texels per column (rows y0, y1), blended vertically
// once -- into shared memory; each texel then blends its two neighbouring
// columns horizontally.  This is the bilinear filter of Sec. 3.1 evaluated in
// separable order, with every BC1 block decoded once per tile instead of once
// per tap.  Direct mode (uv lists, ragged grids) samples each texel on its own.
#pragma once

#include "common.cuh"
#include "sm100.cuh"

namespace nbtc {

constexpr int kColCap = 136;  // columns per level per group (>= 128 + 2)

__device__ __forceinline__ int wrap_or_clamp(int x, int n, bool wrap) {
  if (wrap) {
    x %= n;
    return x < 0 ? x + n : x;
  }
  return min(max(x, 0), n - 1);
}

// Texel coordinate along one axis, unwrapped: t = u * n - 0.5 + shift.
__device__ __forceinline__ float texel_coord(float u, int n, float shift) {
  return fmaf(u, (float)n, shift - 0.5f);
}

// Level k (0..3, runtime value) without indexing the kernel-parameter array
// at run time (which would copy it to local memory).
__device__ __forceinline__ LevelView pick_level(const DecodeArgs& a, int k) {
  LevelView L = a.lv[0];
  if (k == 1) L = a.lv[1];
  if (k == 2) L = a.lv[2];
  if (k == 3) L = a.lv[3];
  return L;
}

template <typename T>
__device__ __forceinline__ T pick4(const T (&v)[4], int k) {
  return k == 0 ? v[0] : k == 1 ? v[1] : k == 2 ? v[2] : v[3];
}

// Features of texel (tile_start + tid) into feat[12] (values in [0, 1]).
// `colbuf` holds 4 * kColCap float4 of group scratch.  All NT threads of the
// group must call it (it contains one group barrier).
template <int NT>
__device__ __forceinline__ void footprint_features(const DecodeArgs& a, int64_t tile_start, int tid,
                                                   float4* colbuf, int bar_id, float (&feat)[12]) {
  const int j = (int)(tile_start / a.grid_w);
  const int i0 = (int)(tile_start - (int64_t)j * a.grid_w);
  const float u0 = ((float)i0 + 0.5f) * a.inv_gw;
  const float u1 = ((float)(i0 + NT - 1) + 0.5f) * a.inv_gw;
  const bool wrap = a.wrap;
  int base[4], pre[4], span[4];
  int total = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int b0 = (int)floorf(texel_coord(u0, a.lv[k].w, a.lv[k].shift));
    const int b1 = (int)floorf(texel_coord(u1, a.lv[k].w, a.lv[k].shift));
    base[k] = b0;
    pre[k] = total;
    span[k] = min(b1 - b0 + 2, kColCap);
    total += span[k];
  }
  // decode + vertical blend of every touched column of every level
  if (tid < total) {
    const float v = ((float)j + 0.5f) * a.inv_gh;
    for (int job = tid; job < total; job += NT) {
      const int k = (job >= pre[1]) + (job >= pre[2]) + (job >= pre[3]);
      const LevelView L = pick_level(a, k);
      const int rel = job - pick4(pre, k);
      const float ty = texel_coord(v, L.h, L.shift);
      const float fty = floorf(ty);
      const float fy = ty - fty;
      const int y0 = wrap_or_clamp((int)fty, L.h, wrap);
      const int y1 = wrap_or_clamp((int)fty + 1, L.h, wrap);
      const int x = wrap_or_clamp(pick4(base, k) + rel, L.w, wrap);
      const uint32_t t0 = fetch_texel(L, x, y0);
      const uint32_t t1 = fetch_texel(L, x, y1);
      float4 c;
      c.x = fmaf(fy, (float)((t1 >> 0) & 255u) - (float)((t0 >> 0) & 255u), (float)((t0 >> 0) & 255u));
      c.y = fmaf(fy, (float)((t1 >> 8) & 255u) - (float)((t0 >> 8) & 255u), (float)((t0 >> 8) & 255u));
      c.z = fmaf(fy, (float)((t1 >> 16) & 255u) - (float)((t0 >> 16) & 255u), (float)((t0 >> 16) & 255u));
      c.w = 0.f;
      colbuf[k * kColCap + rel] = c;
    }
  }
  sm100::named_bar_sync(bar_id, NT);
  const float u = ((float)(i0 + tid) + 0.5f) * a.inv_gw;
  const float s = 1.0f / 255.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float tx = texel_coord(u, a.lv[k].w, a.lv[k].shift);
    const float ftx = floorf(tx);
    const float fx = tx - ftx;
    // floor is monotone in u, so rel lies in [0, span - 2]; the clamp only guards the buffer
    const int rel = min(max((int)ftx - base[k], 0), span[k] - 2);
    const float4 A = colbuf[k * kColCap + rel];
    const float4 B = colbuf[k * kColCap + rel + 1];
    feat[3 * k + 0] = s * fmaf(fx, B.x - A.x, A.x);
    feat[3 * k + 1] = s * fmaf(fx, B.y - A.y, A.y);
    feat[3 * k + 2] = s * fmaf(fx, B.z - A.z, A.z);
  }
}

// Features of one texel sampled on its own (any uv).
__device__ __forceinline__ void direct_features(const DecodeArgs& a, int64_t t, float (&feat)[12]) {
  const float2 uv = texel_uv(a, t);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float3 c = sample_bilinear(a.lv[k], uv.x, uv.y, a.wrap);
    feat[3 * k + 0] = c.x;
    feat[3 * k + 1] = c.y;
    feat[3 * k + 2] = c.z;
  }
}

}  // namespace nbtc
