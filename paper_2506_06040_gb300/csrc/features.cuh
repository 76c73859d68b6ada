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

template <typename T>
__device__ __forceinline__ T pick4(const T (&v)[4], int k) {
  return k == 0 ? v[0] : k == 1 ? v[1] : k == 2 ? v[2] : v[3];
}

// ---- row-footprint feature stage in three steps, so a tile's block loads can
// be issued long before they are decoded:
//   plan      per-level column range of the tile (every thread, identical)
//   prefetch  thread `tid` issues the two block loads of column job `tid`
//   decode    the prefetched (and any further) columns -> colbuf
//   blend     after a group barrier, each texel blends its two columns

struct TilePlan {
  int j, i0;
  int base[4], span[4], pre[4];
  int total;
};

template <int NT>
__device__ __forceinline__ TilePlan plan_tile(const DecodeArgs& a, int64_t tile_start) {
  TilePlan P;
  if (tile_start <= 0xFFFFFFFFll) {
    P.j = (int)((uint32_t)tile_start / (uint32_t)a.grid_w);
    P.i0 = (int)((uint32_t)tile_start - (uint32_t)P.j * (uint32_t)a.grid_w);
  } else {
    P.j = (int)(tile_start / a.grid_w);
    P.i0 = (int)(tile_start - (int64_t)P.j * a.grid_w);
  }
  const float u0 = ((float)P.i0 + 0.5f) * a.inv_gw;
  const float u1 = ((float)(P.i0 + NT - 1) + 0.5f) * a.inv_gw;
  int total = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int b0 = (int)floorf(texel_coord(u0, a.lv[k].w, a.lv[k].shift));
    const int b1 = (int)floorf(texel_coord(u1, a.lv[k].w, a.lv[k].shift));
    P.base[k] = b0;
    P.pre[k] = total;
    P.span[k] = min(b1 - b0 + 2, kColCap);
    total += P.span[k];
  }
  P.total = total;
  return P;
}

// Texel coordinates of column job `job` (< P.total): level, column slot, the
// two texels (x, y0) and (x, y1) and the vertical weight.
struct ColumnJob {
  int k, rel, x, y0, y1;
  float fy;
};

__device__ __forceinline__ ColumnJob column_job(const DecodeArgs& a, const TilePlan& P, int job) {
  ColumnJob J;
  J.k = (job >= P.pre[1]) + (job >= P.pre[2]) + (job >= P.pre[3]);
  J.rel = job - pick4(P.pre, J.k);
  const LevelView& L = a.lv[J.k];
  const float v = ((float)P.j + 0.5f) * a.inv_gh;
  const float ty = texel_coord(v, L.h, L.shift);
  const float fty = floorf(ty);
  J.fy = ty - fty;
  J.y0 = wrap_or_clamp((int)fty, L.h, a.wrap);
  J.y1 = wrap_or_clamp((int)fty + 1, L.h, a.wrap);
  J.x = wrap_or_clamp(pick4(P.base, J.k) + J.rel, L.w, a.wrap);
  return J;
}

struct BlockPair {
  uint64_t b0, b1;
};

__device__ __forceinline__ BlockPair load_column(const DecodeArgs& a, const ColumnJob& J) {
  const LevelView& L = a.lv[J.k];
  BlockPair B;
  B.b0 = __ldg(L.blocks + (size_t)(J.y0 >> 2) * L.wb + (J.x >> 2));
  B.b1 = __ldg(L.blocks + (size_t)(J.y1 >> 2) * L.wb + (J.x >> 2));
  return B;
}

__device__ __forceinline__ void store_column(float4* colbuf, const ColumnJob& J, const BlockPair& B) {
  const uint32_t t0 = bc1_texel(B.b0, J.x & 3, J.y0 & 3);
  const uint32_t t1 = bc1_texel(B.b1, J.x & 3, J.y1 & 3);
  const float fy = J.fy;
  float4 c;
  c.x = fmaf(fy, (float)((t1 >> 0) & 255u) - (float)((t0 >> 0) & 255u), (float)((t0 >> 0) & 255u));
  c.y = fmaf(fy, (float)((t1 >> 8) & 255u) - (float)((t0 >> 8) & 255u), (float)((t0 >> 8) & 255u));
  c.z = fmaf(fy, (float)((t1 >> 16) & 255u) - (float)((t0 >> 16) & 255u), (float)((t0 >> 16) & 255u));
  c.w = 0.f;
  colbuf[J.k * kColCap + J.rel] = c;
}

// Issues the loads of column job `tid` (if any); returns them unconsumed.
__device__ __forceinline__ BlockPair prefetch_columns(const DecodeArgs& a, const TilePlan& P, int tid) {
  BlockPair B{0, 0};
  if (tid < P.total) B = load_column(a, column_job(a, P, tid));
  return B;
}

// Decodes column job `tid` from its prefetched blocks, and any further jobs
// (tid + NT, ...) with fresh loads, into colbuf.
template <int NT>
__device__ __forceinline__ void decode_columns(const DecodeArgs& a, const TilePlan& P, int tid, const BlockPair& pf,
                                               float4* colbuf) {
  if (tid < P.total) store_column(colbuf, column_job(a, P, tid), pf);
  for (int job = tid + NT; job < P.total; job += NT) {
    const ColumnJob J = column_job(a, P, job);
    store_column(colbuf, J, load_column(a, J));
  }
}

// Horizontal blend of texel tid from the decoded columns (after a barrier).
template <int NT>
__device__ __forceinline__ void blend_columns(const DecodeArgs& a, const TilePlan& P, int tid, const float4* colbuf,
                                              float (&feat)[12]) {
  const float u = ((float)(P.i0 + tid) + 0.5f) * a.inv_gw;
  const float s = 1.0f / 255.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float tx = texel_coord(u, a.lv[k].w, a.lv[k].shift);
    const float ftx = floorf(tx);
    const float fx = tx - ftx;
    // floor is monotone in u, so rel lies in [0, span - 2]; the clamp only guards the buffer
    const int rel = min(max((int)ftx - P.base[k], 0), P.span[k] - 2);
    const float4 A = colbuf[k * kColCap + rel];
    const float4 B = colbuf[k * kColCap + rel + 1];
    feat[3 * k + 0] = s * fmaf(fx, B.x - A.x, A.x);
    feat[3 * k + 1] = s * fmaf(fx, B.y - A.y, A.y);
    feat[3 * k + 2] = s * fmaf(fx, B.z - A.z, A.z);
  }
}

// All three steps back to back (one group barrier): features of texel
// tile_start + tid of a tile lying in one output row.
template <int NT>
__device__ __forceinline__ void footprint_features(const DecodeArgs& a, int64_t tile_start, int tid,
                                                   float4* colbuf, int bar_id, float (&feat)[12]) {
  const TilePlan P = plan_tile<NT>(a, tile_start);
  const BlockPair pf = prefetch_columns(a, P, tid);
  decode_columns<NT>(a, P, tid, pf, colbuf);
  sm100::named_bar_sync(bar_id, NT);
  blend_columns<NT>(a, P, tid, colbuf, feat);
}

// Per-material description used by the batched and frame decodes: the level
// views of mip 0 (in `d`) plus every level's mip chain for trilinear sampling.
struct MatDev {
  DecodeArgs d;          // mip-0 views, wrap flag, output grid and buffer of the full decode
  const void* packed;    // FP16 packed MLP
  int nout;
  int tiles_per_row;     // full decode: grid_w / 128
  int64_t tiles;         // full decode: tiles of the grid
  int mips[4];
  float log2w[4];        // log2 of each level's mip-0 width
  int mip_off[4][16];    // block offset of mip m of level k
};

__device__ __forceinline__ LevelView mip_view(const MatDev& M, int k, int m) {
  LevelView v = M.d.lv[k];
  v.blocks = v.blocks + M.mip_off[k][m];
  v.w = max(4, v.w >> m);
  v.h = max(4, v.h >> m);
  v.wb = v.w / 4;
  return v;
}

// Features of one pixel of the frame: per level, lod_k = lod + log2(W_k)
// clamped to the mip range, trilinear (bilinear in mips floor(lod_k) and the
// next, blended by its fraction), the material's address mode.
__device__ __forceinline__ void trilinear_features(const MatDev& M, float u, float v, float lod, float (&feat)[12]) {
  const bool wrap = M.d.wrap;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float lam = fminf(fmaxf(lod + M.log2w[k], 0.f), (float)(M.mips[k] - 1));
    const int m0 = (int)floorf(lam);
    const int m1 = min(m0 + 1, M.mips[k] - 1);
    const float t = lam - (float)m0;
    const float3 c0 = sample_bilinear(mip_view(M, k, m0), u, v, wrap);
    const float3 c1 = sample_bilinear(mip_view(M, k, m1), u, v, wrap);
    feat[3 * k + 0] = fmaf(t, c1.x - c0.x, c0.x);
    feat[3 * k + 1] = fmaf(t, c1.y - c0.y, c0.y);
    feat[3 * k + 2] = fmaf(t, c1.z - c0.z, c0.z);
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
