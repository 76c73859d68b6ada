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

#include <climits>

#include "common.cuh"
#include "fastdiv.h"
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
  const float u0 = grid_coord((float)P.i0, a.cw);
  const float u1 = grid_coord((float)(P.i0 + NT - 1), a.cw);
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
  const float v = grid_coord((float)(P.j + a.row0), a.ch);
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
  B.b0 = __ldg(L.blocks + block_index(L, J.x >> 2, J.y0 >> 2));
  B.b1 = __ldg(L.blocks + block_index(L, J.x >> 2, J.y1 >> 2));
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
  const float u = grid_coord((float)(P.i0 + tid), a.cw);
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

// ---- row-footprint feature stage with a per-thread column cache, for a group
// of NT threads that decodes vertically consecutive tiles of one column strip
// (the same first column i0, output rows j, j+1, ...).  Across such tiles the
// column plan, each thread's column job and each texel's horizontal taps stay
// fixed, and a latent column's two vertical taps (rows floor(ty), floor(ty)+1)
// change only when ty crosses a texel boundary: every 4th output row for a
// latent at 1/4 of the output side, every 32nd at 1/32.  So each thread keeps
// its job's two decoded texels (as floats scaled to [0, 1]) and reloads and
// decodes the BC1 blocks only when floor(ty) changes; per tile it only redoes
// the vertical blend of its column and the horizontal blend of its texel.
struct StripCache {
  int i0;          // first output column of the cached strip (-1: none)
  int total;       // column jobs of the strip
  int job;         // own job: level | colbuf slot << 2 (-1: none)
  int jx;          // own job: latent column (wrapped or clamped)
  int key;         // floor(ty) of the decoded pair (INT_MIN + 1: none)
  uint32_t rel4;   // own texel: left tap's colbuf slot per level, 8 bits each
  float fx[4];     // own texel: horizontal weight per level
  uint32_t t1;     // own job: RGB8 of texel (jx, y1) -- the next pair's (jx, y0) when the key steps by one
  float c0[3];     // own job: texel (jx, y0), RGB / 255
  float dc[3];     // own job: texel (jx, y1) minus texel (jx, y0), RGB / 255
};

__device__ __forceinline__ void strip_reset(StripCache& C) { C.i0 = -1; }

// Features of texel i0 + tid of output row j; (j, i0) is a tile of NT texels
// in one row (i0 + NT <= grid_w).
template <int NT>
__device__ __forceinline__ void strip_features(const DecodeArgs& a, int j, int i0, int tid, uint32_t colbuf,
                                               int bar_id, StripCache& C, float (&feat)[12]) {
  const float s = 1.0f / 255.0f;
  if (i0 != C.i0) {  // new strip: column plan, own job, own texel's taps
    C.i0 = i0;
    C.key = INT_MIN + 1;  // no pair decoded (and key == C.key + 1 cannot hold)
    const float u0 = grid_coord((float)i0, a.cw);
    const float u1 = grid_coord((float)(i0 + NT - 1), a.cw);
    const float u = grid_coord((float)(i0 + tid), a.cw);
    int total = 0, job = -1, jx = 0;
    uint32_t rel4 = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const LevelView& L = a.lv[k];
      const int b0 = (int)floorf(texel_coord(u0, L.w, L.shift));
      const int b1 = (int)floorf(texel_coord(u1, L.w, L.shift));
      const int span = min(b1 - b0 + 2, kColCap);
      if (tid >= total && tid < total + span) {
        job = k | (tid - total) << 2;
        jx = wrap_or_clamp(b0 + tid - total, L.w, a.wrap);
      }
      total += span;
      const float tx = texel_coord(u, L.w, L.shift);
      const float ftx = floorf(tx);
      C.fx[k] = tx - ftx;
      // floor is monotone in u, so the slot lies in [0, span - 2]; the clamp only guards the buffer
      rel4 |= (uint32_t)min(max((int)ftx - b0, 0), span - 2) << (8 * k);
    }
    C.total = total;
    C.job = job;
    C.jx = jx;
    C.rel4 = rel4;
  }
  if (C.job >= 0) {
    const int k = C.job & 3;
    const LevelView& L = a.lv[k];
    const float ty = texel_coord(grid_coord((float)(j + a.row0), a.ch), L.h, L.shift);
    const float fty = floorf(ty);
    const float fy = ty - fty;
    const int key = (int)fty;
    if (key != C.key) {
      // moving down one latent row, the new pair's upper texel is the old pair's
      // lower one: decode only the new lower texel
      uint32_t t0;
      if (key == C.key + 1) {
        t0 = C.t1;
      } else {
        const int y0 = wrap_or_clamp(key, L.h, a.wrap);
        t0 = bc1_texel(__ldg(L.blocks + block_index(L, C.jx >> 2, y0 >> 2)), C.jx & 3, y0 & 3);
      }
      const int y1 = wrap_or_clamp(key + 1, L.h, a.wrap);
      const uint32_t t1 = bc1_texel(__ldg(L.blocks + block_index(L, C.jx >> 2, y1 >> 2)), C.jx & 3, y1 & 3);
      C.key = key;
      C.t1 = t1;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v0 = (float)((t0 >> (8 * c)) & 255u), v1 = (float)((t1 >> (8 * c)) & 255u);
        C.c0[c] = s * v0;
        C.dc[c] = s * (v1 - v0);
      }
    }
    sm100::sts128f(colbuf + 16u * (uint32_t)(k * kColCap + (C.job >> 2)), fmaf(fy, C.dc[0], C.c0[0]),
                   fmaf(fy, C.dc[1], C.c0[1]), fmaf(fy, C.dc[2], C.c0[2]), 0.f);
    // the next row's pair changes here too: start pulling its blocks into L1
    const float tyn = texel_coord(grid_coord((float)(j + a.row0 + 1), a.ch), L.h, L.shift);
    const int keyn = (int)floorf(tyn);
    if (keyn != key && j + 1 < a.grid_h) {
      const int y1 = wrap_or_clamp(keyn + 1, L.h, a.wrap);
      sm100::prefetch_l1(L.blocks + block_index(L, C.jx >> 2, y1 >> 2));
    }
  }
  if (C.total > NT) {
    // a strip wider than NT columns over all levels: the jobs past the first
    // per thread are decoded afresh for every tile (only unusual level-to-output
    // ratios get here; the 1/4..1/32 pyramid needs 68 columns per 128 texels)
    const TilePlan P = plan_tile<NT>(a, (int64_t)j * a.grid_w + i0);
    for (int job = tid + NT; job < P.total; job += NT) {
      const ColumnJob J = column_job(a, P, job);
      const BlockPair B = load_column(a, J);
      const uint32_t t0 = bc1_texel(B.b0, J.x & 3, J.y0 & 3), t1 = bc1_texel(B.b1, J.x & 3, J.y1 & 3);
      float c[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float v0 = (float)((t0 >> (8 * ch)) & 255u), v1 = (float)((t1 >> (8 * ch)) & 255u);
        c[ch] = fmaf(J.fy, s * (v1 - v0), s * v0);
      }
      sm100::sts128f(colbuf + 16u * (uint32_t)(J.k * kColCap + J.rel), c[0], c[1], c[2], 0.f);
    }
  }
  sm100::named_bar_sync(bar_id, NT);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t at = colbuf + 16u * (uint32_t)(k * kColCap + ((C.rel4 >> (8 * k)) & 255));
    const float4 A = sm100::lds128f(at);
    const float4 B = sm100::lds128f(at + 16);
    feat[3 * k + 0] = fmaf(C.fx[k], B.x - A.x, A.x);
    feat[3 * k + 1] = fmaf(C.fx[k], B.y - A.y, A.y);
    feat[3 * k + 2] = fmaf(C.fx[k], B.z - A.z, A.z);
  }
}

// ---- row-footprint feature stage of one warp, with the latent columns shared
// between its lanes by shuffles.  The warp's 32 consecutive texels of one
// output row read at most ceil(31 W_k / W_out) + 2 columns of level k: 23 jobs
// over the four levels of the 1/4..1/32 pyramid, 32 for 1/4, 1/4, 1/8, 1/8.
// Lane L owns column job L (the strip cache above, per warp: it keeps its two
// decoded texels across rows and re-decodes only when the vertical tap pair
// moves), blends them vertically once per row, and each texel reads its two
// horizontal neighbours from the lanes that hold them -- no shared memory and
// no barrier across warps.  A footprint of more than 32 jobs (level-to-output
// ratios above ~1/4) samples each texel on its own.
__device__ __forceinline__ void direct_features(const DecodeArgs& a, int64_t t, float (&feat)[12]);

__device__ __forceinline__ void warp_strip_features(const DecodeArgs& a, int j, int i0w, int lane, StripCache& C,
                                                    float (&feat)[12]) {
  const float s = 1.0f / 255.0f;
  if (i0w != C.i0) {  // new strip: the warp's column plan, own job, own texel's source lanes
    C.i0 = i0w;
    C.key = INT_MIN + 1;
    const float u0 = grid_coord((float)i0w, a.cw);
    const float u1 = grid_coord((float)(i0w + 31), a.cw);
    const float u = grid_coord((float)(i0w + lane), a.cw);
    int total = 0, job = -1, jx = 0;
    uint32_t src4 = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const LevelView& L = a.lv[k];
      const int b0 = (int)floorf(texel_coord(u0, L.w, L.shift));
      const int b1 = (int)floorf(texel_coord(u1, L.w, L.shift));
      const int span = b1 - b0 + 2;
      if (lane >= total && lane < total + span) {
        job = k | (lane - total) << 2;
        jx = wrap_or_clamp(b0 + lane - total, L.w, a.wrap);
      }
      const float tx = texel_coord(u, L.w, L.shift);
      const float ftx = floorf(tx);
      C.fx[k] = tx - ftx;
      // floor is monotone in u, so the left tap's job lies in [0, span - 2]; the clamp only guards the lanes
      src4 |= (uint32_t)min(total + min(max((int)ftx - b0, 0), span - 2), 30) << (8 * k);
      total += span;
    }
    C.total = total;
    C.job = job;
    C.jx = jx;
    C.rel4 = src4;
  }
  if (C.total > 32) {  // warp-uniform: a footprint wider than the warp's lanes
    direct_features(a, (int64_t)j * a.grid_w + i0w + lane, feat);
    return;
  }
  float cv0 = 0.f, cv1 = 0.f, cv2 = 0.f;
  if (C.job >= 0) {
    const int k = C.job & 3;
    const LevelView& L = a.lv[k];
    const float ty = texel_coord(grid_coord((float)(j + a.row0), a.ch), L.h, L.shift);
    const float fty = floorf(ty);
    const float fy = ty - fty;
    const int key = (int)fty;
    if (key != C.key) {
      uint32_t t0;
      if (key == C.key + 1) {
        t0 = C.t1;
      } else {
        const int y0 = wrap_or_clamp(key, L.h, a.wrap);
        t0 = bc1_texel(__ldg(L.blocks + block_index(L, C.jx >> 2, y0 >> 2)), C.jx & 3, y0 & 3);
      }
      const int y1 = wrap_or_clamp(key + 1, L.h, a.wrap);
      const uint32_t t1 = bc1_texel(__ldg(L.blocks + block_index(L, C.jx >> 2, y1 >> 2)), C.jx & 3, y1 & 3);
      C.key = key;
      C.t1 = t1;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v0 = (float)((t0 >> (8 * c)) & 255u), v1 = (float)((t1 >> (8 * c)) & 255u);
        C.c0[c] = s * v0;
        C.dc[c] = s * (v1 - v0);
      }
    }
    cv0 = fmaf(fy, C.dc[0], C.c0[0]);
    cv1 = fmaf(fy, C.dc[1], C.c0[1]);
    cv2 = fmaf(fy, C.dc[2], C.c0[2]);
    const float tyn = texel_coord(grid_coord((float)(j + a.row0 + 1), a.ch), L.h, L.shift);
    const int keyn = (int)floorf(tyn);
    if (keyn != key && j + 1 < a.grid_h) {
      const int y1 = wrap_or_clamp(keyn + 1, L.h, a.wrap);
      sm100::prefetch_l1(L.blocks + block_index(L, C.jx >> 2, y1 >> 2));
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int src = (C.rel4 >> (8 * k)) & 255;
    const float a0 = __shfl_sync(0xffffffffu, cv0, src), b0 = __shfl_sync(0xffffffffu, cv0, src + 1);
    const float a1 = __shfl_sync(0xffffffffu, cv1, src), b1 = __shfl_sync(0xffffffffu, cv1, src + 1);
    const float a2 = __shfl_sync(0xffffffffu, cv2, src), b2 = __shfl_sync(0xffffffffu, cv2, src + 1);
    feat[3 * k + 0] = fmaf(C.fx[k], b0 - a0, a0);
    feat[3 * k + 1] = fmaf(C.fx[k], b1 - a1, a1);
    feat[3 * k + 2] = fmaf(C.fx[k], b2 - a2, a2);
  }
}

// Per-material description used by the batched and frame decodes: the level
// views of mip 0 (in `d`) plus every level's mip chain for trilinear sampling.
struct MatDev {
  DecodeArgs d;          // mip-0 views, wrap flag, output grid and buffer of the full decode
  const void* packed;    // FP16 packed MLP
  int nout;
  FastDiv hdiv;          // full decode: division by grid_h (tile number -> column block)
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

// Anisotropic latent filter of one frame pixel (the reference formulas of the
// anisotropic-filtering extension, in texture-coordinate units -- the square
// latents make Pmax / Pmin the same for every level): N = min(ceil(Pmax /
// Pmin), max_aniso) trilinear probes at uv + (i / (N + 1) - 1/2) d along the
// major-axis derivative d, each level at lod bias + log2(Pmax W_k / N),
// averaged.  N is decided with correctly rounded FP32 operations in a fixed
// order (no contraction), so any IEEE implementation decides it alike.
__device__ __forceinline__ void aniso_features(const MatDev& M, float u, float v, float4 d, float bias,
                                               int max_aniso, float (&feat)[12]) {
  const float px = __fsqrt_rn(__fadd_rn(__fmul_rn(d.x, d.x), __fmul_rn(d.y, d.y)));
  const float py = __fsqrt_rn(__fadd_rn(__fmul_rn(d.z, d.z), __fmul_rn(d.w, d.w)));
  const bool along_x = px >= py;
  const float pmax = along_x ? px : py, pmin = along_x ? py : px;
  int n = 1;
  if (pmax > 0.f) n = pmin > 0.f ? (int)fminf(ceilf(__fdiv_rn(pmax, pmin)), (float)max_aniso) : max_aniso;
  const float au = along_x ? d.x : d.z, av = along_x ? d.y : d.w;
  const float base = bias + log2f(pmax / (float)n);  // -inf for a zero footprint: clamps to mip 0
  const bool wrap = M.d.wrap;
  float acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = 0.f;
  for (int i = 1; i <= n; ++i) {
    const float off = (float)i / (float)(n + 1) - 0.5f;
    const float uu = fmaf(off, au, u), vv = fmaf(off, av, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float lam = fminf(fmaxf(base + M.log2w[k], 0.f), (float)(M.mips[k] - 1));
      const int m0 = (int)floorf(lam);
      const int m1 = min(m0 + 1, M.mips[k] - 1);
      const float t = lam - (float)m0;
      const float3 c0 = sample_bilinear(mip_view(M, k, m0), uu, vv, wrap);
      const float3 c1 = sample_bilinear(mip_view(M, k, m1), uu, vv, wrap);
      acc[3 * k + 0] += fmaf(t, c1.x - c0.x, c0.x);
      acc[3 * k + 1] += fmaf(t, c1.y - c0.y, c0.y);
      acc[3 * k + 2] += fmaf(t, c1.z - c0.z, c0.z);
    }
  }
  const float inv = 1.0f / (float)n;
#pragma unroll
  for (int c = 0; c < 12; ++c) feat[c] = acc[c] * inv;
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
