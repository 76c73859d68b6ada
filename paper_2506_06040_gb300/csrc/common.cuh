// Shared device-side pieces of the decoder: status reporting, BC1 texel
// decode, bilinear latent sampling.  Host code includes it for the argument
// structs only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nbtc.h"
#include "gridcoord.h"

namespace nbtc {

constexpr int kMaxLevels = NBTC_MAX_LEVELS;

// Device-side view of one latent level at one mip.
struct LevelView {
  const uint64_t* blocks;  // row-major 8-byte BC1 blocks of this mip
  int32_t w, h;            // texels
  int32_t wb;              // blocks per row (w / 4)
  float shift;             // texels, both axes
#ifdef NBTC_CHECKED
  int* status;             // checked build: where an index outside the level is recorded
  int32_t plant;           // checked build, tests only: added to every block index (0 otherwise)
#endif
};

// ---------------------------------------------------------------- status word

// First fault wins; later faults leave the recorded code in place.
__device__ __forceinline__ void record_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------- bounds checks
//
// The checked build (compiled with NBTC_CHECKED) tests every gather index the
// kernels form against the extent of the array it indexes: an index outside
// it records NBTC_ERR_BOUNDS in the launch's status word and is replaced by 0,
// a valid element, so no access leaves its array and nothing traps.  The
// default build compiles the checks away.
#ifdef NBTC_CHECKED
__device__ __forceinline__ int64_t checked_index(int64_t i, int64_t n, int* status) {
  if (i < 0 || i >= n) {
    record_status(status, NBTC_ERR_BOUNDS);
    return 0;
  }
  return i;
}
#define NBTC_CHECK_INDEX(i, n, status) ((i) = ::nbtc::checked_index((i), (n), (status)))
#else
#define NBTC_CHECK_INDEX(i, n, status) ((void)0)
#endif

// Index of block (bx, by) of a level view.
__device__ __forceinline__ int64_t block_index(const LevelView& L, int bx, int by) {
  int64_t i = (int64_t)by * L.wb + bx;
#ifdef NBTC_CHECKED
  i += L.plant;
  NBTC_CHECK_INDEX(i, (int64_t)L.wb * (L.h / 4), L.status);
#endif
  return i;
}

// ---------------------------------------------------------------- BC1 decode

// RGB565 -> 8-bit channels by bit replication, as three ints.
__device__ __forceinline__ void expand565(uint32_t c, int& r, int& g, int& b) {
  const int r5 = (c >> 11) & 31, g6 = (c >> 5) & 63, b5 = c & 31;
  r = (r5 << 3) | (r5 >> 2);
  g = (g6 << 2) | (g6 >> 4);
  b = (b5 << 3) | (b5 >> 2);
}

// One palette channel.  Four-colour blocks (c0 > c1) weight the endpoints
// (3,0) (0,3) (2,1) (1,2) for indices 0..3 and divide by 3 after adding 1;
// three-colour blocks weight them (2,0) (0,2) (1,1) and divide by 2 after adding
// 1, index 3 being black.  (3 e + 1) / 3 == e and (2 e + 1) / 2 == e, so the
// endpoints come out unchanged.
__device__ __forceinline__ int palette_channel(int e0, int e1, int a0, int a1, bool four) {
  const int num = a0 * e0 + a1 * e1 + 1;
  return four ? num / 3 : num >> 1;
}

// Decoded RGB8 of texel (tx, ty) of a block, packed r | g << 8 | b << 16.
__device__ __forceinline__ uint32_t bc1_texel(uint64_t blk, int tx, int ty) {
  const uint32_t c0 = (uint32_t)(blk & 0xFFFFu);
  const uint32_t c1 = (uint32_t)((blk >> 16) & 0xFFFFu);
  const int idx = (int)((uint32_t)(blk >> 32) >> (2 * (4 * ty + tx))) & 3;
  const bool four = c0 > c1;
  int r0, g0, b0, r1, g1, b1;
  expand565(c0, r0, g0, b0);
  expand565(c1, r1, g1, b1);
  // endpoint weights per index
  int a0, a1;
  if (four) {
    a0 = (idx == 0) ? 3 : (idx == 1) ? 0 : (idx == 2) ? 2 : 1;
    a1 = 3 - a0;
  } else {
    a0 = (idx == 0) ? 2 : (idx == 1) ? 0 : (idx == 2) ? 1 : 0;
    a1 = (idx == 3) ? 0 : 2 - a0;
  }
  uint32_t r = palette_channel(r0, r1, a0, a1, four);
  uint32_t g = palette_channel(g0, g1, a0, a1, four);
  uint32_t b = palette_channel(b0, b1, a0, a1, four);
  if (!four && idx == 3) r = g = b = 0;
  return r | (g << 8) | (b << 16);
}

__device__ __forceinline__ uint32_t fetch_texel(const LevelView& L, int x, int y) {
  const uint64_t blk = __ldg(L.blocks + block_index(L, x >> 2, y >> 2));
  return bc1_texel(blk, x & 3, y & 3);
}

// ---------------------------------------------------------------- sampling

// Integer neighbours and fractional weight along one axis.  The texel
// coordinate is t = u * n - 0.5 + shift; neighbours floor(t) and floor(t) + 1
// are clamped to [0, n-1] or wrapped modulo n.
__device__ __forceinline__ void axis_taps(float u, int n, float shift, bool wrap, int& i0, int& i1,
                                          float& f) {
  // wrap: drop whole periods of u first (u - floor(u) is exact), so the texel
  // coordinate keeps its fraction even for tiled uv far from [0, 1)
  if (wrap) u -= floorf(u);
  float t = fmaf(u, (float)n, shift - 0.5f);
  if (!wrap) t = fminf(fmaxf(t, -1.0f), (float)n);  // outside this range clamping decides
  const float fl = floorf(t);
  f = t - fl;  // exact
  const int a = (int)fl;
  if (wrap) {  // u in [0, 1] and |shift| <= 1/2: a in [-1, n], wrapped as an integer
    i0 = a < 0 ? a + n : (a >= n ? a - n : a);
    i1 = i0 + 1 >= n ? i0 + 1 - n : i0 + 1;
  } else {
    i0 = min(max(a, 0), n - 1);
    i1 = min(max(a + 1, 0), n - 1);
  }
}

// Bilinear sample of one BC1 level at uv, FP32, channels in [0, 1].
__device__ __forceinline__ float3 sample_bilinear(const LevelView& L, float u, float v, bool wrap) {
  int x0, x1, y0, y1;
  float fx, fy;
  axis_taps(u, L.w, L.shift, wrap, x0, x1, fx);
  axis_taps(v, L.h, L.shift, wrap, y0, y1, fy);
  const uint32_t t00 = fetch_texel(L, x0, y0), t10 = fetch_texel(L, x1, y0);
  const uint32_t t01 = fetch_texel(L, x0, y1), t11 = fetch_texel(L, x1, y1);
  const float w00 = (1.f - fx) * (1.f - fy), w10 = fx * (1.f - fy);
  const float w01 = (1.f - fx) * fy, w11 = fx * fy;
  float3 c;
  const float s = 1.0f / 255.0f;
#define NBTC_CH(sh)                                                                          \
  (s * (w00 * (float)((t00 >> sh) & 255u) + w10 * (float)((t10 >> sh) & 255u) +             \
        w01 * (float)((t01 >> sh) & 255u) + w11 * (float)((t11 >> sh) & 255u)))
  c.x = NBTC_CH(0);
  c.y = NBTC_CH(8);
  c.z = NBTC_CH(16);
#undef NBTC_CH
  return c;
}

// Arguments shared by the decode kernels (passed by value).
struct DecodeArgs {
  LevelView lv[4];
  int32_t wrap;
  const float* uv;  // NULL = grid mode
  int64_t n;
  int32_t grid_w, grid_h;  // grid mode: texels per row, rows decoded by this call
  int32_t row0;            // grid mode: first row (of the full grid) decoded by this call
  GridCoord cw, ch;        // grid mode: width and height of the full grid (texel-centre coordinates)
  void* out;
  int* status;
};

// uv of output texel t.
__device__ __forceinline__ float2 texel_uv(const DecodeArgs& a, int64_t t) {
  if (a.uv) return __ldg(reinterpret_cast<const float2*>(a.uv) + t);
  int64_t j, i;
  if (a.n <= 0xFFFFFFFFll) {  // 32-bit division when the grid allows it
    const uint32_t tj = (uint32_t)t / (uint32_t)a.grid_w;
    j = tj;
    i = (uint32_t)t - tj * (uint32_t)a.grid_w;
  } else {
    j = t / a.grid_w;
    i = t - j * a.grid_w;
  }
  return make_float2(grid_coord((float)i, a.cw), grid_coord((float)(j + a.row0), a.ch));
}

}  // namespace nbtc
