// Types shared by the tensor-core decode kernel and its launchers (single
// material, batched materials, frame).
#pragma once

#include "features.cuh"
#include "host.h"
#include "shade.cuh"

namespace nbtc {

constexpr int kTile = 128;           // texels per tile = MMA M
constexpr int kHid = 64;             // hidden width of the tensor-core forms
constexpr int kOutPad = 16;          // output layer N (channels padded)
constexpr int kMaxOut = 16;

// Operand forms of the tensor-core decode.  The split forms carry every weight
// and activation as a pair hi + lo of the narrow format and run three products
// per layer into one FP32 accumulator: hi(A) hi(W) + lo(A) hi(W) + hi(A) lo(W).
// kF32Split is kF16Split with the output layer's FP32 accumulator written as
// FP32 (no output rounding): the FP32-accurate form.
enum TcForm { kF16 = 0, kF8 = 1, kF16Split = 2, kF8Split = 3, kF32Split = 4 };

// Bytes of per-warp output staging: 32 texels x up to 16 channels of FP16, or FP32.
__host__ __device__ constexpr int stage_bytes(int form) { return form == kF32Split ? 2048 : 1024; }

// Byte layout of a packed MLP (identical in global memory and shared memory).
// FP16 forms: every layer's bias enters the MMA as FP16 operand(s) -- layer 1
// through a K column of W1 (A0 carries a 1 there), later layers through a
// small [N x 16] bias tile multiplied by a tile of ones (split: column 0 holds
// hi(b), column 1 lo(b)).  FP8 forms: the FP32 bias and the per-layer scale are
// applied in the epilogue.  Split forms store every weight tile twice, hi then lo.
//
// W1 (layer 1, K-major, no swizzle) rows:
//   FP16        [W(12) b 0 0 0]                                   K = 16
//   FP8         [W(12) 0 x 20]                                    K = 32
//   FP16 split  [hiW(12) hib 000 | hiW(12) lob 000 | loW(12) 0000] K = 48
//   FP8 split   [hiW(12) 0000 | hiW(12) 0000 | loW(12) 0000 | 0 x 16]  K = 64
// against A0 rows [x(12) 1 000] / [x(12) 0 x 20] / [hi x(12) 1 000 | lo x(12) 1 000]
// / [hi x(12) 0000 | lo x(12) 0000].
struct TcLayout {
  int nhid;   // hidden layers (1..3)
  int form;   // TcForm
  __host__ __device__ bool fp8() const { return form == kF8 || form == kF8Split; }
  __host__ __device__ bool f16split() const { return form == kF16Split || form == kF32Split; }
  __host__ __device__ bool split() const { return f16split() || form == kF8Split; }
  __host__ __device__ int esz() const { return fp8() ? 1 : 2; }
  __host__ __device__ int parts() const { return split() ? 2 : 1; }
  __host__ __device__ int w1_row() const { return f16split() ? 96 : form == kF8Split ? 64 : 32; }
  __host__ __device__ int a0_row() const { return f16split() ? 64 : 32; }
  __host__ __device__ int wh_part() const { return kHid * kHid * esz(); }                // 64 x 64
  __host__ __device__ int wh_bytes() const { return parts() * wh_part(); }
  __host__ __device__ int bth_bytes() const { return fp8() ? 0 : kHid * 16 * 2; }       // 64 x 16 bias tile
  __host__ __device__ int wo_part() const { return kOutPad * kHid * esz(); }             // 16 x 64
  __host__ __device__ int wo_bytes() const { return parts() * wo_part(); }
  __host__ __device__ int bto_bytes() const { return fp8() ? 0 : kOutPad * 16 * 2; }    // 16 x 16 bias tile
  __host__ __device__ int off_w1() const { return 0; }
  __host__ __device__ int off_wh(int l) const { return kHid * w1_row() + l * (wh_bytes() + bth_bytes()); }  // l < nhid-1
  __host__ __device__ int off_bth(int l) const { return off_wh(l) + wh_bytes(); }
  __host__ __device__ int off_wo() const { return off_wh(nhid - 1); }
  __host__ __device__ int off_bto() const { return off_wo() + wo_bytes(); }
  __host__ __device__ int off_bias() const { return off_bto() + bto_bytes(); }    // nhid*64 + 16 floats
  __host__ __device__ int off_alpha() const { return off_bias() + (nhid * kHid + kOutPad) * 4; }  // 8 floats
  __host__ __device__ int bytes() const { return (off_alpha() + 8 * 4 + 15) & ~15; }
};

// Offset of element (row, k) in a K-major operand tile.
//  no swizzle, 16-byte core matrices of 8 rows: LBO = 128 B (next K chunk),
//  SBO = 8 rows x `row` bytes (next 8 rows); `row` = bytes of K per row
__host__ __device__ inline uint32_t off_ilv(int row, int kbyte, int rowbytes) {
  return (uint32_t)((row >> 3) * 8 * rowbytes + (kbyte >> 4) * 128 + (row & 7) * 16 + (kbyte & 15));
}
__host__ __device__ inline uint32_t off_interleave(int row, int kbyte) { return off_ilv(row, kbyte, 32); }
//  128-byte swizzle, 128-byte rows (64 f16): atom 8 rows x 128 B, SBO = 1024 B
__host__ __device__ inline uint32_t off_sw128(int row, int kbyte) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((kbyte >> 4) ^ (row & 7)) & 7) << 4) + (kbyte & 15));
}
//  64-byte swizzle, 64-byte rows (64 e4m3): atom 8 rows x 64 B, SBO = 512 B
__host__ __device__ inline uint32_t off_sw64(int row, int kbyte) {
  return (uint32_t)((row >> 3) * 512 + (row & 7) * 64 + ((((kbyte >> 4) ^ ((row & 7) >> 1)) & 3) << 4) +
                    (kbyte & 15));
}

// A run of tiles of one material: full-decode row tiles (numbered column-major
// within the material), or frame tiles -- uniform (a list of 128-pixel screen
// tiles) or packed (128-slot lists of pixel indices).
enum ChunkKind { kChunkGrid = 0, kChunkUniform = 1, kChunkPacked = 2 };
struct WorkChunk {
  int mat;
  int kind;
  int64_t first;
  int count;
  int pad;
};

enum TcMode { kModeSingle = 0, kModeBatch = 1 };

struct TcArgs {
  DecodeArgs d;
  const void* packed;
  int nout;
  int footprint;       // 1: row-footprint feature stage
  FastDiv hdiv;        // footprint mode: division by grid_h (tile number -> column block)
  int64_t tiles;
  int64_t per_cta;     // tiles per CTA (contiguous range)
  long long budget;    // polls per bounded wait
  // batched materials / frame
  int mode;
  const MatDev* mats;
  const WorkChunk* chunks;
  const int* nchunks_dev;  // chunk count, read on the device
  int* chunk_counter;      // next chunk to take (zeroed before the launch)
  const int* ulist;        // frame: uniform screen tiles
  const int* plist;        // frame: packed pixel indices (128 per tile, -1 = none)
  const int* fmat;         // frame: per-pixel material id
  const float* fuv;        // frame: per-pixel uv
  const float* flod;       // frame: per-pixel lod (log2 of the uv footprint + bias), or the bias with fduv
  const float* fduv;       // frame: per-pixel uv derivatives (anisotropic filter) or NULL
  int max_aniso;           // frame: probe cap of the anisotropic filter
  float* fshade;           // frame: lighting pass output (FP32 RGBA per pixel) or NULL
  LightDev light;          // frame: lighting constants
  uint16_t* fout;          // frame: per-pixel output (nout FP16)
  int frame_w, tile_w, tile_h, tiles_x;
  int64_t frame_pixels;    // frame: pixel count (bounds of the checked build)
  int tmem_a;              // 1 = MMA A operands in TMEM (else shared memory)
};

// Per-CTA view of the chunk being decoded (in shared memory).
struct TcWork {
  MatDev m;
  WorkChunk c;
  int valid;
  int reload;
};



struct TcArgs;
// Launches the decode kernel (any mode) with W warpgroups of `slots` tile
// slots each on `grid` CTAs.
nbtc_status launch_tc_args(nbtc_context* ctx, const struct TcArgs& p, int nhid, int form, int W, int slots, int grid,
                           cudaStream_t s);

}  // namespace nbtc
