// Tensor-core forms of the fused decode (FP16 and FP8 E4M3 operands, FP32
// accumulation in TMEM, FP16 output) -- the GB300 counterpart of the paper's
// cooperative-vector MLP (Sec. 4, "Neural inference in G-Buffer pass"): the
// MLP of every 128-texel tile runs as a chain of tcgen05.mma with M = 128
// texels, N = layer width, the weights resident in shared memory.
//
// Work split: a CTA of G groups x 128 threads, one CTA per SM (persistent).
// Each group owns a tile at a time and walks it through
//   features (BC1 decode + bilinear, SIMT) -> A0 tile in smem
//   -> MMA layer 1 -> epilogue (bias, ReLU, narrow) -> A tile -> MMA layer 2 ...
//   -> output epilogue -> smem staging -> bulk store to global.
// One elected thread per group issues that group's MMAs; the G groups
// interleave, so one group's SIMT work overlaps another group's MMAs.
#include "features.cuh"
#include "host.h"
#include "sm100.cuh"

namespace nbtc {

using namespace sm100;

constexpr int kTile = 128;           // texels per tile = MMA M
constexpr int kHid = 64;             // hidden width of the tensor-core forms
constexpr int kOutPad = 16;          // output layer N (channels padded)
constexpr int kMaxOut = 16;

// Byte layout of a packed MLP (identical in global memory and shared memory).
// FP16: every layer's bias enters the MMA as an FP16 operand -- layer 1 through
// K column 12 of W1 (A0 carries a 1 there), later layers through a small
// [N x 16] bias tile multiplied by a tile of ones.  FP8: the FP32 bias and the
// per-layer scale are applied in the epilogue.
struct TcLayout {
  int nhid;   // hidden layers (1..3)
  bool fp8;
  __host__ __device__ int esz() const { return fp8 ? 1 : 2; }
  __host__ __device__ int wh_bytes() const { return kHid * kHid * esz(); }   // 64 x 64
  __host__ __device__ int bth_bytes() const { return fp8 ? 0 : kHid * 16 * 2; }   // 64 x 16 bias tile
  __host__ __device__ int wo_bytes() const { return kOutPad * kHid * esz(); }   // 16 x 64
  __host__ __device__ int bto_bytes() const { return fp8 ? 0 : kOutPad * 16 * 2; }  // 16 x 16 bias tile
  __host__ __device__ int off_w1() const { return 0; }                                // 64 x K1: 2048 B
  __host__ __device__ int off_wh(int l) const { return 2048 + l * (wh_bytes() + bth_bytes()); }  // l < nhid-1
  __host__ __device__ int off_bth(int l) const { return off_wh(l) + wh_bytes(); }
  __host__ __device__ int off_wo() const { return off_wh(nhid - 1); }
  __host__ __device__ int off_bto() const { return off_wo() + wo_bytes(); }
  __host__ __device__ int off_bias() const { return off_bto() + bto_bytes(); }    // nhid*64 + 16 floats
  __host__ __device__ int off_alpha() const { return off_bias() + (nhid * kHid + kOutPad) * 4; }  // 8 floats
  __host__ __device__ int bytes() const { return (off_alpha() + 8 * 4 + 15) & ~15; }
};

// Offset of element (row, k) in a K-major operand tile.
//  no swizzle, 16-byte core matrices of 8 rows: LBO = 128 B (next K chunk), SBO = 256 B (next 8 rows)
__host__ __device__ inline uint32_t off_interleave(int row, int kbyte) {
  return (uint32_t)((row >> 3) * 256 + (kbyte >> 4) * 128 + (row & 7) * 16 + (kbyte & 15));
}
//  128-byte swizzle, 128-byte rows (64 f16): atom 8 rows x 128 B, SBO = 1024 B
__host__ __device__ inline uint32_t off_sw128(int row, int kbyte) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((kbyte >> 4) ^ (row & 7)) & 7) << 4) + (kbyte & 15));
}
//  64-byte swizzle, 64-byte rows (64 e4m3): atom 8 rows x 64 B, SBO = 512 B
__host__ __device__ inline uint32_t off_sw64(int row, int kbyte) {
  return (uint32_t)((row >> 3) * 512 + (row & 7) * 64 + ((((kbyte >> 4) ^ ((row & 7) >> 1)) & 3) << 4) +
                    (kbyte & 15));
}

struct TcArgs {
  DecodeArgs d;
  const void* packed;
  int nout;
  int footprint;       // 1: row-footprint feature stage
  int tiles_per_row;   // footprint mode: grid_w / 128
  int64_t tiles;
  int64_t per_cta;     // tiles per CTA (contiguous range)
  long long budget;    // polls per bounded wait
};

constexpr int kMmaWarps = 4;       // one MMA-issuing warp per SM sub-partition

// Tile numbering.  Each CTA owns a contiguous range of tile numbers; in
// row-footprint mode consecutive numbers run down a column of 128-texel tiles
// (number -> row = T % H, column block = T / H), so the tiles a CTA decodes at
// the same time sit on neighbouring rows and share latent blocks in L1.
// Returns the first output texel of tile T.
__device__ __forceinline__ int64_t tile_first_texel(const TcArgs& p, int64_t T) {
  if (!p.footprint) return T * 128;
  const uint32_t t = (uint32_t)T, h = (uint32_t)p.d.grid_h;
  const uint32_t col = t / h, row = t - col * h;
  return (int64_t)row * p.d.grid_w + (int64_t)col * 128;
}

constexpr int kSlots = 2;          // tile slots per warpgroup (ping-pong)
constexpr int kStageBytes = 1024;  // per-warp output staging (32 texels x <= 16 halves)

// Shared-memory plan.  Per slot: A0 (128 x K1 operand) and Ah (128 x 64
// operand, also the feature stage's column buffer while no MMA reads it).
struct TcSmem {
  int image;       // packed MLP (rounded to 1 KB)
  int ones;        // 128 x 16 FP16 tile of ones in column 0
  int slots;       // first slot
  int slot;        // bytes per slot
  int a0, ah;      // offsets inside a slot
  int stage;       // per-warp output staging
  int bars;        // A-ready[NS], D-ready[NS], weight barrier
  int tslot;       // TMEM address slot
  int total;
};

__host__ __device__ inline TcSmem tc_smem(const TcLayout& L, int W) {
  TcSmem s;
  const int NS = W * kSlots;
  s.image = (L.bytes() + 1023) & ~1023;
  s.ones = s.image;
  s.slots = s.ones + 4096;
  s.a0 = 0;
  s.ah = 4096;
  s.slot = 4096 + 16384;
  s.stage = s.slots + NS * s.slot;
  s.bars = s.stage + W * 4 * kStageBytes;
  s.tslot = s.bars + (2 * NS + 1) * 8;
  s.total = s.tslot + 16 + 1024 /* alignment slack */;
  return s;
}

// Warp-specialised persistent kernel: W warpgroups (4 warps, one thread per
// tile row) compute features and epilogues; warp 4W issues every MMA.  Each
// warpgroup owns two tile slots (TMEM columns + A buffers) and alternates
// between them, so one slot's epilogue runs while the other slot's MMAs run.
// Slot q walks tiles q + NS * (blockIdx.x + gridDim.x * i).
//
// Hand-offs (all mbarriers, all waits bounded):
//   A-ready[q]  (128 arrivals): slot q's A operand for its next layer is in smem
//   D-ready[q]  (tcgen05.commit): that layer's accumulator is in TMEM
// After a timeout a thread stops waiting but keeps its schedule (every
// barrier and arrival still happens), so the kernel always terminates.
template <int NHID, bool FP8, int W>
__global__ void __launch_bounds__(W * 128 + 32 * kMmaWarps, 1) k_decode_tc(TcArgs p) {
  constexpr TcLayout L{NHID, FP8};
  constexpr int NS = W * kSlots;
  constexpr uint32_t kTmemCols = NS * kHid <= 256 ? 256 : 512;
  static_assert(NS * kHid <= 512, "TMEM holds at most 512 columns");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const TcSmem S = tc_smem(L, W);
  const uint32_t sbase = smem_u32(smem);
  const int tid = threadIdx.x;
  const int warp = tid / 32, lane = tid % 32;
  const uint32_t abar0 = sbase + S.bars, dbar0 = abar0 + NS * 8, wbar = dbar0 + NS * 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S.tslot);

  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) {
      mbar_init(abar0 + q * 8, kTile);
      mbar_init(dbar0 + q * 8, 1);
    }
    mbar_init(wbar, 1);
    fence_mbar_init();
    mbar_expect_tx(wbar, (uint32_t)L.bytes());
    bulk_g2s(sbase, p.packed, (uint32_t)L.bytes(), wbar);
  }
  if (!FP8 && tid < kTile) {  // ones tile: column 0 = 1.0 (FP16), rest 0
    sts128(sbase + S.ones + off_interleave(tid, 0), 0x3C00u, 0u, 0u, 0u);
    sts128(sbase + S.ones + off_interleave(tid, 16), 0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  bool failed = !mbar_wait_bounded(wbar, 0, p.budget);
  failed = __syncthreads_or(failed);
  const int64_t range_begin = (int64_t)blockIdx.x * p.per_cta;
  const int64_t range_end = range_begin + p.per_cta < p.tiles ? range_begin + p.per_cta : p.tiles;

  if (warp >= 4 * W) {
    // ------------------------------------------------------------ MMA warps
    // MMA warp m issues for slots q = m, m + kMmaWarps, ...  Descriptors are
    // built once; per MMA only the 32-bit low word advances along K.
    const int m = warp - 4 * W;
    if (lane == 0 && m < NS) {
      constexpr int NQ = (NS + kMmaWarps - 1) / kMmaWarps;
      constexpr uint32_t ID_HID = idesc(0, kTile, kHid);
      constexpr uint32_t ID_OUT = idesc(0, kTile, kOutPad);
      // high words: SBO, version, swizzle; low words: start address, LBO
      const uint32_t hi_int = (uint32_t)(smem_desc(0, 128, 256, kSwzNone) >> 32);
      const uint32_t hi_w = FP8 ? (uint32_t)(smem_desc(0, 16, 512, kSwz64) >> 32)
                                : (uint32_t)(smem_desc(0, 16, 1024, kSwz128) >> 32);
      auto lo = [](uint32_t addr, uint32_t lbo) { return (uint32_t)smem_desc(addr, lbo, 0, 0); };
      const uint32_t lo_w1 = lo(sbase + L.off_w1(), 128);
      const uint32_t lo_ones = lo(sbase + S.ones, 128);
      int64_t next[NQ];
      int stage[NQ];
      uint32_t aph[NQ];
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        next[i] = range_begin + m + i * kMmaWarps;
        stage[i] = 0;
        aph[i] = 0;
      }
      long long idle = 0;
      for (;;) {
        bool any = false, progressed = false;
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
          const int q = m + i * kMmaWarps;
          if (q >= NS || next[i] >= range_end) continue;
          any = true;
          if (!failed && !mbar_test_wait(abar0 + q * 8, aph[i])) continue;
          aph[i] ^= 1u;
          progressed = true;
          tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(q * kHid);
          const uint32_t slot = sbase + S.slots + q * S.slot;
          const int l = stage[i];
          if (l == 0) {
            const uint64_t ad = ((uint64_t)hi_int << 32) | lo(slot + S.a0, 128);
            const uint64_t bd = ((uint64_t)hi_int << 32) | lo_w1;
            if constexpr (FP8) mma_f8(d, ad, bd, ID_HID, 0);
            else mma_f16(d, ad, bd, ID_HID, 0);
          } else {
            const bool last = l == NHID;
            const uint32_t id = last ? ID_OUT : ID_HID;
            const uint32_t lo_a = lo(slot + S.ah, 16);
            const uint32_t lo_b = lo(sbase + (last ? L.off_wo() : L.off_wh(l - 1)), 16);
            if constexpr (FP8) {
#pragma unroll
              for (int kk = 0; kk < 2; ++kk)
                mma_f8(d, ((uint64_t)hi_w << 32) | (lo_a + 2 * kk), ((uint64_t)hi_w << 32) | (lo_b + 2 * kk), id,
                       kk > 0);
            } else {
              const uint32_t lo_bt = lo(sbase + (last ? L.off_bto() : L.off_bth(l - 1)), 128);
              mma_f16(d, ((uint64_t)hi_int << 32) | lo_ones, ((uint64_t)hi_int << 32) | lo_bt, id, 0);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_f16(d, ((uint64_t)hi_w << 32) | (lo_a + 2 * kk), ((uint64_t)hi_w << 32) | (lo_b + 2 * kk), id, 1);
            }
          }
          mma_commit(dbar0 + q * 8);
          if (++stage[i] > NHID) {
            stage[i] = 0;
            next[i] += NS;
          }
        }
        if (!any) break;
        if (progressed) {
          idle = 0;
        } else if (++idle > p.budget) {
          failed = true;  // stop waiting; finish the schedule without waits
          record_status(p.d.status, NBTC_ERR_TIMEOUT);
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ warpgroups
    const int wg = warp / 4, wq = warp & 3;
    const int gt = tid % kTile;
    const int bar_id = 1 + wg;
    const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
    unsigned char* stage_w = smem + S.stage + warp * kStageBytes;
    const float* bias = reinterpret_cast<const float*>(smem + L.off_bias());
    const float* alpha = reinterpret_cast<const float*>(smem + L.off_alpha());
    int64_t tile[kSlots];
    int stg[kSlots];
    uint32_t dph[kSlots];

    // features of slot s's current tile -> A0, then A-ready
    auto start_tile = [&](int s) {
      const int q = wg * kSlots + s;
      unsigned char* slot = smem + S.slots + q * S.slot;
      const uint32_t a0 = sbase + S.slots + q * S.slot + S.a0;
      const int64_t t0 = tile_first_texel(p, tile[s]);
      float f[12];
      if (p.footprint) {
        // Ah is free: the previous tile's last MMA (which read it) has completed
        footprint_features<kTile>(p.d, t0, gt, reinterpret_cast<float4*>(slot + S.ah), bar_id, f);
      } else {
        const int64_t tex = t0 + gt;
        direct_features(p.d, tex < p.d.n ? tex : p.d.n - 1, f);
      }
      if constexpr (!FP8) {
        sts128(a0 + off_interleave(gt, 0), cvt_f16x2(f[0], f[1]), cvt_f16x2(f[2], f[3]), cvt_f16x2(f[4], f[5]),
               cvt_f16x2(f[6], f[7]));
        sts128(a0 + off_interleave(gt, 16), cvt_f16x2(f[8], f[9]), cvt_f16x2(f[10], f[11]),
               0x3C00u /* k = 12: 1.0 for the bias */, 0u);
      } else {
        const float is = alpha[NHID + 1];  // 1 / input scale
        uint32_t w[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          w[i] = (uint32_t)cvt_e4m3x2(f[4 * i] * is, f[4 * i + 1] * is) |
                 ((uint32_t)cvt_e4m3x2(f[4 * i + 2] * is, f[4 * i + 3] * is) << 16);
        sts128(a0 + off_interleave(gt, 0), w[0], w[1], w[2], 0u);
        sts128(a0 + off_interleave(gt, 16), 0u, 0u, 0u, 0u);
      }
      fence_proxy_async_smem();
      mbar_arrive(abar0 + q * 8);
      stg[s] = 0;
    };

#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      tile[s] = range_begin + wg * kSlots + s;
      dph[s] = 0;
      stg[s] = 0;
      if (tile[s] < range_end) start_tile(s);
    }
    for (;;) {
      bool any = false;
#pragma unroll
      for (int s = 0; s < kSlots; ++s) {
        if (tile[s] >= range_end) continue;
        any = true;
        const int q = wg * kSlots + s;
        if (!failed) failed = !mbar_wait_bounded(dbar0 + q * 8, dph[s], p.budget);
        dph[s] ^= 1u;
        failed = __any_sync(0xffffffffu, failed);  // warp-uniform: tcgen05.ld is .sync.aligned
        tc_fence_after();
        const uint32_t taddr = tmem_base + (uint32_t)(q * kHid) + lane_off;
        if (stg[s] < NHID) {
          // ---- hidden epilogue: accumulator -> (bias,) ReLU -> narrow -> Ah
          const uint32_t ah = sbase + S.slots + q * S.slot + S.ah;
          const float alp = alpha[stg[s]];
          const float* b = bias + stg[s] * kHid;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            uint32_t r[32];
            if (!failed) {
              tmem_ld16(taddr + 32 * half, r);
              tmem_ld16(taddr + 32 * half + 16, r + 16);
              tmem_wait_ld32(r);
            }
            if constexpr (!FP8) {
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const int j = 8 * c;
                sts128(ah + off_sw128(gt, 16 * (4 * half + c)),
                       cvt_relu_f16x2(__uint_as_float(r[j + 0]), __uint_as_float(r[j + 1])),
                       cvt_relu_f16x2(__uint_as_float(r[j + 2]), __uint_as_float(r[j + 3])),
                       cvt_relu_f16x2(__uint_as_float(r[j + 4]), __uint_as_float(r[j + 5])),
                       cvt_relu_f16x2(__uint_as_float(r[j + 6]), __uint_as_float(r[j + 7])));
              }
            } else {
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const int j = 16 * c + 4 * e, jj = 32 * half + j;
                  w[e] = (uint32_t)cvt_relu_e4m3x2(fmaf(__uint_as_float(r[j]), alp, b[jj]),
                                                   fmaf(__uint_as_float(r[j + 1]), alp, b[jj + 1])) |
                         ((uint32_t)cvt_relu_e4m3x2(fmaf(__uint_as_float(r[j + 2]), alp, b[jj + 2]),
                                                    fmaf(__uint_as_float(r[j + 3]), alp, b[jj + 3]))
                          << 16);
                }
                sts128(ah + off_sw64(gt, 16 * (2 * half + c)), w[0], w[1], w[2], w[3]);
              }
            }
          }
          fence_proxy_async_smem();
          tc_fence_before();
          mbar_arrive(abar0 + q * 8);
          ++stg[s];
        } else {
          // ---- output epilogue: accumulator -> FP16 -> global (per-warp coalesced)
          uint32_t r[16];
          if (!failed) {
            tmem_ld16(taddr, r);
            tmem_wait_ld16(r);
          }
          tc_fence_before();
          const float alp = alpha[NHID];
          const float* b = bias + NHID * kHid;
          const int64_t t0 = tile_first_texel(p, tile[s]);
          const int64_t tex = t0 + gt;
          const int nout = p.nout;
          uint16_t hv[kMaxOut];
#pragma unroll
          for (int k = 0; k < kMaxOut; ++k)
            hv[k] = __half_as_ushort(FP8 ? __float2half_rn(fmaf(__uint_as_float(r[k]), alp, b[k]))
                                         : __float2half_rn(__uint_as_float(r[k])));
          if (t0 + kTile <= p.d.n) {
            uint16_t* st = reinterpret_cast<uint16_t*>(stage_w);
#pragma unroll
            for (int k = 0; k < kMaxOut; ++k)
              if (k < nout) st[lane * nout + k] = hv[k];
            __syncwarp();
            const int n16 = 4 * nout;  // 32 texels x nout x 2 B / 16 B
            uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(p.d.out) + (t0 + 32 * wq) * nout);
            const uint4* src = reinterpret_cast<const uint4*>(stage_w);
            for (int c = lane; c < n16; c += 32) dst[c] = src[c];
            __syncwarp();
          } else if (tex < p.d.n) {
            uint16_t* o = reinterpret_cast<uint16_t*>(p.d.out) + tex * nout;
#pragma unroll
            for (int k = 0; k < kMaxOut; ++k)
              if (k < nout) o[k] = hv[k];
          }
          tile[s] += NS;
          if (tile[s] < range_end) start_tile(s);
        }
      }
      if (!any) break;
    }
    if (failed && gt == 0) record_status(p.d.status, NBTC_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem_base, kTmemCols);
}

// ------------------------------------------------------------------ packing

// pow2ceil(x / 448) computed exactly: the smallest 2^e with 448 * 2^e >= x.
__device__ float scale_for_absmax(float x) {
  x = fmaxf(x, 1e-30f);
  int e;
  frexpf(x, &e);  // x in [2^(e-1), 2^e)
  int k = e - 9;
  while (ldexpf(448.f, k) < x) ++k;
  while (ldexpf(448.f, k - 1) >= x) --k;
  return ldexpf(1.f, k);
}

// One CTA: converts the FP32 MLP into the shared-memory image.
__global__ void k_pack_mlp(const float* __restrict__ W, const float* __restrict__ B, int nhid, int nin, int nout,
                           int fp8, const float* __restrict__ act_absmax, unsigned char* __restrict__ out) {
  const TcLayout L{nhid, fp8 != 0};
  __shared__ float wmax[8];
  __shared__ float sw[8], sa[8];
  const int nl = nhid + 1;
  if (threadIdx.x < 8) wmax[threadIdx.x] = 0.f;
  __syncthreads();
  // per-layer weight absmax
  int off = 0;
  for (int l = 0; l < nl; ++l) {
    const int in = l == 0 ? nin : kHid, o = l == nhid ? nout : kHid;
    float m = 0.f;
    for (int e = threadIdx.x; e < in * o; e += blockDim.x) m = fmaxf(m, fabsf(W[off + e]));
    atomicMax(reinterpret_cast<int*>(&wmax[l]), __float_as_int(m));
    off += in * o;
  }
  __syncthreads();
  if (threadIdx.x < nl) {
    const int l = threadIdx.x;
    sw[l] = fp8 ? scale_for_absmax(wmax[l]) : 1.f;
    sa[l] = fp8 ? scale_for_absmax(act_absmax[l]) : 1.f;
  }
  __syncthreads();
  // clear the image
  for (int e = threadIdx.x; e < L.bytes(); e += blockDim.x) out[e] = 0;
  __syncthreads();
  off = 0;
  for (int l = 0; l < nl; ++l) {
    const int in = l == 0 ? nin : kHid, o = l == nhid ? nout : kHid;
    for (int e = threadIdx.x; e < in * o; e += blockDim.x) {
      const int n = e / in, k = e - n * in;
      const float w = W[off + e];
      uint32_t dst;
      if (l == 0) dst = L.off_w1() + off_interleave(n, k * L.esz());
      else if (l == nhid) dst = L.off_wo() + (fp8 ? off_sw64(n, k) : off_sw128(n, 2 * k));
      else dst = L.off_wh(l - 1) + (fp8 ? off_sw64(n, k) : off_sw128(n, 2 * k));
      if (fp8) {
        out[dst] = (unsigned char)(cvt_e4m3x2(w / sw[l], 0.f) & 0xFF);
      } else {
        const __half h = __float2half_rn(w);
        *reinterpret_cast<__half*>(out + dst) = h;
      }
    }
    off += in * o;
  }
  if (!fp8) {  // FP16 biases as MMA operands: W1 column 12, then [N x 16] tiles (column 0)
    int bo = 0;
    for (int l = 0; l < nl; ++l) {
      const int o = l == nhid ? nout : kHid;
      for (int e = threadIdx.x; e < o; e += blockDim.x) {
        uint32_t dst;
        if (l == 0) dst = L.off_w1() + off_interleave(e, 2 * nin);
        else if (l == nhid) dst = L.off_bto() + off_interleave(e, 0);
        else dst = L.off_bth(l - 1) + off_interleave(e, 0);
        *reinterpret_cast<__half*>(out + dst) = __float2half_rn(B[bo + e]);
      }
      bo += o;
    }
  }
  // biases (hidden layers pre-divided by the next layer's input scale) and epilogue multipliers
  float* bias = reinterpret_cast<float*>(out + L.off_bias());
  float* alpha = reinterpret_cast<float*>(out + L.off_alpha());
  int boff = 0;
  for (int l = 0; l < nl; ++l) {
    const int o = l == nhid ? nout : kHid;
    const float div = (fp8 && l < nhid) ? sa[l + 1] : 1.f;
    for (int e = threadIdx.x; e < o; e += blockDim.x) bias[l * kHid + e] = B[boff + e] / div;
    boff += o;
  }
  if (threadIdx.x < nl) {
    const int l = threadIdx.x;
    alpha[l] = fp8 ? (l < nhid ? sw[l] * sa[l] / sa[l + 1] : sw[l] * sa[l]) : 1.f;
  }
  if (threadIdx.x == 0) {
    alpha[nhid + 1] = fp8 ? 1.f / sa[0] : 1.f;  // input multiplier
    for (int l = 0; l < nl && l < 3; ++l) alpha[nhid + 2 + l] = fp8 ? sa[l] : 1.f;  // kept for inspection
  }
}

// ------------------------------------------------------------------ host

static nbtc_status tc_shape(const nbtc_mlp* mlp, int& nhid) {
  const int L = mlp->num_layers;
  nhid = L - 1;
  if (nhid < 1 || nhid > 3) return fail(NBTC_ERR_UNSUPPORTED, "tensor-core forms take 1..3 hidden layers");
  if (mlp->dims[0] != 12) return fail(NBTC_ERR_UNSUPPORTED, "tensor-core forms take 12 input features");
  for (int l = 1; l < L; ++l)
    if (mlp->dims[l] != kHid) return fail(NBTC_ERR_UNSUPPORTED, "tensor-core forms take hidden width 64");
  if (mlp->dims[L] < 1 || mlp->dims[L] > kMaxOut) return fail(NBTC_ERR_UNSUPPORTED, "at most 16 outputs");
  return NBTC_OK;
}

nbtc_status tc_packed_bytes(const nbtc_mlp* mlp, int precision, size_t* bytes) {
  int nhid;
  nbtc_status st = tc_shape(mlp, nhid);
  if (st) return st;
  *bytes = (size_t)TcLayout{nhid, precision == NBTC_FP8_E4M3}.bytes();
  return NBTC_OK;
}

nbtc_status launch_pack_mlp(nbtc_context* ctx, const nbtc_mlp* mlp, int precision, const float* act_absmax,
                            void* packed, size_t packed_bytes, cudaStream_t s) {
  (void)ctx;
  int nhid;
  nbtc_status st = tc_shape(mlp, nhid);
  if (st) return st;
  const TcLayout L{nhid, precision == NBTC_FP8_E4M3};
  if (packed_bytes < (size_t)L.bytes()) return fail(NBTC_ERR_INVALID_ARG, "packed buffer too small");
  if (!packed || !aligned(packed, 16)) return fail(NBTC_ERR_INVALID_ARG, "packed buffer NULL or not 16-byte aligned");
  if (L.fp8 && !act_absmax) return fail(NBTC_ERR_INVALID_ARG, "FP8 packing needs the calibration absmax");
  k_pack_mlp<<<1, 256, 0, s>>>(mlp->weights, mlp->biases, nhid, mlp->dims[0], mlp->dims[nhid + 1], L.fp8 ? 1 : 0,
                               act_absmax, static_cast<unsigned char*>(packed));
  return cuda_check(cudaGetLastError(), "launch k_pack_mlp");
}

template <int NHID, bool FP8, int W>
static nbtc_status launch_tc_g(nbtc_context* ctx, const TcArgs& p, cudaStream_t s) {
  const TcSmem S = tc_smem(TcLayout{NHID, FP8}, W);
  auto kern = k_decode_tc<NHID, FP8, W>;
  nbtc_status st =
      cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S.total), "smem attribute");
  if (st) return st;
  int64_t grid = (p.tiles + W * kSlots - 1) / (W * kSlots);
  if (grid > ctx->sm_count) grid = ctx->sm_count;
  TcArgs q = p;
  q.per_cta = (p.tiles + grid - 1) / grid;
  kern<<<(int)grid, W * kTile + 32 * kMmaWarps, S.total, s>>>(q);
  return cuda_check(cudaGetLastError(), "launch k_decode_tc");
}

template <int NHID, bool FP8>
static nbtc_status launch_tc_t(nbtc_context* ctx, const TcArgs& p, cudaStream_t s) {
  return ctx->tc_groups == 3 ? launch_tc_g<NHID, FP8, 3>(ctx, p, s) : launch_tc_g<NHID, FP8, 4>(ctx, p, s);
}

nbtc_status launch_decode_tc(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, int precision,
                             const void* packed, cudaStream_t s) {
  int nhid;
  nbtc_status st = tc_shape(mlp, nhid);
  if (st) return st;
  if (!packed || !aligned(packed, 16)) return fail(NBTC_ERR_INVALID_ARG, "packed MLP NULL or not 16-byte aligned");
  TcArgs p;
  p.d = a;
  p.packed = packed;
  p.nout = mlp->dims[nhid + 1];
  p.tiles = (a.n + kTile - 1) / kTile;
  p.budget = ctx->wait_budget > 0 ? ctx->wait_budget : kDefaultWaitBudget;
  bool fp = a.uv == nullptr && (a.grid_w % kTile) == 0;
  for (int k = 0; k < 4; ++k) fp = fp && a.lv[k].w <= a.grid_w;
  p.footprint = fp ? 1 : 0;
  p.tiles_per_row = fp ? a.grid_w / kTile : 0;
  if (p.tiles >= (int64_t)1 << 31) return fail(NBTC_ERR_UNSUPPORTED, "more than 2^31 tiles");
  const bool f8 = precision == NBTC_FP8_E4M3;
  if (nhid == 1) return f8 ? launch_tc_t<1, true>(ctx, p, s) : launch_tc_t<1, false>(ctx, p, s);
  if (nhid == 2) return f8 ? launch_tc_t<2, true>(ctx, p, s) : launch_tc_t<2, false>(ctx, p, s);
  return f8 ? launch_tc_t<3, true>(ctx, p, s) : launch_tc_t<3, false>(ctx, p, s);
}

}  // namespace nbtc
