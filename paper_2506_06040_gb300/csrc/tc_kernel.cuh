// The tensor-core decode kernel (template; instantiated in tc_h*_*.cu).
//
// FP16 or FP8 E4M3 operands -- single or split into hi + lo pairs (three
// products per layer) -- FP32 accumulation in TMEM, FP16 output (FP32 for the
// FP32-accurate split form): the GB300 counterpart of the paper's
// cooperative-vector MLP (Sec. 4, "Neural inference in G-Buffer pass"); each
// layer of a 128-texel tile is one chain of tcgen05.mma with M = 128 texels,
// N = layer width, weights resident in shared memory.
//
// Persistent, warp-specialised CTA (one per SM): W warpgroups of 128 threads
// (one thread per tile row) compute features and run the epilogues, and
// W warps (one per warpgroup) issue the MMAs.  Each warpgroup owns NSL tile
// slots.  With TA (the default) a slot is TMEM only -- its accumulator and the
// next layer's A operand, which the epilogue writes back with tcgen05.st and
// the MMAs read from TMEM -- one slot per warpgroup.  Without TA the A operands
// are shared-memory tiles and a warpgroup with two slots alternates between
// them, so one slot's SIMT work overlaps the other slot's MMAs.  The CTA walks
// "chunks" -- runs of tiles of one material -- and reloads the packed MLP only
// when the material changes.
#pragma once

#include <cstring>

#include "features.cuh"
#include "host.h"
#include "sm100.cuh"
#include "tc.cuh"

namespace nbtc {

using namespace sm100;

// Tile numbering.  Each CTA owns a contiguous range of tile numbers; in
// row-footprint mode consecutive numbers run down a column of 128-texel tiles
// (number -> row = T % H, column block = T / H), so the consecutive tiles a
// warpgroup decodes are consecutive rows of one column strip (the feature
// stage's column cache relies on this).  Returns the first output texel of tile T.
__device__ __forceinline__ int64_t tile_first_texel(const DecodeArgs& d, const FastDiv& hdiv, bool footprint,
                                                    int64_t T) {
  if (!footprint) return T * 128;
  const uint32_t t = (uint32_t)T;
  const uint32_t col = fastdiv(t, hdiv), row = t - col * (uint32_t)d.grid_h;
  return (int64_t)row * d.grid_w + (int64_t)col * 128;
}

// Frame pixel decoded by row `gt` of tile `T` of chunk `c` (-1: none).  A
// uniform tile may hold pixels without a material: those are not decoded.
__device__ __forceinline__ int64_t frame_pixel(const TcArgs& p, const WorkChunk& c, int64_t T, int gt) {
  if (c.kind == kChunkUniform) {
    const int ft = __ldg(p.ulist + c.first + T);
    const int ty = ft / p.tiles_x, tx = ft - ty * p.tiles_x;
    const int r = gt / p.tile_w;
    int64_t px = (int64_t)(ty * p.tile_h + r) * p.frame_w + tx * p.tile_w + (gt - r * p.tile_w);
    NBTC_CHECK_INDEX(px, p.frame_pixels, p.d.status);
    return __ldg(p.fmat + px) == c.mat ? px : -1;
  }
  int64_t px = __ldg(p.plist + (c.first + T) * 128 + gt);
  if (px >= 0) NBTC_CHECK_INDEX(px, p.frame_pixels, p.d.status);
  return px;
}

// Shared-memory plan: the packed MLP image, the ones tile, the per-warp output
// staging and the barriers; with shared-memory A operands (not TA) also, per
// slot, A0 (128 x K operand of layer 1) and Ah (128 x 64 operand of later
// layers; split forms: hi tile then lo tile) -- the FP16 split form lays A0
// over the hi tile (A0 is consumed before the first hidden epilogue writes Ah).
struct TcSmem {
  int image;       // packed MLP (rounded to 1 KB)
  int ones;        // 128 x 16 FP16 tile of ones in column 0 (split: columns 0 and 1)
  int slots;       // first slot
  int slot;        // bytes per slot
  int a0, ah;      // offsets inside a slot
  int ah_lo;       // split forms: lo tile of Ah, from ah
  int stage;       // per-warp output staging
  int bars;        // D-ready[NS], weight barrier, MMA-warp drain[W] (room for 2 NS + 1)
  int tslot;       // TMEM address slot
  int work;        // TcWork
  int total;
};

__host__ __device__ inline TcSmem tc_smem(const TcLayout& L, int W, int NSL, bool ta = false) {
  TcSmem s;
  const int NS = W * NSL;
  s.image = (L.bytes() + 1023) & ~1023;
  s.ones = s.image;
  s.slots = s.ones + 4096;
  if (L.f16split()) {
    s.a0 = 0;
    s.ah = 0;
    s.ah_lo = 16384;
    s.slot = ta ? 0 : 32768;  // A operands in TMEM: no slot buffers
  } else {
    s.a0 = 0;
    s.ah = 4096;
    s.ah_lo = 8192;   // FP8 split: 128 x 64 E4M3 hi, then lo
    s.slot = ta ? 0 : 4096 + 16384;  // A operands in TMEM: no slot buffers
  }
  s.stage = s.slots + NS * s.slot;
  s.bars = s.stage + W * 4 * stage_bytes(L.form);
  s.tslot = s.bars + (2 * NS + 1) * 8;
  s.work = (s.tslot + 16 + 15) & ~15;
  s.total = s.work + (int)((sizeof(TcWork) + 15) & ~(size_t)15) + 1024 /* alignment slack */;
  return s;
}

// Warp-specialised persistent kernel: W warpgroups (4 warps, one thread per
// tile row) compute features and epilogues; warp 4W + g issues the MMAs of
// warpgroup g.  Each warpgroup owns NSL tile slots (TMEM columns + A buffers);
// with two it alternates between them, so one slot's epilogue runs while the
// other slot's MMAs run.  Inside a chunk, warpgroup g takes the g-th of W
// contiguous tile ranges, its slots alternating over it.
//
// Hand-offs:
//   A-ready[q]  named barrier (warpgroup: bar.arrive, its MMA warp: bar.sync,
//               160 threads): slot q's A operand for its next layer is in smem
//               and its previous accumulator has been read out of TMEM
//   D-ready[q]  mbarrier (tcgen05.commit; bounded waits): that layer's
//               accumulator is in TMEM
// Every thread keeps its whole schedule whatever happens -- after a timed-out
// wait it stops waiting but still makes every arrival -- so both barrier kinds
// always complete and the kernel always terminates.
// MODE kModeSingle: one material whose views are kernel parameters; kModeBatch:
// chunks of many materials (and frame tiles) whose views live in shared memory.
template <int NHID, int FORM, int W, int MODE, int NSL, bool TA = false>
__global__ void __launch_bounds__(W * 128 + 32 * W, 1) k_decode_tc(TcArgs p) {
  constexpr TcLayout L{NHID, FORM};
  constexpr bool FP8 = FORM == kF8 || FORM == kF8Split;
  constexpr bool F16S = FORM == kF16Split || FORM == kF32Split;  // split FP16 operands
  constexpr bool SPLIT = F16S || FORM == kF8Split;
  constexpr bool OUT32 = FORM == kF32Split;                      // FP32 output
  constexpr int kSlots = NSL;
  constexpr int NS = W * kSlots;
  // TMEM columns: the slots' FP32 accumulators first (64 columns each, on
  // 64-column boundaries); with TA then every slot's A operand -- one part of a
  // hidden layer's 64 activations is 32 columns of FP16 pairs or 16 of E4M3
  // quads; split forms hold the hi part, then the lo part -- and, for the plain
  // FP16 form, an 8-column tile of ones (the bias products' A; the split forms
  // read the shared-memory ones tile)
  constexpr uint32_t kApart = FP8 ? kHid / 4 : kHid / 2;
  constexpr uint32_t kAcols = TA ? (SPLIT ? 2 : 1) * kApart : 0;
  constexpr bool kOnesT = TA && FORM == kF16;
  constexpr uint32_t kOnesCol = NS * (kHid + kAcols);
  constexpr uint32_t kUsedCols = NS * (kHid + kAcols) + (kOnesT ? 8 : 0);
  constexpr uint32_t kTmemCols = kUsedCols <= 256 ? 256 : 512;
  static_assert(kUsedCols <= 512, "TMEM holds at most 512 columns");
  auto a_col = [](int q) { return (uint32_t)(NS * kHid) + (uint32_t)q * kAcols; };  // TA: slot q's A (hi)
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned base, formed by pointer arithmetic on the shared array so
  // accesses through it compile to shared-memory loads (not generic ones)
  unsigned char* smem = smem_raw + ((1024u - (uint32_t)(reinterpret_cast<uintptr_t>(smem_raw) & 1023u)) & 1023u);
  const TcSmem S = tc_smem(L, W, NSL, TA);
  const uint32_t sbase = smem_u32(smem);
  const int tid = threadIdx.x;
  const int warp = tid / 32, lane = tid % 32;
  const uint32_t dbar0 = sbase + S.bars, wbar = dbar0 + NS * 8;
  // named barriers: 0 = __syncthreads, 1 + W + q = A-ready of slot q; with TA
  // (one slot per warpgroup) 1 + q = D-ready of slot q
  static_assert(1 + W + NS <= 16, "named barrier ids");
  static_assert(!TA || NS <= W, "TMEM operands: one slot per warpgroup");
  auto bar_a = [](int q) { return 1 + W + q; };
  auto bar_d = [](int q) { return 1 + q; };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S.tslot);
  TcWork& work = *reinterpret_cast<TcWork*>(smem + S.work);
  int* status = p.d.status;

  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) mbar_init(dbar0 + q * 8, 1);
    mbar_init(wbar, 1);
    for (int m = 0; m < W; ++m) mbar_init(wbar + 8 + m * 8, 1);  // drain barriers
    fence_mbar_init();
    work.m.packed = nullptr;
    work.c.mat = -1;
  }
  if (!FP8 && tid < kTile) {  // ones tile: column 0 (split: columns 0 and 1) = 1.0 (FP16), rest 0
    sts128(sbase + S.ones + off_interleave(tid, 0), SPLIT ? 0x3C003C00u : 0x3C00u, 0u, 0u, 0u);
    sts128(sbase + S.ones + off_interleave(tid, 16), 0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  if constexpr (kOnesT) {
    // element k = 0 of every row is 1.0 (FP16), the rest 0; warp w < 4 writes
    // the rows of its lane quarter
    if (warp < 4) {
      const uint32_t ones[8] = {0x3C00u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
      tmem_st8(tmem_base + kOnesCol + ((uint32_t)(32 * warp) << 16), ones);
      tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  bool failed = false;
  uint32_t wph = 0;  // phase of the weight barrier

  // slot state that lives across chunks (mbarrier phases)
  uint32_t dph[kSlots] = {};
  bool first_chunk = true;

  for (;;) {
    // ---- take the next chunk (thread 0), load its material's MLP if it changed
    if (tid == 0) {
      int valid = 0, reload = 0;
      if (MODE == kModeSingle) {
        if (first_chunk) {
          const int64_t b = (int64_t)blockIdx.x * p.per_cta;
          const int64_t e = b + p.per_cta < p.tiles ? b + p.per_cta : p.tiles;
          work.m.d = p.d;
          work.m.packed = p.packed;
          work.m.nout = p.nout;
          work.c.mat = 0;
          work.c.kind = kChunkGrid;
          work.c.first = b;
          work.c.count = (int)(e > b ? e - b : 0);
          valid = e > b;
          reload = 1;
        }
      } else {
        const int c = atomicAdd(p.chunk_counter, 1);
        if (c < *p.nchunks_dev) {
          const WorkChunk ch = p.chunks[c];
          reload = ch.mat != work.c.mat;
          if (reload) work.m = p.mats[ch.mat];
          work.c = ch;
          valid = 1;
        }
      }
      if (valid && reload) {
        mbar_expect_tx(wbar, (uint32_t)L.bytes());
        bulk_g2s(sbase, work.m.packed, (uint32_t)L.bytes(), wbar);
      }
      work.valid = valid;
      work.reload = reload;
    }
    __syncthreads();
    first_chunk = false;
    if (!work.valid) break;
    if (work.reload) {
      // always waited (fixed budget), also after a timed-out D-ready wait: the
      // copy must land before the MMAs read the image and before the CTA exits
      if (!mbar_wait_bounded(wbar, wph, kDrainBudget)) failed = true;
      wph ^= 1u;
    }
    failed = __syncthreads_or(failed);
    const bool grid_chunk = work.c.kind == kChunkGrid;
    const bool footprint = MODE == kModeSingle ? p.footprint != 0 : grid_chunk;
    const int64_t range_end = work.c.count;   // tiles are numbered 0 .. count-1 inside the chunk

    // Schedule.  Warpgroup g decodes the contiguous tile range [g_begin, g_end)
    // of the chunk in rounds of two tiles (slot 0: g_begin + 2i, slot 1:
    // g_begin + 2i + 1); in row-footprint mode these are consecutive rows of one
    // column strip.  Within a round both slots advance one layer per stage, slot
    // 0 first; a slot's next tile starts (features -> A0) right after its output
    // epilogue.  The warpgroup and its MMA warp walk this same schedule, so the
    // hand-offs always pair up.
    const int64_t per_wg = (range_end + W - 1) / W;

    if (warp >= 4 * W) {
      // ---------------------------------------------------------- MMA warps
      // MMA warp m serves warpgroup m: it blocks in the hardware barrier (no
      // polling) until the warpgroup has handed a slot over, then lane 0 issues
      // that layer's MMAs and commits them to the slot's D-ready mbarrier.
      // Descriptors are built once; per MMA only the 32-bit low word advances.
      const int m = warp - 4 * W;
      constexpr uint32_t ID_HID = idesc(0, kTile, kHid);
      constexpr uint32_t ID_OUT = idesc(0, kTile, kOutPad);
      // high words: SBO, version, swizzle; low words: start address, LBO
      const uint32_t hi_int = (uint32_t)(smem_desc(0, 128, 256, kSwzNone) >> 32);
      const uint32_t hi_a0 = (uint32_t)(smem_desc(0, 128, 8 * L.a0_row(), kSwzNone) >> 32);
      const uint32_t hi_w1 = (uint32_t)(smem_desc(0, 128, 8 * L.w1_row(), kSwzNone) >> 32);
      const uint32_t hi_w = FP8 ? (uint32_t)(smem_desc(0, 16, 512, kSwz64) >> 32)
                                : (uint32_t)(smem_desc(0, 16, 1024, kSwz128) >> 32);
      auto lo = [](uint32_t addr, uint32_t lbo) { return (uint32_t)smem_desc(addr, lbo, 0, 0); };
      auto dsc = [](uint32_t hi, uint32_t lo) { return ((uint64_t)hi << 32) | lo; };
      const uint32_t lo_w1 = lo(sbase + L.off_w1(), 128);
      const uint32_t lo_ones = lo(sbase + S.ones, 128);
      const int64_t g_begin = min((int64_t)m * per_wg, range_end);
      const int64_t g_end = min(g_begin + per_wg, range_end);
      for (int64_t base = g_begin; base < g_end; base += kSlots) {
        const bool two = base + 1 < g_end;
#pragma unroll
        for (int l = 0; l <= NHID; ++l) {
#pragma unroll
          for (int s = 0; s < kSlots; ++s) {
            if (s == 1 && !two) break;
            const int q = m * kSlots + s;
            named_bar_sync(bar_a(q), kTile + 32);
            if (lane == 0) {
              tc_fence_after();
              const uint32_t d = tmem_base + (uint32_t)q * kHid;
              const uint32_t slot = sbase + S.slots + q * S.slot;
              if constexpr (TA) {
                // A from TMEM (8 columns per product: K = 16 FP16 or 32 E4M3),
                // B from shared memory; the FP16 bias product's A is the ones tile
                const uint32_t ah = tmem_base + a_col(q), al = ah + kApart;
                if constexpr (FP8) {
                  if (l == 0) {
                    if constexpr (SPLIT) {
                      mma_f8_ts(d, ah, dsc(hi_w1, lo_w1), ID_HID, 0);       // [hi x | lo x] . hi W
                      mma_f8_ts(d, ah, dsc(hi_w1, lo_w1 + 16), ID_HID, 1);  // [hi x | lo x] . [lo W | 0]
                    } else {
                      mma_f8_ts(d, ah, dsc(hi_w1, lo_w1), ID_HID, 0);
                    }
                  } else {
                    const bool last = l == NHID;
                    const uint32_t id = last ? ID_OUT : ID_HID;
                    const uint32_t lo_b = lo(sbase + (last ? L.off_wo() : L.off_wh(l - 1)), 16);
                    const uint32_t db = (uint32_t)(last ? L.wo_part() : L.wh_part()) >> 4;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                      mma_f8_ts(d, ah + 8 * kk, dsc(hi_w, lo_b + 2 * kk), id, kk > 0);
                      if constexpr (SPLIT) {
                        mma_f8_ts(d, al + 8 * kk, dsc(hi_w, lo_b + 2 * kk), id, 1);
                        mma_f8_ts(d, ah + 8 * kk, dsc(hi_w, lo_b + db + 2 * kk), id, 1);
                      }
                    }
                  }
                } else if (l == 0) {
                  if constexpr (F16S) {
                    // A0: hi [x 1 000] in the 8 columns at ah, lo [x 1 000] at al
                    mma_f16_ts(d, ah, dsc(hi_w1, lo_w1), ID_HID, 0);       // hi x . hi W + hi b
                    mma_f16_ts(d, al, dsc(hi_w1, lo_w1 + 16), ID_HID, 1);  // lo x . hi W + lo b
                    mma_f16_ts(d, ah, dsc(hi_w1, lo_w1 + 32), ID_HID, 1);  // hi x . lo W
                  } else {
                    mma_f16_ts(d, ah, dsc(hi_w1, lo_w1), ID_HID, 0);       // [x 1 0 0 0] . [W b 0 0 0]
                  }
                } else {
                  const bool last = l == NHID;
                  const uint32_t id = last ? ID_OUT : ID_HID;
                  const uint32_t lo_b = lo(sbase + (last ? L.off_wo() : L.off_wh(l - 1)), 16);
                  const uint32_t lo_bt = lo(sbase + (last ? L.off_bto() : L.off_bth(l - 1)), 128);
                  const uint32_t db = (uint32_t)(last ? L.wo_part() : L.wh_part()) >> 4;  // lo W, 16-byte units
                  if constexpr (kOnesT)
                    mma_f16_ts(d, tmem_base + kOnesCol, dsc(hi_int, lo_bt), id, 0);
                  else
                    mma_f16(d, dsc(hi_int, lo_ones), dsc(hi_int, lo_bt), id, 0);
#pragma unroll
                  for (int kk = 0; kk < 4; ++kk) {
                    mma_f16_ts(d, ah + 8 * kk, dsc(hi_w, lo_b + 2 * kk), id, 1);
                    if constexpr (F16S) {
                      mma_f16_ts(d, al + 8 * kk, dsc(hi_w, lo_b + 2 * kk), id, 1);
                      mma_f16_ts(d, ah + 8 * kk, dsc(hi_w, lo_b + db + 2 * kk), id, 1);
                    }
                  }
                }
              } else if (l == 0) {
                // K chunks of 32 bytes (16 FP16 / 32 E4M3), 256 bytes apart in
                // the no-swizzle layout
                const uint32_t la = lo(slot + S.a0, 128);
                if constexpr (F16S) {
                  mma_f16(d, dsc(hi_a0, la), dsc(hi_w1, lo_w1), ID_HID, 0);                // hi x . hi W + hi b
                  mma_f16(d, dsc(hi_a0, la + 16), dsc(hi_w1, lo_w1 + 16), ID_HID, 1);      // lo x . hi W + lo b
                  mma_f16(d, dsc(hi_a0, la), dsc(hi_w1, lo_w1 + 32), ID_HID, 1);           // hi x . lo W
                } else if constexpr (FORM == kF8Split) {
                  mma_f8(d, dsc(hi_a0, la), dsc(hi_w1, lo_w1), ID_HID, 0);                 // [hi x | lo x] . hi W
                  mma_f8(d, dsc(hi_a0, la), dsc(hi_w1, lo_w1 + 16), ID_HID, 1);            // [hi x | lo x] . [lo W | 0]
                } else if constexpr (FP8) {
                  mma_f8(d, dsc(hi_int, la), dsc(hi_int, lo_w1), ID_HID, 0);
                } else {
                  mma_f16(d, dsc(hi_int, la), dsc(hi_int, lo_w1), ID_HID, 0);
                }
              } else {
                const bool last = l == NHID;
                const uint32_t id = last ? ID_OUT : ID_HID;
                const uint32_t lo_a = lo(slot + S.ah, 16);
                const uint32_t lo_b = lo(sbase + (last ? L.off_wo() : L.off_wh(l - 1)), 16);
                // lo halves of A and W (split forms), in 16-byte units
                const uint32_t da = (uint32_t)S.ah_lo >> 4;
                const uint32_t db = (uint32_t)(last ? L.wo_part() : L.wh_part()) >> 4;
                if constexpr (FP8) {
#pragma unroll
                  for (int kk = 0; kk < 2; ++kk) {
                    mma_f8(d, dsc(hi_w, lo_a + 2 * kk), dsc(hi_w, lo_b + 2 * kk), id, kk > 0);
                    if constexpr (SPLIT) {
                      mma_f8(d, dsc(hi_w, lo_a + da + 2 * kk), dsc(hi_w, lo_b + 2 * kk), id, 1);
                      mma_f8(d, dsc(hi_w, lo_a + 2 * kk), dsc(hi_w, lo_b + db + 2 * kk), id, 1);
                    }
                  }
                } else {
                  const uint32_t lo_bt = lo(sbase + (last ? L.off_bto() : L.off_bth(l - 1)), 128);
                  mma_f16(d, dsc(hi_int, lo_ones), dsc(hi_int, lo_bt), id, 0);
#pragma unroll
                  for (int kk = 0; kk < 4; ++kk) {
                    mma_f16(d, dsc(hi_w, lo_a + 2 * kk), dsc(hi_w, lo_b + 2 * kk), id, 1);
                    if constexpr (SPLIT) {
                      mma_f16(d, dsc(hi_w, lo_a + da + 2 * kk), dsc(hi_w, lo_b + 2 * kk), id, 1);
                      mma_f16(d, dsc(hi_w, lo_a + 2 * kk), dsc(hi_w, lo_b + db + 2 * kk), id, 1);
                    }
                  }
                }
              }
              mma_commit(dbar0 + q * 8);
            }
            __syncwarp();  // converged before the next (aligned) barrier
            if constexpr (TA) {
              // this warp waits for the layer's products (bounded) and then
              // releases the warpgroup through a hardware barrier, so the
              // warpgroup's 128 threads sleep instead of polling the mbarrier
              if (!mbar_wait_bounded(dbar0 + q * 8, dph[s], p.budget)) {
                failed = true;
                mbar_wait_bounded(dbar0 + q * 8, dph[s], kDrainBudget);
              }
              dph[s] ^= 1u;
              tc_fence_before();
              __syncwarp();
              named_bar_arrive(bar_d(q), kTile + 32);
            }
          }
        }
      }
    } else {
      // ---------------------------------------------------------- warpgroups
      const int wg = warp / 4, wq = warp & 3;
      const int gt = tid % kTile;
      const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
      const uint32_t stage_s = sbase + S.stage + warp * stage_bytes(FORM);
      const float* bias = reinterpret_cast<const float*>(smem + L.off_bias());
      const float* alpha = reinterpret_cast<const float*>(smem + L.off_alpha());
      const DecodeArgs& D = MODE == kModeSingle ? p.d : work.m.d;
      const FastDiv& hdiv = MODE == kModeSingle ? p.hdiv : work.m.hdiv;
      const int nout = work.m.nout;
      const int64_t g_begin = min((int64_t)wg * per_wg, range_end);
      const int64_t g_end = min(g_begin + per_wg, range_end);
      StripCache cache;
      strip_reset(cache);
      uint32_t next_a0[16];  // TA: the next tile's A0, computed during the output layer's MMAs

      // features of tile T (chunk numbering) into slot s's A0, then A-ready
      // the 12 features of this thread's texel (or frame pixel) of tile T
      auto tile_features = [&](int64_t T, float (&f)[12]) {
        if (MODE == kModeSingle || grid_chunk) {
          if (footprint) {
            // tile number = column block x H + row; each warp decodes its own
            // 32 texels' latent columns and shares them by shuffles
            const uint32_t t = (uint32_t)(work.c.first + T), H = (uint32_t)D.grid_h;
            const uint32_t cb = fastdiv(t, hdiv);
            warp_strip_features(D, (int)(t - cb * H), (int)cb * kTile + 32 * wq, lane, cache, f);
          } else {
            const int64_t tex = (work.c.first + T) * kTile + gt;
            direct_features(D, tex < D.n ? tex : D.n - 1, f);
          }
        } else {
          const int64_t px = frame_pixel(p, work.c, T, gt);
          const int64_t pq = px < 0 ? 0 : px;
          const float2 uv = __ldg(reinterpret_cast<const float2*>(p.fuv) + pq);
          if (p.fduv)
            aniso_features(work.m, uv.x, uv.y, __ldg(reinterpret_cast<const float4*>(p.fduv) + pq), __ldg(p.flod + pq),
                           p.max_aniso, f);
          else
            trilinear_features(work.m, uv.x, uv.y, __ldg(p.flod + pq), f);
        }
      };
      // TA: a tile's A0 row as it goes into TMEM (8 columns; split FP16: hi in
      // av[0..7], lo in av[8..15]), and its store + A-ready
      auto pack_a0 = [&](const float (&f)[12], uint32_t (&av)[16]) {
        if constexpr (FP8) {
          // A0 row of 32 E4M3: [x(12) 0 x 20], split: [hi x(12) 0000 | lo x(12) 0000]
          const float is = alpha[NHID + 1];  // 1 / input scale
#pragma unroll
          for (int i = 0; i < 8; ++i) av[i] = 0u;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            if constexpr (SPLIT) {
              uint16_t h0, r0, h1, r1;
              split_e4m3x2(cvt_f16x2(f[4 * i] * is, f[4 * i + 1] * is), h0, r0);
              split_e4m3x2(cvt_f16x2(f[4 * i + 2] * is, f[4 * i + 3] * is), h1, r1);
              av[i] = (uint32_t)h0 | ((uint32_t)h1 << 16);
              av[4 + i] = (uint32_t)r0 | ((uint32_t)r1 << 16);
            } else {
              av[i] = (uint32_t)cvt_e4m3x2(f[4 * i] * is, f[4 * i + 1] * is) |
                      ((uint32_t)cvt_e4m3x2(f[4 * i + 2] * is, f[4 * i + 3] * is) << 16);
            }
          }
        } else if constexpr (F16S) {
#pragma unroll
          for (int i = 0; i < 6; ++i) split_f16x2(f[2 * i], f[2 * i + 1], av[i], av[8 + i]);
          av[6] = av[14] = 0x3C00u;  // k = 12: 1.0 for hi(b) / lo(b)
          av[7] = av[15] = 0u;
        } else {
#pragma unroll
          for (int i = 0; i < 6; ++i) av[i] = cvt_f16x2(f[2 * i], f[2 * i + 1]);
          av[6] = 0x3C00u;  // k = 12: 1.0 for the bias
          av[7] = 0u;
        }
      };
      auto store_a0 = [&](int s, const uint32_t (&av)[16]) {
        const int q = wg * kSlots + s;
        const uint32_t ta = tmem_base + a_col(q) + lane_off;  // the slot's A (hi) columns
        tmem_st8(ta, av);
        if constexpr (F16S) tmem_st8(ta + kApart, av + 8);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        named_bar_arrive(bar_a(q), kTile + 32);
      };

      // features of tile T (chunk numbering) into slot s's A0, then A-ready
      auto start_tile = [&](int s, int64_t T) {
        const int q = wg * kSlots + s;
        const uint32_t a0 = sbase + S.slots + q * S.slot + S.a0;
        float f[12];
        tile_features(T, f);
        if constexpr (TA) {
          uint32_t av[16];
          pack_a0(f, av);
          store_a0(s, av);
          return;
        } else if constexpr (FORM == kF16) {
          sts128(a0 + off_interleave(gt, 0), cvt_f16x2(f[0], f[1]), cvt_f16x2(f[2], f[3]), cvt_f16x2(f[4], f[5]),
                 cvt_f16x2(f[6], f[7]));
          sts128(a0 + off_interleave(gt, 16), cvt_f16x2(f[8], f[9]), cvt_f16x2(f[10], f[11]),
                 0x3C00u /* k = 12: 1.0 for the bias */, 0u);
        } else if constexpr (F16S) {
          uint32_t h[6], r[6];
#pragma unroll
          for (int i = 0; i < 6; ++i) split_f16x2(f[2 * i], f[2 * i + 1], h[i], r[i]);
          const int R = L.a0_row();
          sts128(a0 + off_ilv(gt, 0, R), h[0], h[1], h[2], h[3]);
          sts128(a0 + off_ilv(gt, 16, R), h[4], h[5], 0x3C00u /* k = 12: 1.0 for hi(b) */, 0u);
          sts128(a0 + off_ilv(gt, 32, R), r[0], r[1], r[2], r[3]);
          sts128(a0 + off_ilv(gt, 48, R), r[4], r[5], 0x3C00u /* k = 28: 1.0 for lo(b) */, 0u);
        } else if constexpr (FORM == kF8) {
          const float is = alpha[NHID + 1];  // 1 / input scale
          uint32_t w[3];
#pragma unroll
          for (int i = 0; i < 3; ++i)
            w[i] = (uint32_t)cvt_e4m3x2(f[4 * i] * is, f[4 * i + 1] * is) |
                   ((uint32_t)cvt_e4m3x2(f[4 * i + 2] * is, f[4 * i + 3] * is) << 16);
          sts128(a0 + off_interleave(gt, 0), w[0], w[1], w[2], 0u);
          sts128(a0 + off_interleave(gt, 16), 0u, 0u, 0u, 0u);
        } else {
          const float is = alpha[NHID + 1];  // 1 / input scale
          uint32_t h[3], r[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            uint16_t h0, r0, h1, r1;
            split_e4m3x2(cvt_f16x2(f[4 * i] * is, f[4 * i + 1] * is), h0, r0);
            split_e4m3x2(cvt_f16x2(f[4 * i + 2] * is, f[4 * i + 3] * is), h1, r1);
            h[i] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            r[i] = (uint32_t)r0 | ((uint32_t)r1 << 16);
          }
          sts128(a0 + off_interleave(gt, 0), h[0], h[1], h[2], 0u);
          sts128(a0 + off_interleave(gt, 16), r[0], r[1], r[2], 0u);
        }
        fence_proxy_async_smem();
        __syncwarp();
        named_bar_arrive(bar_a(q), kTile + 32);
      };

      // hidden epilogue of layer l of slot s: accumulator -> (bias,) ReLU ->
      // narrow -> Ah, then A-ready
      auto hidden_epilogue = [&](int s, int l) {
        const int q = wg * kSlots + s;
        const uint32_t taddr = tmem_base + (uint32_t)q * kHid + lane_off;
        const uint32_t aaddr = tmem_base + a_col(q) + lane_off;  // TA: the slot's A (hi) columns
        if constexpr (TA && FP8) {
          // scale and bias (packed FP32 FMAs), ReLU -> E4M3 quads (split: hi and
          // lo quads) -> the slot's A columns (8 per 32 activations)
          const float alp = alpha[l];
          const float* b = bias + l * kHid;
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            uint32_t r[32], w[8], wl[8];
            tmem_ld32_wait(taddr + 32 * part, r);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const int j = 4 * c;
              const float4 bb = *reinterpret_cast<const float4*>(b + 32 * part + j);
              const float2 v0 = __ffma2_rn(make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])),
                                           make_float2(alp, alp), make_float2(bb.x, bb.y));
              const float2 v1 = __ffma2_rn(make_float2(__uint_as_float(r[j + 2]), __uint_as_float(r[j + 3])),
                                           make_float2(alp, alp), make_float2(bb.z, bb.w));
              if constexpr (SPLIT) {
                uint16_t h0, r0, h1, r1;
                split_e4m3x2(cvt_relu_f16x2(v0.x, v0.y), h0, r0);
                split_e4m3x2(cvt_relu_f16x2(v1.x, v1.y), h1, r1);
                w[c] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                wl[c] = (uint32_t)r0 | ((uint32_t)r1 << 16);
              } else {
                w[c] = (uint32_t)cvt_relu_e4m3x2(v0.x, v0.y) | ((uint32_t)cvt_relu_e4m3x2(v1.x, v1.y) << 16);
              }
            }
            tmem_st8(aaddr + 8 * part, w);
            if constexpr (SPLIT) tmem_st8(aaddr + kApart + 8 * part, wl);
          }
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          named_bar_arrive(bar_a(q), kTile + 32);
          return;
        } else if constexpr (TA) {
          // ReLU -> FP16 pairs (split: hi and lo pairs) -> the slot's A columns
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            uint32_t r[32], h[16];
            tmem_ld32_wait(taddr + 32 * part, r);
            if constexpr (F16S) {
              uint32_t lw[16];
#pragma unroll
              for (int j = 0; j < 16; ++j)
                split_relu_f16x2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]), h[j], lw[j]);
              tmem_st16(aaddr + kApart + 16 * part, lw);
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                h[j] = cvt_relu_f16x2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
            }
            tmem_st16(aaddr + 16 * part, h);
          }
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          named_bar_arrive(bar_a(q), kTile + 32);
          return;
        }
        const uint32_t ah = sbase + S.slots + q * S.slot + S.ah;
        const float alp = alpha[l];
        const float* b = bias + l * kHid;
        // after a timed-out wait the loads still run (they cannot fault) and the
        // results are discarded with the status
        // the accumulator row comes out of TMEM in two 32-column parts, one wait
        // each (measured faster than one 64-column load and one wait)
        constexpr int kParts = 2;
        constexpr int kPc = kHid / kParts;
#pragma unroll
        for (int part = 0; part < kParts; ++part) {
          uint32_t r[kPc];
          tmem_ld32_wait(taddr + kPc * part, r);
          if constexpr (FORM == kF16) {
#pragma unroll
            for (int c = 0; c < kPc / 8; ++c) {
              const int j = 8 * c;
              sts128(ah + off_sw128(gt, 16 * (part * (kPc / 8) + c)),
                     cvt_relu_f16x2(__uint_as_float(r[j + 0]), __uint_as_float(r[j + 1])),
                     cvt_relu_f16x2(__uint_as_float(r[j + 2]), __uint_as_float(r[j + 3])),
                     cvt_relu_f16x2(__uint_as_float(r[j + 4]), __uint_as_float(r[j + 5])),
                     cvt_relu_f16x2(__uint_as_float(r[j + 6]), __uint_as_float(r[j + 7])));
            }
          } else if constexpr (F16S) {
#pragma unroll
            for (int c = 0; c < kPc / 8; ++c) {
              const int j = 8 * c;
              uint32_t h[4], lw[4];
#pragma unroll
              for (int e = 0; e < 4; ++e)
                split_relu_f16x2(__uint_as_float(r[j + 2 * e]), __uint_as_float(r[j + 2 * e + 1]), h[e], lw[e]);
              const uint32_t o = off_sw128(gt, 16 * (part * (kPc / 8) + c));
              sts128(ah + o, h[0], h[1], h[2], h[3]);
              sts128(ah + S.ah_lo + o, lw[0], lw[1], lw[2], lw[3]);
            }
          } else {
#pragma unroll
            for (int c = 0; c < kPc / 16; ++c) {
              uint32_t w[4], wl[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                // scale and bias as packed FMAs (two IEEE FP32 FMAs each)
                const int j = 16 * c + 4 * e, jj = kPc * part + j;
                const float4 bb = *reinterpret_cast<const float4*>(b + jj);
                const float2 v0 = __ffma2_rn(make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])),
                                             make_float2(alp, alp), make_float2(bb.x, bb.y));
                const float2 v1 = __ffma2_rn(make_float2(__uint_as_float(r[j + 2]), __uint_as_float(r[j + 3])),
                                             make_float2(alp, alp), make_float2(bb.z, bb.w));
                if constexpr (FORM == kF8) {
                  w[e] = (uint32_t)cvt_relu_e4m3x2(v0.x, v0.y) | ((uint32_t)cvt_relu_e4m3x2(v1.x, v1.y) << 16);
                } else {
                  uint16_t h0, r0, h1, r1;
                  split_e4m3x2(cvt_relu_f16x2(v0.x, v0.y), h0, r0);
                  split_e4m3x2(cvt_relu_f16x2(v1.x, v1.y), h1, r1);
                  w[e] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                  wl[e] = (uint32_t)r0 | ((uint32_t)r1 << 16);
                }
              }
              const uint32_t o = off_sw64(gt, 16 * (part * (kPc / 16) + c));
              sts128(ah + o, w[0], w[1], w[2], w[3]);
              if constexpr (SPLIT) sts128(ah + S.ah_lo + o, wl[0], wl[1], wl[2], wl[3]);
            }
          }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncwarp();
        named_bar_arrive(bar_a(q), kTile + 32);
      };

      // output epilogue of slot s, tile T: accumulator -> FP16 -> global
      // (TA, store_next: once the accumulator row is in registers, the next
      // tile's A0 goes into TMEM and its layer-1 MMA may start while this
      // epilogue converts and stores)
      auto output_epilogue = [&](int s, int64_t T, bool store_next) {
        const int q = wg * kSlots + s;
        const uint32_t taddr = tmem_base + (uint32_t)q * kHid + lane_off;
        uint32_t r[16];
        tmem_ld16_wait(taddr, r);
        tc_fence_before();
        if constexpr (TA) {
          if (store_next) store_a0(s, next_a0);
        }
        const float alp = alpha[NHID];
        const float* b = bias + NHID * kHid;
        uint16_t hv[kMaxOut];
        if constexpr (FP8) {
#pragma unroll
          for (int k = 0; k < kMaxOut; k += 2) {
            const float2 v = __ffma2_rn(make_float2(__uint_as_float(r[k]), __uint_as_float(r[k + 1])),
                                        make_float2(alp, alp), *reinterpret_cast<const float2*>(b + k));
            hv[k] = __half_as_ushort(__float2half_rn(v.x));
            hv[k + 1] = __half_as_ushort(__float2half_rn(v.y));
          }
        } else {
#pragma unroll
          for (int k = 0; k < kMaxOut; ++k) hv[k] = __half_as_ushort(__float2half_rn(__uint_as_float(r[k])));
        }
        if constexpr (OUT32) {
          // FP32 output (single-material grids and uv lists): the accumulator as is
          const int64_t t0 = tile_first_texel(D, hdiv, footprint, work.c.first + T);
          const int64_t tex = t0 + gt;
          if (t0 + kTile <= D.n) {
            // the warp's 32 texels x nout floats are contiguous: one bulk copy of
            // 128 nout bytes at a 128-byte multiple of the 16-byte aligned output
            if (lane == 0) bulk_wait_read0();
            __syncwarp();
#pragma unroll
            for (int k = 0; k < kMaxOut; ++k)
              if (k < nout) sts32(stage_s + 4u * (uint32_t)(lane * nout + k), r[k]);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              bulk_s2g(reinterpret_cast<float*>(D.out) + (t0 + 32 * wq) * nout, stage_s, 128u * (uint32_t)nout);
              bulk_commit();
            }
          } else if (tex < D.n) {
            float* o = reinterpret_cast<float*>(D.out) + tex * nout;
#pragma unroll
            for (int k = 0; k < kMaxOut; ++k)
              if (k < nout) o[k] = __uint_as_float(r[k]);
          }
        } else if (MODE == kModeSingle || grid_chunk) {
          const int64_t t0 = tile_first_texel(D, hdiv, footprint, work.c.first + T);
          const int64_t tex = t0 + gt;
          if (t0 + kTile <= D.n) {
            // the warp's 32 texels x nout halves are contiguous in the output:
            // stage them and write them with one bulk copy (64 nout bytes at a
            // 64-byte multiple of the 16-byte aligned output)
            if (lane == 0) bulk_wait_read0();  // the warp's previous bulk copy has read the stage
            __syncwarp();
#pragma unroll
            for (int k = 0; k < kMaxOut; ++k)
              if (k < nout) sts16(stage_s + 2u * (uint32_t)(lane * nout + k), hv[k]);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              bulk_s2g(reinterpret_cast<uint16_t*>(D.out) + (t0 + 32 * wq) * nout, stage_s, 64u * (uint32_t)nout);
              bulk_commit();
            }
          } else if (tex < D.n) {
            uint16_t* o = reinterpret_cast<uint16_t*>(D.out) + tex * nout;
#pragma unroll
            for (int k = 0; k < kMaxOut; ++k)
              if (k < nout) o[k] = hv[k];
          }
        } else {
          const int64_t px = frame_pixel(p, work.c, T, gt);
          if (px >= 0) {
            uint16_t* o = p.fout + px * nout;
#pragma unroll
            for (int k = 0; k < kMaxOut; ++k)
              if (k < nout) o[k] = hv[k];
            if (p.fshade) {  // lighting pass on the pixel's FP16 G-buffer channels
              float y[8];
#pragma unroll
              for (int k = 0; k < 8; ++k) y[k] = __half2float(__ushort_as_half(hv[k]));
              const float3 c = shade_pixel(y, p.light);
              *reinterpret_cast<float4*>(p.fshade + 4 * px) = make_float4(c.x, c.y, c.z, 1.f);
            }
          }
        }
      };

#pragma unroll
      for (int s = 0; s < kSlots; ++s)  // prime each of this warpgroup's own slots
        if (g_begin + s < g_end) start_tile(s, g_begin + s);
      for (int64_t base = g_begin; base < g_end; base += kSlots) {
        const bool two = base + 1 < g_end;
#pragma unroll
        for (int l = 0; l <= NHID; ++l) {
#pragma unroll
          for (int s = 0; s < kSlots; ++s) {
            if (s == 1 && !two) break;
            const int q = wg * kSlots + s;
            // past the budget: record the timeout, then keep waiting (fixed budget)
            // so the warpgroup never runs ahead of its MMA warp -- running ahead
            // would arrive twice on one A-ready named barrier before it completes
            if constexpr (TA) {
              named_bar_sync(bar_d(q), kTile + 32);  // the MMA warp saw the products complete
            } else {
              if (!mbar_wait_bounded(dbar0 + q * 8, dph[s], p.budget)) {
                failed = true;
                mbar_wait_bounded(dbar0 + q * 8, dph[s], kDrainBudget);
              }
              dph[s] ^= 1u;
            }
            failed = __any_sync(0xffffffffu, failed);  // one failure state per warp
            tc_fence_after();
            if (l < NHID) {
              hidden_epilogue(s, l);
              if constexpr (TA) {
                // the next tile's features while the output layer's MMAs run
                // (stored into TMEM once those have read this tile's A)
                if (l == NHID - 1 && base + s + kSlots < g_end) {
                  float f[12];
                  tile_features(base + s + kSlots, f);
                  pack_a0(f, next_a0);
                }
              }
            } else {
              const bool more = base + s + kSlots < g_end;
              output_epilogue(s, base + s, TA && more);
              if constexpr (!TA) {
                if (more) start_tile(s, base + s + kSlots);
              }
            }
          }
        }
      }
    }
    // chunk end: every MMA of this chunk has been consumed; the MLP image and the
    // material view may change
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  // Drain: the issuing lane of each MMA warp commits once more and waits for it
  // (drain budget), so that TMEM is released only after every MMA it issued has
  // completed -- also when a D-ready wait gave up and the warpgroup ran ahead.
  if (warp >= 4 * W && lane == 0) {
    const uint32_t db = wbar + 8 + (warp - 4 * W) * 8;
    mma_commit(db);
    if (!mbar_wait_bounded(db, 0, kDrainBudget)) failed = true;
  }
  if (failed) record_status(status, NBTC_ERR_TIMEOUT);
  bulk_wait0();  // this thread's bulk output copies (if any) are complete
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem_base, kTmemCols);
}


template <int NHID, int FORM, int W, int MODE, int NSL, bool TA = false>
nbtc_status launch_tc_w(const TcArgs& p, int grid, cudaStream_t s) {
  const TcSmem S = tc_smem(TcLayout{NHID, FORM}, W, NSL, TA);
  auto kern = k_decode_tc<NHID, FORM, W, MODE, NSL, TA>;
  nbtc_status st =
      cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S.total), "smem attribute");
  if (st) return st;
  kern<<<grid, W * kTile + 32 * W, S.total, s>>>(p);
  return cuda_check(cudaGetLastError(), "launch k_decode_tc");
}

}  // namespace nbtc
