// Tensor-core training kernel (included by train.cu after the shared training
// definitions): the step's MLP products -- forward, backward and weight
// gradients -- on tcgen05 with split FP16 operands (hi + lo, three products
// per GEMM, FP32 accumulation in TMEM), which keeps FP32-level accuracy.
//
// Two warpgroups per CTA (one thread per sample of a 128-sample tile) and one
// MMA-issuing warp each.  Per tile, six hand-offs (named barrier A-ready ->
// MMAs -> mbarrier D-ready), all operands in shared memory:
//   1  X (features + a ones column)    F1: Z1 = X W1^T + b1               (D)
//   2  H1 = relu(Z1)                    F2: Z2 = H1 W2^T + b2              (D)
//   3  H2 = relu(Z2)                    F3: Y  = H2 W3^T + b3              (D)
//   4  G = dL/dy, unscaled (2 r; L1: sign r)
//                                       B1: dH2 = G W3 (D);  G3 += H2^T G
//   5  dZ2 = dH2 [Z2 > 0]  (over H2)    B2: dH1 = dZ2 W2 (D); G2 += dZ2^T H1, G2b += dZ2^T 1
//   6  dZ1 = dH1 [Z1 > 0]  (over H1)    B3: dX = dZ1 W1 (D);  G1 += dZ1^T X
// then dX (times the loss scale) is scattered into the latent gradients.  The
// weight-gradient products reduce over the tile's samples: their operands are
// the same shared-memory tiles read MN-major (the instruction's transpose
// bits), M = 64 (rows in the first 16 lanes of each warp's TMEM quarter).  The
// G accumulators start afresh each tile (a 128-sample sum); the epilogue adds
// each tile's G to the warpgroup's running FP32 sums, which it keeps in the
// other 16 lanes of each quarter of the same columns -- an accumulator chain
// over all of a warpgroup's samples would lose FP32 accuracy as it grows.  At
// the end the running sums are scaled, the two warpgroups added (with the
// rounding error kept as the compensation) and written as the CTA's partial
// sums.  The loss and db3 use per-thread
// Neumaier sums and a fixed-order CTA reduction, as the SIMT kernel does.
#pragma once

#include "sm100.cuh"

namespace nbtc {

namespace ttc {

// ---- shared-memory plan (bytes from a 1024-aligned base)
// weight images (K-major unless noted; SW32 = 32-byte rows, SW128 = 128-byte rows)
constexpr int oW1H = 0, oW1L = 2048;          // [64 out][16 in] SW32, hi / lo
constexpr int oBT1 = 4096;                    // [64][16] SW32: column 0 hi(b1), 1 lo(b1)
constexpr int oW3TH = 6144, oW3TL = 8192;     // W3^T [64 hidden][16 channel] SW32
constexpr int oONES = 10240;                  // [128][16] SW32: columns 0 and 1 = 1
constexpr int oBT3 = 14336;                   // [16][16] SW32: b3
constexpr int oBT2 = 15360;                   // [64][16] SW32: b2
constexpr int oW2H = 17408, oW2L = 25600;     // [64 out][64 in] SW128
constexpr int oW2TH = 33792, oW2TL = 41984;   // W2^T [64 in][64 out] SW128
constexpr int oW3H = 50176, oW3L = 52224;     // [16 channel][64 in] SW128
constexpr int oW1TH = 54272, oW1TL = 56320;   // W1^T [16 feature][64 hidden] SW128
constexpr int oTiles = 58368;
// per warpgroup
constexpr int kTileBytes = 81920;
constexpr int oXH = 0, oXL = 4096, oDYH = 8192, oDYL = 12288;     // [128][16] SW32
constexpr int oH1H = 16384, oH1L = 32768, oH2H = 49152, oH2L = 65536;  // [128][64] SW128
constexpr int kWG = 2;
constexpr int oBars = oTiles + kWG * kTileBytes;  // D-ready[2], spare[2]
constexpr int oTslot = oBars + 32;
constexpr int kSmem = oTslot + 16 + 1024;
// TMEM columns per warpgroup (base g * 256)
constexpr uint32_t cD = 0, cG2 = 64, cG2b = 128, cG3 = 144, cG1 = 160;

__device__ __forceinline__ uint32_t sw32(int row, int kbyte) {
  return (uint32_t)((row >> 3) * 256 + (row & 7) * 32 + ((((kbyte >> 4) ^ ((row & 7) >> 2)) & 1) << 4) +
                    (kbyte & 15));
}
__device__ __forceinline__ uint32_t sw128(int row, int kbyte) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((kbyte >> 4) ^ (row & 7)) & 7) << 4) + (kbyte & 15));
}
__device__ __forceinline__ void st_half(unsigned char* s, uint32_t off, float v) {
  *reinterpret_cast<__half*>(s + off) = __float2half_rn(v);
}
// hi / lo halves of one FP32 value (hi = RN16(v), lo = RN16(v - hi))
__device__ __forceinline__ void put_split(unsigned char* s, uint32_t oh, uint32_t ol, float v) {
  uint32_t h, l;
  sm100::split_f16x2(v, 0.f, h, l);
  *reinterpret_cast<uint16_t*>(s + oh) = (uint16_t)(h & 0xFFFF);
  *reinterpret_cast<uint16_t*>(s + ol) = (uint16_t)(l & 0xFFFF);
}

}  // namespace ttc

template <bool LV>
__global__ void __launch_bounds__(ttc::kWG * 160, 1) k_train_tc(TrainDev a) {
  using namespace ttc;
  using namespace sm100;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sb = smem_u32(sm);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int C = a.C;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + oTslot);

  // ---- weight images from the FP32 MLP (every CTA builds its own)
  for (int e = tid; e < oTiles / 4; e += blockDim.x) reinterpret_cast<uint32_t*>(sm)[e] = 0u;
  if (warp == 0) {
    tmem_alloc(smem_u32(tslot), 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int g = 0; g < kWG; ++g) mbar_init(sb + oBars + 8 * g, 1);
    fence_mbar_init();
  }
  __syncthreads();
  {
    const float* W1 = a.W;                // [64][12]
    const float* W2 = a.W + kH * kIn;     // [64][64]
    const float* W3 = W2 + kH * kH;       // [C][64]
    const float* b1 = a.B;
    const float* b2 = a.B + kH;
    const float* b3 = a.B + 2 * kH;
    for (int e = tid; e < kH * kIn; e += blockDim.x) {
      const int n = e / kIn, k = e - n * kIn;
      const float w = W1[e];
      put_split(sm, oW1H + sw32(n, 2 * k), oW1L + sw32(n, 2 * k), w);
      put_split(sm, oW1TH + sw128(k, 2 * n), oW1TL + sw128(k, 2 * n), w);
    }
    for (int e = tid; e < kH * kH; e += blockDim.x) {
      const int n = e / kH, k = e - n * kH;
      const float w = W2[e];
      put_split(sm, oW2H + sw128(n, 2 * k), oW2L + sw128(n, 2 * k), w);
      put_split(sm, oW2TH + sw128(k, 2 * n), oW2TL + sw128(k, 2 * n), w);
    }
    for (int e = tid; e < C * kH; e += blockDim.x) {
      const int c = e / kH, k = e - c * kH;
      const float w = W3[e];
      put_split(sm, oW3H + sw128(c, 2 * k), oW3L + sw128(c, 2 * k), w);
      put_split(sm, oW3TH + sw32(k, 2 * c), oW3TL + sw32(k, 2 * c), w);
    }
    for (int e = tid; e < kH; e += blockDim.x) {
      put_split(sm, oBT1 + sw32(e, 0), oBT1 + sw32(e, 2), b1[e]);
      put_split(sm, oBT2 + sw32(e, 0), oBT2 + sw32(e, 2), b2[e]);
    }
    for (int e = tid; e < C; e += blockDim.x) put_split(sm, oBT3 + sw32(e, 0), oBT3 + sw32(e, 2), b3[e]);
    for (int r = tid; r < 128; r += blockDim.x) {
      st_half(sm, oONES + sw32(r, 0), 1.f);
      st_half(sm, oONES + sw32(r, 2), 1.f);
    }
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const int64_t tiles = (a.batch + 127) / 128;
  const int64_t stride = (int64_t)gridDim.x * kWG;
  bool failed = false;

  if (warp >= 4 * kWG) {
    // ------------------------------------------------------------ MMA warps
    const int g = warp - 4 * kWG;
    const uint32_t d = tmem + (uint32_t)(g * 256);
    const uint32_t T0 = sb + oTiles + g * kTileBytes;
    constexpr uint32_t ID128_64 = idesc(0, 128, 64), ID128_16 = idesc(0, 128, 16);
    constexpr uint32_t IDT64_64 = idesc(0, 64, 64) | (1u << 15) | (1u << 16);
    constexpr uint32_t IDT64_16 = idesc(0, 64, 16) | (1u << 15) | (1u << 16);
    auto k32 = [&](uint32_t addr) { return smem_desc(addr, 16, 256, 6); };                    // SW32 K-major, K = 16
    auto k128 = [&](uint32_t addr, int kk) { return smem_desc(addr + 32 * kk, 16, 1024, 2); };  // SW128 K-major chunk
    auto m128 = [&](uint32_t addr, int kk) { return smem_desc(addr + 2048 * kk, 1024, 1024, 2); };  // SW128 MN-major
    auto m32 = [&](uint32_t addr, int kk) { return smem_desc(addr + 512 * kk, 256, 256, 6); };      // SW32 MN-major
    for (int64_t tile = (int64_t)blockIdx.x * kWG + g; tile < tiles; tile += stride) {
#pragma unroll 1
      for (int ph = 1; ph <= 6; ++ph) {
        named_bar_sync(1 + g, 160);
        if (lane == 0) {
          tc_fence_after();
          const uint32_t D = d + cD;
          if (ph == 1) {
            mma_f16(D, k32(sb + oONES), k32(sb + oBT1), ID128_64, 0);
            mma_f16(D, k32(T0 + oXH), k32(sb + oW1H), ID128_64, 1);
            mma_f16(D, k32(T0 + oXL), k32(sb + oW1H), ID128_64, 1);
            mma_f16(D, k32(T0 + oXH), k32(sb + oW1L), ID128_64, 1);
          } else if (ph == 2 || ph == 3) {
            const uint32_t AH = T0 + (ph == 2 ? oH1H : oH2H), AL = T0 + (ph == 2 ? oH1L : oH2L);
            const uint32_t BH = sb + (ph == 2 ? oW2H : oW3H), BL = sb + (ph == 2 ? oW2L : oW3L);
            const uint32_t id = ph == 2 ? ID128_64 : ID128_16;
            mma_f16(D, k32(sb + oONES), k32(sb + (ph == 2 ? oBT2 : oBT3)), id, 0);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              mma_f16(D, k128(AH, kk), k128(BH, kk), id, 1);
              mma_f16(D, k128(AL, kk), k128(BH, kk), id, 1);
              mma_f16(D, k128(AH, kk), k128(BL, kk), id, 1);
            }
          } else if (ph == 4) {
            mma_f16(D, k32(T0 + oDYH), k32(sb + oW3TH), ID128_64, 0);
            mma_f16(D, k32(T0 + oDYL), k32(sb + oW3TH), ID128_64, 1);
            mma_f16(D, k32(T0 + oDYH), k32(sb + oW3TL), ID128_64, 1);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              mma_f16(d + cG3, m128(T0 + oH2H, kk), m32(T0 + oDYH, kk), IDT64_16, kk == 0 ? 0 : 1);
              mma_f16(d + cG3, m128(T0 + oH2L, kk), m32(T0 + oDYH, kk), IDT64_16, 1);
              mma_f16(d + cG3, m128(T0 + oH2H, kk), m32(T0 + oDYL, kk), IDT64_16, 1);
            }
          } else if (ph == 5) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              mma_f16(D, k128(T0 + oH2H, kk), k128(sb + oW2TH, kk), ID128_64, kk > 0);
              mma_f16(D, k128(T0 + oH2L, kk), k128(sb + oW2TH, kk), ID128_64, 1);
              mma_f16(D, k128(T0 + oH2H, kk), k128(sb + oW2TL, kk), ID128_64, 1);
            }
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              mma_f16(d + cG2, m128(T0 + oH2H, kk), m128(T0 + oH1H, kk), IDT64_64, kk == 0 ? 0 : 1);
              mma_f16(d + cG2, m128(T0 + oH2L, kk), m128(T0 + oH1H, kk), IDT64_64, 1);
              mma_f16(d + cG2, m128(T0 + oH2H, kk), m128(T0 + oH1L, kk), IDT64_64, 1);
              mma_f16(d + cG2b, m128(T0 + oH2H, kk), m32(sb + oONES, kk), IDT64_16, kk == 0 ? 0 : 1);
              mma_f16(d + cG2b, m128(T0 + oH2L, kk), m32(sb + oONES, kk), IDT64_16, 1);
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              mma_f16(D, k128(T0 + oH1H, kk), k128(sb + oW1TH, kk), ID128_16, kk > 0);
              mma_f16(D, k128(T0 + oH1L, kk), k128(sb + oW1TH, kk), ID128_16, 1);
              mma_f16(D, k128(T0 + oH1H, kk), k128(sb + oW1TL, kk), ID128_16, 1);
            }
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              mma_f16(d + cG1, m128(T0 + oH1H, kk), m32(T0 + oXH, kk), IDT64_16, kk == 0 ? 0 : 1);
              mma_f16(d + cG1, m128(T0 + oH1L, kk), m32(T0 + oXH, kk), IDT64_16, 1);
              mma_f16(d + cG1, m128(T0 + oH1H, kk), m32(T0 + oXL, kk), IDT64_16, 1);
            }
          }
          mma_commit(sb + oBars + 8 * g);
        }
        __syncwarp();
      }
    }
  } else {
    // ------------------------------------------------------------ warpgroups
    const int g = warp / 4, wq = warp & 3, t = tid & 127;
    const uint32_t d = tmem + (uint32_t)(g * 256) + ((uint32_t)(32 * wq) << 16);
    unsigned char* T = sm + oTiles + g * kTileBytes;
    const uint32_t dbar = sb + oBars + 8 * g;
    uint32_t dph = 0;
    float loss_s = 0.f, loss_e = 0.f;
    float b3s[kCMax], b3e[kCMax];
#pragma unroll
    for (int c = 0; c < kCMax; ++c) b3s[c] = b3e[c] = 0.f;
    auto wait_d = [&]() {
      if (!mbar_wait_bounded(dbar, dph, kDefaultWaitBudget)) {
        failed = true;
        mbar_wait_bounded(dbar, dph, kDrainBudget);
      }
      dph ^= 1u;
      tc_fence_after();
    };
    auto handoff = [&]() {
      fence_proxy_async_smem();
      tc_fence_before();
      __syncwarp();
      named_bar_arrive(1 + g, 160);
    };
    // split of 32 consecutive accumulator columns (two x16 loads) into a row of a
    // SW128 hi / lo tile pair, through f (ReLU or the derivative mask)
    auto epi64 = [&](uint32_t oh, uint32_t ol, uint32_t mask_lo, uint32_t mask_hi, bool relu, uint32_t& m_lo,
                     uint32_t& m_hi) {
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        uint32_t r[32];
        tmem_ld32_wait(d + cD + 32 * part, r);
        uint32_t mk = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t h[4], l[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int j = 8 * c + 2 * e;
            float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
            if (relu) {
              mk |= (v0 > 0.f ? 1u : 0u) << j;
              mk |= (v1 > 0.f ? 1u : 0u) << (j + 1);
              v0 = fmaxf(v0, 0.f);
              v1 = fmaxf(v1, 0.f);
            } else {
              const uint32_t m = part ? mask_hi : mask_lo;
              if (!((m >> j) & 1u)) v0 = 0.f;
              if (!((m >> (j + 1)) & 1u)) v1 = 0.f;
            }
            split_f16x2(v0, v1, h[e], l[e]);
          }
          const uint32_t o = sw128(t, 16 * (4 * part + c));
          sts128(smem_u32(T + oh + o), h[0], h[1], h[2], h[3]);
          sts128(smem_u32(T + ol + o), l[0], l[1], l[2], l[3]);
        }
        if (part == 0) m_lo = mk;
        else m_hi = mk;
      }
    };
    bool first_tile = true;
    for (int64_t tile = (int64_t)blockIdx.x * kWG + g; tile < tiles; tile += stride) {
      const int64_t sid = tile * 128 + t;
      const bool valid = sid < a.batch;
      // the sample's uv for the latent scatter at the end of the tile, loaded now
      // so its latency hides behind the tile's six phases
      const float2 uv = valid ? __ldg(reinterpret_cast<const float2*>(a.uv) + sid) : make_float2(0.f, 0.f);
      // ---- 1: X (12 features, column 12 = 1 in the hi tile) and the target
      float tv[kCMax];
      {
        float f[kIn];
#pragma unroll
        for (int c = 0; c < kCMax; ++c) tv[c] = 0.f;
        const float4* rec = reinterpret_cast<const float4*>(a.xt + (valid ? sid : 0) * a.rs);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float4 v = valid ? __ldg(rec + q) : make_float4(0.f, 0.f, 0.f, 0.f);
          f[4 * q] = v.x; f[4 * q + 1] = v.y; f[4 * q + 2] = v.z; f[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < kCMax / 4; ++q)
          if (4 * q < C) {
            const float4 v = valid ? __ldg(rec + 3 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            tv[4 * q] = v.x; tv[4 * q + 1] = v.y; tv[4 * q + 2] = v.z; tv[4 * q + 3] = v.w;
          }
        // the next tile's record into L2 (its loads then wait on L2, not DRAM)
        const int64_t nsid = (tile + stride) * 128 + t;
        if (nsid < a.batch) {
          const float* nrec = a.xt + nsid * a.rs;
          sm100::prefetch_l2(nrec);
          sm100::prefetch_l2(nrec + a.rs - 1);
        }
        uint32_t h[8], l[8];
#pragma unroll
        for (int i = 0; i < 6; ++i) split_f16x2(f[2 * i], f[2 * i + 1], h[i], l[i]);
        h[6] = 0x3C00u; l[6] = 0u;  // column 12: 1 (hi) / 0 (lo)
        h[7] = 0u; l[7] = 0u;
        sts128(smem_u32(T + oXH + sw32(t, 0)), h[0], h[1], h[2], h[3]);
        sts128(smem_u32(T + oXH + sw32(t, 16)), h[4], h[5], h[6], h[7]);
        sts128(smem_u32(T + oXL + sw32(t, 0)), l[0], l[1], l[2], l[3]);
        sts128(smem_u32(T + oXL + sw32(t, 16)), l[4], l[5], l[6], l[7]);
      }
      handoff();
      // ---- 2, 3: hidden activations (and their ReLU masks)
      uint32_t m1l, m1h, m2l, m2h;
      wait_d();
      epi64(oH1H, oH1L, 0, 0, true, m1l, m1h);
      handoff();
      wait_d();
      epi64(oH2H, oH2L, 0, 0, true, m2l, m2h);
      handoff();
      // ---- 4: y -> loss, unscaled dL/dy
      wait_d();
      {
        uint32_t r[16];
        tmem_ld16_wait(d + cD, r);
        float gv[kCMax];
#pragma unroll
        for (int c = 0; c < kCMax; ++c) {
          float gc = 0.f;
          if (c < C && valid) {
            const float res = __uint_as_float(r[c]) - tv[c];
            neumaier(loss_s, loss_e, a.loss_l1 ? fabsf(res) : res * res);
            gc = a.loss_l1 ? (res > 0.f ? 1.f : (res < 0.f ? -1.f : 0.f)) : 2.f * res;
            neumaier(b3s[c], b3e[c], gc);
          }
          gv[c] = gc;
        }
        uint32_t h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) split_f16x2(gv[2 * i], gv[2 * i + 1], h[i], l[i]);
        sts128(smem_u32(T + oDYH + sw32(t, 0)), h[0], h[1], h[2], h[3]);
        sts128(smem_u32(T + oDYH + sw32(t, 16)), h[4], h[5], h[6], h[7]);
        sts128(smem_u32(T + oDYL + sw32(t, 0)), l[0], l[1], l[2], l[3]);
        sts128(smem_u32(T + oDYL + sw32(t, 16)), l[4], l[5], l[6], l[7]);
      }
      handoff();
      // ---- 5, 6: dZ2 over H2, dZ1 over H1
      uint32_t dummy0, dummy1;
      wait_d();
      epi64(oH2H, oH2L, m2l, m2h, false, dummy0, dummy1);
      handoff();
      wait_d();
      epi64(oH1H, oH1L, m1l, m1h, false, dummy0, dummy1);
      handoff();
      // ---- dX (times the loss scale) into the latent gradients
      wait_d();
      {
        uint32_t r[16];
        tmem_ld16_wait(d + cD, r);
        // this tile's G (lanes 0..15 of the quarter, complete with the last commit)
        // into the running sums (lanes 16..31): lane j + 16 adds lane j's value
#pragma unroll 1
        for (int part = 0; part < 7; ++part) {
          const uint32_t col = part < 4 ? cG2 + 16 * part : part == 4 ? cG2b : part == 5 ? cG3 : cG1;
          uint32_t q[16];
          tmem_ld16_wait(d + col, q);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float tv = __shfl_up_sync(0xFFFFFFFFu, __uint_as_float(q[j]), 16);
            if (lane >= 16) q[j] = __float_as_uint(first_tile ? tv : __uint_as_float(q[j]) + tv);
          }
          tmem_st16(d + col, q);
        }
        tmem_wait_st();
        first_tile = false;
        tc_fence_before();
        if (valid) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            Taps Tp = clamp_taps(uv.x, uv.y, a.lw[k], a.lh[k], a.shift[k]);
            check_taps(Tp, (int64_t)a.lw[k] * a.lh[k], a);
            float* G = a.lgrad[k];
            const float g0 = a.scale * __uint_as_float(r[3 * k]), g1 = a.scale * __uint_as_float(r[3 * k + 1]),
                        g2 = a.scale * __uint_as_float(r[3 * k + 2]);
            if constexpr (LV) {
              float4* G4 = reinterpret_cast<float4*>(G);
              atomicAdd(G4 + Tp.i00, make_float4(Tp.w00 * g0, Tp.w00 * g1, Tp.w00 * g2, 0.f));
              atomicAdd(G4 + Tp.i10, make_float4(Tp.w10 * g0, Tp.w10 * g1, Tp.w10 * g2, 0.f));
              atomicAdd(G4 + Tp.i01, make_float4(Tp.w01 * g0, Tp.w01 * g1, Tp.w01 * g2, 0.f));
              atomicAdd(G4 + Tp.i11, make_float4(Tp.w11 * g0, Tp.w11 * g1, Tp.w11 * g2, 0.f));
            } else {
              const float gg[3] = {g0, g1, g2};
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                atomicAdd(G + 3 * Tp.i00 + c, Tp.w00 * gg[c]);
                atomicAdd(G + 3 * Tp.i10 + c, Tp.w10 * gg[c]);
                atomicAdd(G + 3 * Tp.i01 + c, Tp.w01 * gg[c]);
                atomicAdd(G + 3 * Tp.i11 + c, Tp.w11 * gg[c]);
              }
            }
          }
        }
      }
    }
    // ---- this warpgroup's gradient sums: G2 (dW2), G2b (db2), G3 (dW3^T), G1 (dW1, db1)
    //      row 16 wq + j of the running sums: lane 16 + j of warp wq's quarter
    const bool has_tiles = (int64_t)blockIdx.x * kWG + g < tiles;
    // stash: per warpgroup a [rows 64][cols] block in its own tile area (the tiles are done)
    float* gs = reinterpret_cast<float*>(T);  // 64 x (64 + 16 + 16 + 16) floats = 28 KB
    {
      const int row = 16 * wq + lane - 16;
      for (int part = 0; part < 7; ++part) {
        // columns: G2 0..63 (4 x 16), G2b 64..79, G3 80..95, G1 96..111
        const uint32_t col = part < 4 ? cG2 + 16 * part : part == 4 ? cG2b : part == 5 ? cG3 : cG1;
        uint32_t r[16];
        tmem_ld16_wait(d + col, r);
        if (lane >= 16) {
#pragma unroll
          for (int j = 0; j < 16; ++j) gs[row * 112 + 16 * part + j] = has_tiles ? __uint_as_float(r[j]) * a.scale : 0.f;
        }
      }
    }
    // loss and db3: this warpgroup's per-thread compensated sums, reduced in a fixed order
    float* red = reinterpret_cast<float*>(T + 64 * 112 * 4);  // 128 threads x (1 + 16) x 2
    red[t * 34] = loss_s;
    red[t * 34 + 1] = loss_e;
#pragma unroll
    for (int c = 0; c < kCMax; ++c) {
      red[t * 34 + 2 + 2 * c] = b3s[c] * a.scale;
      red[t * 34 + 3 + 2 * c] = b3e[c] * a.scale;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // ---- the CTA's partials: warpgroup 0 + warpgroup 1, compensated
  {
    float* part = a.part + (size_t)blockIdx.x * kPart;
    const float* g0 = reinterpret_cast<const float*>(sm + oTiles);
    const float* g1 = reinterpret_cast<const float*>(sm + oTiles + kTileBytes);
    auto put = [&](int slot, float x0, float x1) {
      float s = 0.f, e = 0.f;
      neumaier(s, e, x0);
      neumaier(s, e, x1);
      part[2 * slot] = s;
      part[2 * slot + 1] = e;
    };
    for (int e = tid; e < 64 * 112; e += blockDim.x) {
      const int row = e / 112, col = e - row * 112;
      const float x0 = g0[e], x1 = g1[e];
      if (col < 64) put(kGW2 + row * kH + col, x0, x1);                     // dW2[out = row][in = col]
      else if (col == 64) put(kGB2 + row, x0, x1);                          // db2
      else if (col >= 80 && col < 96) {                                     // dW3[c][in = row]
        const int c = col - 80;
        if (c < kCMax) put(kGW3 + c * kH + row, c < C ? x0 : 0.f, c < C ? x1 : 0.f);
      } else if (col >= 96 && col < 96 + kIn) put(kGW1 + row * kIn + (col - 96), x0, x1);  // dW1
      else if (col == 96 + kIn) put(kGB1 + row, x0, x1);                    // db1 (the ones column of X)
    }
    if (tid <= kCMax) {  // thread q: the loss (q = 0) or db3[q - 1], over both warpgroups in a fixed order
      const float* r0 = reinterpret_cast<const float*>(sm + oTiles + 64 * 112 * 4);
      const float* r1 = reinterpret_cast<const float*>(sm + oTiles + kTileBytes + 64 * 112 * 4);
      {
        const int q = tid;
        float s = 0.f, e = 0.f;
        for (int w = 0; w < kWG; ++w) {
          const float* r = w ? r1 : r0;
          for (int th = 0; th < 128; ++th) {
            neumaier(s, e, r[th * 34 + 2 * q]);
            e += r[th * 34 + 2 * q + 1];
          }
        }
        if (q == 0) {
          part[2 * kGN] = s;
          part[2 * kGN + 1] = e;
        } else {
          part[2 * (kGB3 + q - 1)] = q - 1 < C ? s : 0.f;
          part[2 * (kGB3 + q - 1) + 1] = q - 1 < C ? e : 0.f;
        }
      }
    }
  }
  if (failed) record_status(a.status, NBTC_ERR_TIMEOUT);
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace nbtc
