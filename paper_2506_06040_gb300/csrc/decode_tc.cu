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
  int64_t tiles;
  long long budget;    // polls per bounded wait
};

// Shared-memory plan.  Per group: A0 (128 x K1 operand, reused as the output
// staging buffer) and Ah (128 x 64 operand, reused as the feature stage's
// column buffer while no MMA reads it).
struct TcSmem {
  int image;       // packed MLP (rounded to 1 KB)
  int ones;        // 128 x 16 FP16 tile of ones in column 0
  int groups;      // first group
  int group;       // bytes per group
  int a0, ah, bar; // offsets inside a group
  int misc;        // weight barrier + TMEM slot
  int total;
};

__host__ __device__ inline TcSmem tc_smem(const TcLayout& L, int kGroups) {
  TcSmem s;
  s.image = (L.bytes() + 1023) & ~1023;
  s.ones = s.image;
  s.groups = s.ones + 4096;
  s.a0 = 0;
  s.ah = 4096;
  s.bar = s.ah + 16384;
  s.group = (s.bar + 16 + 1023) & ~1023;
  s.misc = s.groups + kGroups * s.group;
  s.total = s.misc + 64 + 1024 /* alignment slack */;
  return s;
}

// kGroups tile groups of 128 threads per CTA, one CTA per SM.
template <int NHID, bool FP8, int kGroups>
__global__ void __launch_bounds__(kGroups * kTile, 1) k_decode_tc(TcArgs p) {
  constexpr TcLayout L{NHID, FP8};
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const TcSmem S = tc_smem(L, kGroups);
  const uint32_t sbase = smem_u32(smem);
  const int tid = threadIdx.x;
  const int g = tid / kTile;          // group
  const int gt = tid % kTile;         // texel row inside the tile
  const int warp = tid / 32;
  const bool leader = gt == 0;
  unsigned char* gsm = smem + S.groups + g * S.group;
  const uint32_t gbase = sbase + S.groups + g * S.group;
  const uint32_t wbar = sbase + S.misc;                                  // weight-load barrier
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S.misc + 16);
  const uint32_t gbar = gbase + S.bar;
  const int bar_id = 1 + g;
  constexpr uint32_t kTmemCols = kGroups * kHid <= 256 ? 256 : 512;

  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(wbar, 1);
    for (int q = 0; q < kGroups; ++q) mbar_init(sbase + S.groups + q * S.group + S.bar, 1);
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
  const uint32_t tmem = *tmem_slot + (uint32_t)(g * kHid);                 // group's columns
  const uint32_t tmem_row = tmem + ((uint32_t)(32 * (warp & 3)) << 16);   // this warp's lanes
  bool failed = !mbar_wait_bounded(wbar, 0, p.budget);
  failed = __syncthreads_or(failed);
  if (failed && tid == 0) record_status(p.d.status, NBTC_ERR_TIMEOUT);

  const float* bias = reinterpret_cast<const float*>(smem + L.off_bias());
  const float* alpha = reinterpret_cast<const float*>(smem + L.off_alpha());
  const uint32_t a0 = gbase + S.a0, ah = gbase + S.ah;
  float4* colbuf = reinterpret_cast<float4*>(gsm + S.ah);
  uint16_t* stage = reinterpret_cast<uint16_t*>(gsm + S.a0);
  constexpr uint32_t ID_HID = idesc(0, kTile, kHid);
  constexpr uint32_t ID_OUT = idesc(0, kTile, kOutPad);
  uint32_t phase = 0;

  for (int64_t tile = (int64_t)blockIdx.x * kGroups + g; !failed && tile < p.tiles;
       tile += (int64_t)gridDim.x * kGroups) {
    const int64_t t0 = tile * kTile;
    const int64_t tex = t0 + gt;
    const bool full = t0 + kTile <= p.d.n;
    if (leader) bulk_wait_read0();  // the previous tile's staged output (in A0) has been read

    // ---- features -> A0
    float f[12];
    if (p.footprint) {
      footprint_features<kTile>(p.d, t0, gt, colbuf, bar_id, f);  // includes a group barrier
    } else {
      direct_features(p.d, tex < p.d.n ? tex : p.d.n - 1, f);
      named_bar_sync(bar_id, kTile);
    }
    if constexpr (!FP8) {
      const uint32_t w0 = cvt_f16x2(f[0], f[1]), w1 = cvt_f16x2(f[2], f[3]);
      const uint32_t w2 = cvt_f16x2(f[4], f[5]), w3 = cvt_f16x2(f[6], f[7]);
      const uint32_t w4 = cvt_f16x2(f[8], f[9]), w5 = cvt_f16x2(f[10], f[11]);
      sts128(a0 + off_interleave(gt, 0), w0, w1, w2, w3);
      sts128(a0 + off_interleave(gt, 16), w4, w5, 0x3C00u /* k = 12: 1.0 for the bias */, 0u);
    } else {
      const float is = alpha[NHID + 1];  // 1 / input scale
      uint32_t q[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        q[i] = (uint32_t)cvt_e4m3x2(f[4 * i] * is, f[4 * i + 1] * is) |
               ((uint32_t)cvt_e4m3x2(f[4 * i + 2] * is, f[4 * i + 3] * is) << 16);
      sts128(a0 + off_interleave(gt, 0), q[0], q[1], q[2], 0u);
      sts128(a0 + off_interleave(gt, 16), 0u, 0u, 0u, 0u);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    named_bar_sync(bar_id, kTile);

#pragma unroll 1
    for (int layer = 0; layer <= NHID; ++layer) {
      const bool last = layer == NHID;
      // ---- issue this layer's MMAs
      if (leader) {
        tc_fence_after();
        if (layer == 0) {
          const uint64_t ad = smem_desc(a0, 128, 256, kSwzNone);
          const uint64_t bd = smem_desc(sbase + L.off_w1(), 128, 256, kSwzNone);
          if constexpr (FP8) mma_f8(tmem, ad, bd, ID_HID, 0);
          else mma_f16(tmem, ad, bd, ID_HID, 0);
        } else {
          const uint32_t wb = sbase + (last ? L.off_wo() : L.off_wh(layer - 1));
          const uint32_t id = last ? ID_OUT : ID_HID;
          if constexpr (FP8) {
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
              mma_f8(tmem, smem_desc(ah + kk * 32, 16, 512, kSwz64), smem_desc(wb + kk * 32, 16, 512, kSwz64), id,
                     kk > 0);
          } else {
            const uint32_t bt = sbase + (last ? L.off_bto() : L.off_bth(layer - 1));
            mma_f16(tmem, smem_desc(sbase + S.ones, 128, 256, kSwzNone), smem_desc(bt, 128, 256, kSwzNone), id, 0);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_f16(tmem, smem_desc(ah + kk * 32, 16, 1024, kSwz128), smem_desc(wb + kk * 32, 16, 1024, kSwz128),
                      id, 1);
          }
        }
        mma_commit(gbar);
      }
      // ---- wait for the accumulator (warp-uniform: tcgen05.ld is a .sync.aligned warp instruction)
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(gbar, phase, p.budget));
      phase ^= 1u;
      tc_fence_after();
      if (!last) {
        const float alp = alpha[layer];
        const float* b = bias + layer * kHid;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          uint32_t r[32];
          if (ok) {
            tmem_ld16(tmem_row + 32 * half, r);
            tmem_ld16(tmem_row + 32 * half + 16, r + 16);
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
        failed = named_bar_or(bar_id, kTile, !ok);
        if (failed) break;
      } else {
        uint32_t r[16];
        if (ok) {
          tmem_ld16(tmem_row, r);
          tmem_wait_ld16(r);
        }
        const float alp = alpha[NHID];
        const float* b = bias + NHID * kHid;
        __half hv[kMaxOut];
#pragma unroll
        for (int k = 0; k < kMaxOut; ++k)
          hv[k] = FP8 ? __float2half_rn(fmaf(__uint_as_float(r[k]), alp, b[k])) : __float2half_rn(__uint_as_float(r[k]));
        if (full) {
#pragma unroll
          for (int k = 0; k < kMaxOut; ++k)
            if (k < p.nout) stage[gt * p.nout + k] = __half_as_ushort(hv[k]);
          fence_proxy_async_smem();
        } else if (tex < p.d.n) {
          uint16_t* o = reinterpret_cast<uint16_t*>(p.d.out) + tex * p.nout;
#pragma unroll
          for (int k = 0; k < kMaxOut; ++k)
            if (k < p.nout) o[k] = __half_as_ushort(hv[k]);
        }
        tc_fence_before();
        failed = named_bar_or(bar_id, kTile, !ok);
        if (!failed && full && leader) {
          bulk_s2g(reinterpret_cast<uint16_t*>(p.d.out) + t0 * p.nout, gbase + S.a0, (uint32_t)(kTile * p.nout * 2));
          bulk_commit();
        }
      }
    }
  }
  if (failed && leader) record_status(p.d.status, NBTC_ERR_TIMEOUT);
  if (leader) bulk_wait0();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(*tmem_slot, kTmemCols);
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

template <int NHID, bool FP8, int kGroups>
static nbtc_status launch_tc_g(nbtc_context* ctx, const TcArgs& p, cudaStream_t s) {
  const TcSmem S = tc_smem(TcLayout{NHID, FP8}, kGroups);
  auto kern = k_decode_tc<NHID, FP8, kGroups>;
  nbtc_status st =
      cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S.total), "smem attribute");
  if (st) return st;
  int64_t grid = (p.tiles + kGroups - 1) / kGroups;
  if (grid > ctx->sm_count) grid = ctx->sm_count;
  kern<<<(int)grid, kGroups * kTile, S.total, s>>>(p);
  return cuda_check(cudaGetLastError(), "launch k_decode_tc");
}

template <int NHID, bool FP8>
static nbtc_status launch_tc_t(nbtc_context* ctx, const TcArgs& p, cudaStream_t s) {
  return ctx->tc_groups == 6 ? launch_tc_g<NHID, FP8, 6>(ctx, p, s) : launch_tc_g<NHID, FP8, 4>(ctx, p, s);
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
  const bool f8 = precision == NBTC_FP8_E4M3;
  if (nhid == 1) return f8 ? launch_tc_t<1, true>(ctx, p, s) : launch_tc_t<1, false>(ctx, p, s);
  if (nhid == 2) return f8 ? launch_tc_t<2, true>(ctx, p, s) : launch_tc_t<2, false>(ctx, p, s);
  return f8 ? launch_tc_t<3, true>(ctx, p, s) : launch_tc_t<3, false>(ctx, p, s);
}

}  // namespace nbtc
