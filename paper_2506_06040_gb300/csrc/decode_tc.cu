// Host side of the tensor-core decode forms: MLP packing (FP16 / E4M3 image
// of shared memory), launch dispatch.  The kernel is in tc_kernel.cuh.
#include <cstring>

#include "host.h"
#include "sm100.cuh"
#include "tc.cuh"

namespace nbtc {

using namespace sm100;

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

// Narrow parts of one weight (already divided by its layer scale, FP8 forms):
// part 0 = hi, part 1 = lo (split forms), as the bytes of one element.
struct WParts {
  uint16_t h16, l16;  // FP16 forms
  uint8_t h8, l8;     // FP8 forms
};
__device__ inline WParts weight_parts(float w) {
  WParts r;
  uint32_t hi, lo;
  split_f16x2(w, 0.f, hi, lo);  // FP16: hi = RN16(w), lo = RN16(w - hi)
  r.h16 = (uint16_t)(hi & 0xFFFF);
  r.l16 = (uint16_t)(lo & 0xFFFF);
  uint16_t h8, l8;
  split_e4m3x2(cvt_f16x2(w, 0.f), h8, l8);  // FP8 split: via RN16(w)
  r.h8 = (uint8_t)(h8 & 0xFF);
  r.l8 = (uint8_t)(l8 & 0xFF);
  return r;
}

// One CTA: converts the FP32 MLP into the shared-memory image of `form`.
// Hidden width `hid` (16, 32 or 64) is zero-padded to the image's 64: the
// padded neurons have zero weights and bias, so they stay exactly 0 through
// ReLU and add exact zeros to the next layer's sums.
__global__ void k_pack_mlp(const float* __restrict__ W, const float* __restrict__ B, int nhid, int nin, int hid,
                           int nout, int form, const float* __restrict__ act_absmax, unsigned char* __restrict__ out) {
  const TcLayout L{nhid, form};
  const bool fp8 = L.fp8(), split = L.split();
  __shared__ float wmax[8];
  __shared__ float sw[8], sa[8];
  const int nl = nhid + 1;
  if (threadIdx.x < 8) wmax[threadIdx.x] = 0.f;
  __syncthreads();
  // per-layer weight absmax
  int off = 0;
  for (int l = 0; l < nl; ++l) {
    const int in = l == 0 ? nin : hid, o = l == nhid ? nout : hid;
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
  const int R1 = L.w1_row();
  off = 0;
  for (int l = 0; l < nl; ++l) {
    const int in = l == 0 ? nin : hid, o = l == nhid ? nout : hid;
    for (int e = threadIdx.x; e < in * o; e += blockDim.x) {
      const int n = e / in, k = e - n * in;
      const float w = W[off + e] / sw[l];  // exact: sw is a power of two (1 for FP16)
      if (l == 0) {
        // W1 rows (see TcLayout): K-major, no swizzle
        if (form == kF16) {
          *reinterpret_cast<__half*>(out + L.off_w1() + off_ilv(n, 2 * k, R1)) = __float2half_rn(w);
        } else if (form == kF8) {
          out[L.off_w1() + off_ilv(n, k, R1)] = (unsigned char)(cvt_e4m3x2(w, 0.f) & 0xFF);
        } else if (L.f16split()) {
          const WParts q = weight_parts(w);
          *reinterpret_cast<uint16_t*>(out + L.off_w1() + off_ilv(n, 2 * k, R1)) = q.h16;
          *reinterpret_cast<uint16_t*>(out + L.off_w1() + off_ilv(n, 2 * (16 + k), R1)) = q.h16;
          *reinterpret_cast<uint16_t*>(out + L.off_w1() + off_ilv(n, 2 * (32 + k), R1)) = q.l16;
        } else {
          const WParts q = weight_parts(w);
          out[L.off_w1() + off_ilv(n, k, R1)] = q.h8;
          out[L.off_w1() + off_ilv(n, 16 + k, R1)] = q.h8;
          out[L.off_w1() + off_ilv(n, 32 + k, R1)] = q.l8;
        }
      } else {
        // later layers: swizzled K-major tiles, the lo tile after the hi tile
        const int base = l == nhid ? L.off_wo() : L.off_wh(l - 1);
        const int part = l == nhid ? L.wo_part() : L.wh_part();
        if (!fp8) {
          const uint32_t dst = base + off_sw128(n, 2 * k);
          if (!split) {
            *reinterpret_cast<__half*>(out + dst) = __float2half_rn(w);
          } else {
            const WParts q = weight_parts(w);
            *reinterpret_cast<uint16_t*>(out + dst) = q.h16;
            *reinterpret_cast<uint16_t*>(out + dst + part) = q.l16;
          }
        } else {
          const uint32_t dst = base + off_sw64(n, k);
          if (!split) {
            out[dst] = (unsigned char)(cvt_e4m3x2(w, 0.f) & 0xFF);
          } else {
            const WParts q = weight_parts(w);
            out[dst] = q.h8;
            out[dst + part] = q.l8;
          }
        }
      }
    }
    off += in * o;
  }
  if (!fp8) {  // FP16 biases as MMA operands: W1 column(s), then [N x 16] tiles (column 0, split: and 1)
    int bo = 0;
    for (int l = 0; l < nl; ++l) {
      const int o = l == nhid ? nout : hid;
      for (int e = threadIdx.x; e < o; e += blockDim.x) {
        const WParts q = weight_parts(B[bo + e]);
        if (l == 0) {
          *reinterpret_cast<uint16_t*>(out + L.off_w1() + off_ilv(e, 2 * nin, R1)) = q.h16;
          if (split) *reinterpret_cast<uint16_t*>(out + L.off_w1() + off_ilv(e, 2 * (16 + nin), R1)) = q.l16;
        } else {
          const int bt = l == nhid ? L.off_bto() : L.off_bth(l - 1);
          *reinterpret_cast<uint16_t*>(out + bt + off_interleave(e, 0)) = q.h16;
          if (split) *reinterpret_cast<uint16_t*>(out + bt + off_interleave(e, 2)) = q.l16;
        }
      }
      bo += o;
    }
  }
  // biases (hidden layers pre-divided by the next layer's input scale) and epilogue multipliers
  float* bias = reinterpret_cast<float*>(out + L.off_bias());
  float* alpha = reinterpret_cast<float*>(out + L.off_alpha());
  int boff = 0;
  for (int l = 0; l < nl; ++l) {
    const int o = l == nhid ? nout : hid;
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
  const int D = mlp->dims[1];
  if (D != 16 && D != 32 && D != kHid) return fail(NBTC_ERR_UNSUPPORTED, "tensor-core forms take hidden width 16, 32 or 64");
  for (int l = 1; l < L; ++l)
    if (mlp->dims[l] != D) return fail(NBTC_ERR_UNSUPPORTED, "hidden layers must share one width");
  if (mlp->dims[L] < 1 || mlp->dims[L] > kMaxOut) return fail(NBTC_ERR_UNSUPPORTED, "at most 16 outputs");
  return NBTC_OK;
}

// TcForm of a tensor-core precision code (-1: none).
static int tc_form(int precision) {
  switch (precision) {
    case NBTC_FP16: return kF16;
    case NBTC_FP8_E4M3: return kF8;
    case NBTC_FP16_SPLIT: return kF16Split;
    case NBTC_FP32_TC: return kF32Split;
    case NBTC_FP8_E4M3_SPLIT: return kF8Split;
  }
  return -1;
}

nbtc_status tc_packed_bytes(const nbtc_mlp* mlp, int precision, size_t* bytes) {
  int nhid;
  nbtc_status st = tc_shape(mlp, nhid);
  if (st) return st;
  const int form = tc_form(precision);
  if (form < 0) return fail(NBTC_ERR_INVALID_ARG, "not a tensor-core precision");
  *bytes = (size_t)TcLayout{nhid, form}.bytes();
  return NBTC_OK;
}

nbtc_status launch_pack_mlp(nbtc_context* ctx, const nbtc_mlp* mlp, int precision, const float* act_absmax,
                            void* packed, size_t packed_bytes, cudaStream_t s) {
  (void)ctx;
  int nhid;
  nbtc_status st = tc_shape(mlp, nhid);
  if (st) return st;
  const int form = tc_form(precision);
  if (form < 0) return fail(NBTC_ERR_INVALID_ARG, "not a tensor-core precision");
  const TcLayout L{nhid, form};
  if (packed_bytes < (size_t)L.bytes()) return fail(NBTC_ERR_INVALID_ARG, "packed buffer too small");
  if (!packed || !aligned(packed, 16)) return fail(NBTC_ERR_INVALID_ARG, "packed buffer NULL or not 16-byte aligned");
  if (L.fp8() && !act_absmax) return fail(NBTC_ERR_INVALID_ARG, "FP8 packing needs the calibration absmax");
  k_pack_mlp<<<1, 256, 0, s>>>(mlp->weights, mlp->biases, nhid, mlp->dims[0], mlp->dims[1], mlp->dims[nhid + 1], form,
                               act_absmax, static_cast<unsigned char*>(packed));
  return cuda_check(cudaGetLastError(), "launch k_pack_mlp");
}

// one per instantiation unit (tc_h<depth>_<form>.cu)
#define NBTC_TC_UNIT(name) nbtc_status name(const TcArgs& p, int W, int slots, int grid, cudaStream_t s);
NBTC_TC_UNIT(launch_tc_h1_f16)
NBTC_TC_UNIT(launch_tc_h2_f16)
NBTC_TC_UNIT(launch_tc_h3_f16)
NBTC_TC_UNIT(launch_tc_h1_f8)
NBTC_TC_UNIT(launch_tc_h2_f8)
NBTC_TC_UNIT(launch_tc_h3_f8)
NBTC_TC_UNIT(launch_tc_h1_f16s)
NBTC_TC_UNIT(launch_tc_h2_f16s)
NBTC_TC_UNIT(launch_tc_h3_f16s)
NBTC_TC_UNIT(launch_tc_h1_f8s)
NBTC_TC_UNIT(launch_tc_h2_f8s)
NBTC_TC_UNIT(launch_tc_h3_f8s)
NBTC_TC_UNIT(launch_tc_h1_f32s)
NBTC_TC_UNIT(launch_tc_h2_f32s)
NBTC_TC_UNIT(launch_tc_h3_f32s)
NBTC_TC_UNIT(launch_tc_h1_f16_batch)
NBTC_TC_UNIT(launch_tc_h2_f16_batch)
NBTC_TC_UNIT(launch_tc_h3_f16_batch)
#undef NBTC_TC_UNIT

nbtc_status launch_tc_args(nbtc_context* ctx, const TcArgs& p, int nhid, int form, int W, int slots, int grid,
                           cudaStream_t s) {
  (void)ctx;
  if (nhid < 1 || nhid > 3) return fail(NBTC_ERR_UNSUPPORTED, "tensor-core decode takes 1..3 hidden layers");
  using Fn = nbtc_status (*)(const TcArgs&, int, int, int, cudaStream_t);
  if (p.mode == kModeBatch) {
    if (form != kF16) return fail(NBTC_ERR_UNSUPPORTED, "batched decode runs the FP16 form");
    static const Fn batch[3] = {launch_tc_h1_f16_batch, launch_tc_h2_f16_batch, launch_tc_h3_f16_batch};
    return batch[nhid - 1](p, W, slots, grid, s);
  }
  static const Fn single[5][3] = {{launch_tc_h1_f16, launch_tc_h2_f16, launch_tc_h3_f16},
                                  {launch_tc_h1_f8, launch_tc_h2_f8, launch_tc_h3_f8},
                                  {launch_tc_h1_f16s, launch_tc_h2_f16s, launch_tc_h3_f16s},
                                  {launch_tc_h1_f8s, launch_tc_h2_f8s, launch_tc_h3_f8s},
                                  {launch_tc_h1_f32s, launch_tc_h2_f32s, launch_tc_h3_f32s}};
  if (form < 0 || form > 4) return fail(NBTC_ERR_INVALID_ARG, "not a tensor-core precision");
  return single[form][nhid - 1](p, W, slots, grid, s);
}

// Warpgroups and tile slots per CTA of a form.  The forms keep their MMA A
// operands in TMEM (default), one slot per warpgroup: a slot takes the 64
// accumulator columns plus its A operand (FP16 32 columns, split FP16 64, E4M3
// 16, split E4M3 32), so the FP16 forms fit 4 warpgroups and the E4M3 forms 5
// (measured: 5 x 1 is 5% / 10% faster for E4M3 / split E4M3, 2% for FP16, whose
// 4 x 1 is kept).  With shared-memory operands (context setting) the split-FP16
// forms, whose two A tiles per slot fill shared memory, run 4 x 1; the others
// two slots of 3 or 4 warpgroups (context setting).
static void tc_shape_of(const nbtc_context* ctx, int form, int& W, int& slots) {
  const bool ta = ctx->tc_tmem_a != 0;
  if (ta || form == kF16Split || form == kF32Split) {
    W = ta && (form == kF8 || form == kF8Split) ? 5 : 4;
    slots = 1;
  } else {
    W = ctx->tc_groups == 3 ? 3 : 4;
    slots = 2;
  }
}

nbtc_status launch_decode_tc(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, int precision,
                             const void* packed, cudaStream_t s) {
  int nhid;
  nbtc_status st = tc_shape(mlp, nhid);
  if (st) return st;
  const int form = tc_form(precision);
  if (form < 0) return fail(NBTC_ERR_INVALID_ARG, "not a tensor-core precision");
  if (!packed || !aligned(packed, 16)) return fail(NBTC_ERR_INVALID_ARG, "packed MLP NULL or not 16-byte aligned");
  TcArgs p;
  memset(&p, 0, sizeof(p));
  p.d = a;
  p.packed = packed;
  p.nout = mlp->dims[nhid + 1];
  p.tiles = (a.n + kTile - 1) / kTile;
  p.budget = ctx->wait_budget > 0 ? ctx->wait_budget : ctx->wait_budget < 0 ? 0 : kDefaultWaitBudget;
  bool fp = a.uv == nullptr && (a.grid_w % kTile) == 0;
  for (int k = 0; k < 4; ++k) fp = fp && a.lv[k].w <= a.grid_w;
  p.footprint = fp ? 1 : 0;
  p.hdiv = make_fastdiv(fp && a.grid_h > 0 ? (uint32_t)a.grid_h : 1u);
  p.mode = kModeSingle;
  if (p.tiles >= (int64_t)1 << 31) return fail(NBTC_ERR_UNSUPPORTED, "more than 2^31 tiles");
  int W, slots;
  tc_shape_of(ctx, form, W, slots);
  p.tmem_a = ctx->tc_tmem_a ? 1 : 0;
  int64_t grid = (p.tiles + W * slots - 1) / (W * slots);
  if (grid > ctx->sm_count) grid = ctx->sm_count;
  p.per_cta = (p.tiles + grid - 1) / grid;
  return launch_tc_args(ctx, p, nhid, form, W, slots, (int)grid, s);
}

}  // namespace nbtc
