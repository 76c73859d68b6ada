// Training step of the decoder on continuous latents (Sec. 3.2): forward
// (bilinear latent sampling + MLP 12-64-64-C), loss against the bilinearly
// sampled target, backward through the MLP into every latent texel, Adam.
//
// k_gather (when the workspace has room): one thread per sample samples the
// latents and the target and writes the sample's features and target channels
// as one record, so the scattered taps of many samples are in flight at once;
// k_train then reads the records coalesced (otherwise it samples them itself).
//
// k_train: persistent CTAs of 256 threads (one per SM) walk 256-sample tiles.
// Per tile all activations live in shared memory, feature-major ([k][sample],
// samples contiguous; backward deltas overwrite the activations they follow),
// and every dense product is a register-blocked SIMT FP32 GEMM on packed FP32x2
// FMAs (true FP32 FFMA; activations are recomputed per call, never stored to
// HBM).  Weight/bias gradients: per-tile sums added into per-thread running
// sums with Neumaier compensation (each thread owns fixed entries), written to
// the workspace at the end; k_reduce_adam adds the CTA partials in a fixed
// order (compensated), writes the gradients and applies Adam.  Latent
// gradients: FP32 atomics (16-byte vector adds with 4-float texels).
#include <mutex>
#include <string>

#include "host.h"

namespace nbtc {

constexpr int kTS = 256;        // samples per tile
constexpr int kLd = kTS + 4;    // row stride of the activations: consecutive rows 4 banks apart
constexpr int kTT = 256;        // threads per CTA
constexpr int kH = 64;          // hidden width
constexpr int kIn = 12;         // features
constexpr int kCMax = 16;       // output channels (padded)

// gradient slots: dW1 [64][12], dW2 [64][64], dW3 [16][64], db1, db2, db3 (padded C)
constexpr int kGW1 = 0, kGW2 = kGW1 + kH * kIn, kGW3 = kGW2 + kH * kH, kGB1 = kGW3 + kCMax * kH,
              kGB2 = kGB1 + kH, kGB3 = kGB2 + kH, kGN = kGB3 + kCMax;  // 6032
constexpr int kPart = 2 * (kGN + 1);  // per CTA: (sum, compensation) of every gradient slot and the loss

enum TrainMode { kModeFwd = 0, kModeBwd = 1, kModeTrain = 2 };

struct TrainDev {
  const float* lat[4];
  float* lgrad[4];
  int lw[4], lh[4];
  float shift[4];
  const float* W;  // W1 [64][12], W2 [64][64], W3 [C][64]
  const float* B;  // b1 [64], b2 [64], b3 [C]
  const float* target;
  int tw, th;
  int ts;  // floats per target texel
  const float* uv;
  int64_t batch;
  int C;
  float scale;      // 1 / (batch * C)
  int loss_l1;
  const float* dy;  // backward mode
  float* y;         // forward mode
  float* part;      // [gridDim.x][kPart]
  const float* xt;  // pre-gathered samples [batch][rs] (features, then target channels), or null
  int rs;           // floats per pre-gathered sample
  int* status;      // checked build: status word the bounds checks record to
  int plant;        // checked build, tests only: offset added to every tap index (0 otherwise)
};

// Neumaier: (s, e) += x, exact sum ~ s + e
__device__ __forceinline__ void neumaier(float& s, float& e, float x) {
  const float t = s + x;
  e += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// Clamp-addressed bilinear taps of texture (w x h) at uv with a shift.
struct Taps {
  int i00, i10, i01, i11;  // texel indices
  float w00, w10, w01, w11;
};
__device__ __forceinline__ Taps clamp_taps(float u, float v, int w, int h, float shift) {
  float x = fmaf(u, (float)w, shift - 0.5f), y = fmaf(v, (float)h, shift - 0.5f);
  x = fminf(fmaxf(x, -1.f), (float)w);
  y = fminf(fmaxf(y, -1.f), (float)h);
  const float fx0 = floorf(x), fy0 = floorf(y);
  const float fx = x - fx0, fy = y - fy0;
  const int x0 = (int)fx0, y0 = (int)fy0;
  const int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
  const int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
  Taps t;
  t.i00 = ya * w + xa;
  t.i10 = ya * w + xb;
  t.i01 = yb * w + xa;
  t.i11 = yb * w + xb;
  t.w00 = (1.f - fx) * (1.f - fy);
  t.w10 = fx * (1.f - fy);
  t.w01 = (1.f - fx) * fy;
  t.w11 = fx * fy;
  return t;
}

// Checked build: the tap indices of a texture of n texels against its extent
// (plus the test-only offset); compiled away otherwise.
__device__ __forceinline__ void check_taps(Taps& T, int64_t n, const TrainDev& a) {
#ifdef NBTC_CHECKED
  int64_t i00 = (int64_t)T.i00 + a.plant, i10 = (int64_t)T.i10 + a.plant;
  int64_t i01 = (int64_t)T.i01 + a.plant, i11 = (int64_t)T.i11 + a.plant;
  NBTC_CHECK_INDEX(i00, n, a.status);
  NBTC_CHECK_INDEX(i10, n, a.status);
  NBTC_CHECK_INDEX(i01, n, a.status);
  NBTC_CHECK_INDEX(i11, n, a.status);
  T.i00 = (int)i00;
  T.i10 = (int)i10;
  T.i01 = (int)i01;
  T.i11 = (int)i11;
#else
  (void)T;
  (void)n;
  (void)a;
#endif
}

}  // namespace nbtc

#include "train_tc.cuh"

namespace nbtc {

// Shared memory of k_train: weights in both orientations (forward products
// read W^T rows, backward products read W rows, both as broadcast 128-bit
// loads), biases, and the tile's activations feature-major [row][sample]:
// X (features), H1, H2 (later overwritten by D1, D2), DY (targets, then dL/dy).
struct TrainSmem {
  float W1t[kIn * kH], W1[kH * kIn], W2t[kH * kH], W2[kH * kH], W3t[kH * kCMax], W3[kCMax * kH];
  float b1[kH], b2[kH], b3[kCMax];
  float X[kIn * kLd], H1[kH * kLd], H2[kH * kLd], DY[kCMax * kLd];
  float red[2 * (kTT / 32)];
};

// Thread (sg, ng) of a [256 samples x 64 outputs] product owns outputs 8 ng +
// {0..7} and samples 4 sg + {0..3}, 128 + 4 sg + {0..3} (each activation load
// contiguous across the warp); accumulators are sample pairs, one packed FMA
// (two IEEE FP32 FMAs) per weight and pair.
__device__ __forceinline__ void load_samples(const float* __restrict__ row, int sg, float2 (&av)[4]) {
  const float4 a0 = *reinterpret_cast<const float4*>(row + 4 * sg);
  const float4 a1 = *reinterpret_cast<const float4*>(row + kTS / 2 + 4 * sg);
  av[0] = make_float2(a0.x, a0.y);
  av[1] = make_float2(a0.z, a0.w);
  av[2] = make_float2(a1.x, a1.y);
  av[3] = make_float2(a1.z, a1.w);
}

// acc[i][j] += sum_k A[k][samples i] * Bm[k][8 ng + j], Bm rows of kH floats
template <int K>
__device__ __forceinline__ void gemm_8x8(const float* __restrict__ A, const float* __restrict__ Bm, int sg, int ng,
                                         float2 (&acc)[4][8]) {
#pragma unroll 8
  for (int k = 0; k < K; ++k) {
    float2 av[4];
    load_samples(A + k * kLd, sg, av);
    const float4 b0 = *reinterpret_cast<const float4*>(Bm + k * kH + 8 * ng);
    const float4 b1 = *reinterpret_cast<const float4*>(Bm + k * kH + 8 * ng + 4);
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float2 w = make_float2(bv[j], bv[j]);
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i][j] = __ffma2_rn(av[i], w, acc[i][j]);
    }
  }
}

__device__ __forceinline__ void store_8x8(float* __restrict__ Out, int sg, int ng, const float2 (&v)[4][8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float* row = Out + (8 * ng + j) * kLd;
    *reinterpret_cast<float4*>(row + 4 * sg) = make_float4(v[0][j].x, v[0][j].y, v[1][j].x, v[1][j].y);
    *reinterpret_cast<float4*>(row + kTS / 2 + 4 * sg) = make_float4(v[2][j].x, v[2][j].y, v[3][j].x, v[3][j].y);
  }
}

// acc[j] = (sum over the tile's samples of A[ra + ...] * B[rb + ...]) for a
// thread's outputs: the sums along samples, 4 at a time (128-bit loads), even
// and odd samples in the two halves of a packed accumulator.
template <int NA, int NB>
__device__ __forceinline__ void sample_dots(const float* __restrict__ A, const int (&ra)[NA],
                                            const float* __restrict__ B, const int (&rb)[NB], float (&out)[NA][NB]) {
  float2 acc[NA][NB];
#pragma unroll
  for (int i = 0; i < NA; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[i][j] = make_float2(0.f, 0.f);
#pragma unroll 8
  for (int s = 0; s < kTS; s += 4) {
    float4 av[NA], bv[NB];
#pragma unroll
    for (int i = 0; i < NA; ++i) av[i] = *reinterpret_cast<const float4*>(A + ra[i] * kLd + s);
#pragma unroll
    for (int j = 0; j < NB; ++j) bv[j] = *reinterpret_cast<const float4*>(B + rb[j] * kLd + s);
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        acc[i][j] = __ffma2_rn(make_float2(av[i].x, av[i].y), make_float2(bv[j].x, bv[j].y), acc[i][j]);
        acc[i][j] = __ffma2_rn(make_float2(av[i].z, av[i].w), make_float2(bv[j].z, bv[j].w), acc[i][j]);
      }
  }
#pragma unroll
  for (int i = 0; i < NA; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) out[i][j] = acc[i][j].x + acc[i][j].y;
}

// k_train: persistent CTAs of 256 threads (one per SM) walk 256-sample tiles.
// Per tile: features and targets (thread = sample), H1, H2, outputs and dL/dy,
// then dW3 / D2, dW2 / D1, dW1 and the latent scatter.  Every thread keeps the
// running (Neumaier) sums of the weight-gradient entries it computes in
// registers across tiles -- the same entries every tile -- and writes them to
// the CTA's partial slots at the end.
// The 12 features of one sample (thread = sample): bilinear taps of the 4 latent
// levels (3 or, LV, 4 floats per texel).
template <bool LV>
__device__ __forceinline__ void sample_features(const TrainDev& a, float u, float v, float (&f)[kIn]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Taps T = clamp_taps(u, v, a.lw[k], a.lh[k], a.shift[k]);
    check_taps(T, (int64_t)a.lw[k] * a.lh[k], a);
    const float* L = a.lat[k];
    if constexpr (LV) {
      const float4* L4 = reinterpret_cast<const float4*>(L);
      const float4 q00 = __ldg(L4 + T.i00), q10 = __ldg(L4 + T.i10), q01 = __ldg(L4 + T.i01), q11 = __ldg(L4 + T.i11);
      f[3 * k + 0] = T.w00 * q00.x + T.w10 * q10.x + T.w01 * q01.x + T.w11 * q11.x;
      f[3 * k + 1] = T.w00 * q00.y + T.w10 * q10.y + T.w01 * q01.y + T.w11 * q11.y;
      f[3 * k + 2] = T.w00 * q00.z + T.w10 * q10.z + T.w01 * q01.z + T.w11 * q11.z;
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        f[3 * k + c] = T.w00 * __ldg(L + 3 * T.i00 + c) + T.w10 * __ldg(L + 3 * T.i10 + c) +
                       T.w01 * __ldg(L + 3 * T.i01 + c) + T.w11 * __ldg(L + 3 * T.i11 + c);
    }
  }
}

// The target's C channels at one sample (bilinear, clamp, no shift), written to
// out[c * stride]; TV: 16-byte reads of a texel stride that is a multiple of 4.
template <bool TV>
__device__ __forceinline__ void sample_target(const TrainDev& a, float u, float v, float* out, int stride) {
  Taps T = clamp_taps(u, v, a.tw, a.th, 0.f);
  check_taps(T, (int64_t)a.tw * a.th, a);
  const size_t ts = (size_t)a.ts;
  const int C = a.C;
  if constexpr (TV) {
    for (int q = 0; 4 * q < C; ++q) {
      const float4 v00 = __ldg(reinterpret_cast<const float4*>(a.target + T.i00 * ts) + q);
      const float4 v10 = __ldg(reinterpret_cast<const float4*>(a.target + T.i10 * ts) + q);
      const float4 v01 = __ldg(reinterpret_cast<const float4*>(a.target + T.i01 * ts) + q);
      const float4 v11 = __ldg(reinterpret_cast<const float4*>(a.target + T.i11 * ts) + q);
      out[(4 * q) * stride] = T.w00 * v00.x + T.w10 * v10.x + T.w01 * v01.x + T.w11 * v11.x;
      if (4 * q + 1 < C) out[(4 * q + 1) * stride] = T.w00 * v00.y + T.w10 * v10.y + T.w01 * v01.y + T.w11 * v11.y;
      if (4 * q + 2 < C) out[(4 * q + 2) * stride] = T.w00 * v00.z + T.w10 * v10.z + T.w01 * v01.z + T.w11 * v11.z;
      if (4 * q + 3 < C) out[(4 * q + 3) * stride] = T.w00 * v00.w + T.w10 * v10.w + T.w01 * v01.w + T.w11 * v11.w;
    }
  } else {
    for (int c = 0; c < C; ++c)
      out[c * stride] = T.w00 * __ldg(a.target + T.i00 * ts + c) + T.w10 * __ldg(a.target + T.i10 * ts + c) +
                        T.w01 * __ldg(a.target + T.i01 * ts + c) + T.w11 * __ldg(a.target + T.i11 * ts + c);
  }
}

// The same taps and arithmetic as sample_target with every load issued before
// the first blend (more registers; for k_gather, whose occupancy allows it).
template <bool TV>
__device__ __forceinline__ void sample_target_ilp(const TrainDev& a, float u, float v, float* out, int stride) {
  Taps T = clamp_taps(u, v, a.tw, a.th, 0.f);
  check_taps(T, (int64_t)a.tw * a.th, a);
  const size_t ts = (size_t)a.ts;
  const int C = a.C;
  if constexpr (TV) {
    // unrolled, loads first: every tap's loads are in flight at once
    float4 v[kCMax / 4][4];
#pragma unroll
    for (int q = 0; q < kCMax / 4; ++q)
      if (4 * q < C) {
        v[q][0] = __ldg(reinterpret_cast<const float4*>(a.target + T.i00 * ts) + q);
        v[q][1] = __ldg(reinterpret_cast<const float4*>(a.target + T.i10 * ts) + q);
        v[q][2] = __ldg(reinterpret_cast<const float4*>(a.target + T.i01 * ts) + q);
        v[q][3] = __ldg(reinterpret_cast<const float4*>(a.target + T.i11 * ts) + q);
      }
#pragma unroll
    for (int q = 0; q < kCMax / 4; ++q) {
      if (4 * q >= C) break;
      const float4 v00 = v[q][0], v10 = v[q][1], v01 = v[q][2], v11 = v[q][3];
      out[(4 * q) * stride] = T.w00 * v00.x + T.w10 * v10.x + T.w01 * v01.x + T.w11 * v11.x;
      if (4 * q + 1 < C) out[(4 * q + 1) * stride] = T.w00 * v00.y + T.w10 * v10.y + T.w01 * v01.y + T.w11 * v11.y;
      if (4 * q + 2 < C) out[(4 * q + 2) * stride] = T.w00 * v00.z + T.w10 * v10.z + T.w01 * v01.z + T.w11 * v11.z;
      if (4 * q + 3 < C) out[(4 * q + 3) * stride] = T.w00 * v00.w + T.w10 * v10.w + T.w01 * v01.w + T.w11 * v11.w;
    }
  } else {
    for (int c = 0; c < C; ++c)
      out[c * stride] = T.w00 * __ldg(a.target + T.i00 * ts + c) + T.w10 * __ldg(a.target + T.i10 * ts + c) +
                        T.w01 * __ldg(a.target + T.i01 * ts + c) + T.w11 * __ldg(a.target + T.i11 * ts + c);
  }
}

// Floats per pre-gathered sample: 12 features (+ the target's C channels padded
// to a multiple of 4 when the mode reads a target).
__host__ __device__ inline int gathered_floats(int C, bool target) { return kIn + (target ? 4 * ((C + 3) / 4) : 0); }

// k_gather: one thread per sample (many warps per SM, so the scattered latent
// and target taps of many samples are in flight at once) writes the sample's
// features and target channels as one contiguous record of a.rs floats, read
// back by k_train with 16-byte coalesced loads.  Same arithmetic as k_train's
// own gather.
template <bool LV, bool TV>
__global__ void __launch_bounds__(256) k_gather(TrainDev a, float* __restrict__ xt, int with_target) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.batch; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 uv = __ldg(reinterpret_cast<const float2*>(a.uv) + i);
    float f[kIn];
    sample_features<LV>(a, uv.x, uv.y, f);
    float4* r = reinterpret_cast<float4*>(xt + i * a.rs);
    r[0] = make_float4(f[0], f[1], f[2], f[3]);
    r[1] = make_float4(f[4], f[5], f[6], f[7]);
    r[2] = make_float4(f[8], f[9], f[10], f[11]);
    if (with_target) {
      float tv[kCMax];
#pragma unroll
      for (int c = 0; c < kCMax; ++c) tv[c] = 0.f;
      sample_target_ilp<TV>(a, uv.x, uv.y, tv, 1);
#pragma unroll
      for (int q = 0; q < kCMax / 4; ++q)
        if (4 * q < a.C) r[3 + q] = make_float4(tv[4 * q], tv[4 * q + 1], tv[4 * q + 2], tv[4 * q + 3]);
    }
  }
}

// LV: latents and latent gradients hold 4 floats per texel (16-byte texel
// loads and 16-byte gradient adds); TV: the target's texel stride is a multiple
// of 4 floats (16-byte loads).  Both give the same arithmetic as the 3-float /
// scalar forms, in the same order.  CP: output channels as the output layer's
// products run them (12 for C <= 12, else 16); the channels past C are zero
// weights and zero deltas, so CP changes no result, only the work.
template <int MODE, bool LV, bool TV, int CP>
__global__ void __launch_bounds__(kTT, 1) k_train(TrainDev a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int t = threadIdx.x;
  const int C = a.C;
  // stage the weights (both orientations), zero padding rows
  for (int e = t; e < kH * kIn; e += kTT) {
    const int j = e / kIn, i = e - j * kIn;
    S.W1[e] = a.W[e];
    S.W1t[i * kH + j] = a.W[e];
  }
  for (int e = t; e < kH * kH; e += kTT) {
    const int j = e / kH, i = e - j * kH;
    const float w = a.W[kH * kIn + e];
    S.W2[e] = w;
    S.W2t[i * kH + j] = w;
  }
  for (int e = t; e < kCMax * kH; e += kTT) {
    const int c = e / kH, i = e - c * kH;
    const float w = c < C ? a.W[kH * kIn + kH * kH + e] : 0.f;
    S.W3[e] = w;
    S.W3t[i * kCMax + c] = w;
  }
  for (int e = t; e < kH; e += kTT) {
    S.b1[e] = a.B[e];
    S.b2[e] = a.B[kH + e];
  }
  if (t < kCMax) S.b3[t] = t < C ? a.B[2 * kH + t] : 0.f;
  for (int e = t; e < kCMax * kLd; e += kTT) S.DY[e] = 0.f;
  __syncthreads();

  const int sg = t & 31, ng = t >> 5;  // product blocking (warp = output group)
  // Weight-gradient entries owned by this thread (the same every tile), chosen
  // so the rows a warp reads at one sample offset sit in distinct banks:
  //   dW2: rows w2o + 4p x cols w2i + 8q (p, q = 0..3), w2o = 16 (warp & 3) + (lane >> 3),
  //        w2i = 32 (warp >> 2) + (lane & 7)
  //   dW3: row 4 (warp & 3) + (lane >> 3) x cols w2i + 8q
  //   dW1: row 8 warp + (lane >> 2) x cols (lane & 3) + 4q (q = 0..2)
  //   biases: db1 (t < 64), db2 (64 <= t < 128), db3 (128 <= t < 144)
  const int lane = t & 31, warp = t >> 5;
  const int w2o = 16 * (warp & 3) + (lane >> 3), w2i = 32 * (warp >> 2) + (lane & 7);
  const int w3c = 4 * (warp & 3) + (lane >> 3);
  const int w1o = 8 * warp + (lane >> 2), w1i = lane & 3;
  float g2s[4][4] = {}, g2e[4][4] = {}, g1s[3] = {}, g1e[3] = {}, g3s[4] = {}, g3e[4] = {}, gbs = 0.f, gbe = 0.f;
  float loss_s = 0.f, loss_e = 0.f;
  const int64_t ntiles = (a.batch + kTS - 1) / kTS;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t sid = tile * kTS + t;
    const bool valid = sid < a.batch;
    const float2 uv = valid ? __ldg(reinterpret_cast<const float2*>(a.uv) + sid) : make_float2(0.f, 0.f);
    // ---- features and targets (thread = sample): pre-gathered records, or the taps here
    if (a.xt) {
      float4 r[3 + kCMax / 4];
      const float4* rec = reinterpret_cast<const float4*>(a.xt + (valid ? sid : 0) * a.rs);
#pragma unroll
      for (int q = 0; q < 3; ++q) r[q] = valid ? __ldg(rec + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (MODE == kModeTrain) {
#pragma unroll
        for (int q = 0; q < kCMax / 4; ++q)
          if (4 * q < C) r[3 + q] = valid ? __ldg(rec + 3 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        S.X[(4 * q + 0) * kLd + t] = r[q].x;
        S.X[(4 * q + 1) * kLd + t] = r[q].y;
        S.X[(4 * q + 2) * kLd + t] = r[q].z;
        S.X[(4 * q + 3) * kLd + t] = r[q].w;
      }
      if (MODE == kModeTrain) {
#pragma unroll
        for (int q = 0; q < kCMax / 4; ++q) {
          if (4 * q >= C) break;
          S.DY[(4 * q) * kLd + t] = r[3 + q].x;
          if (4 * q + 1 < C) S.DY[(4 * q + 1) * kLd + t] = r[3 + q].y;
          if (4 * q + 2 < C) S.DY[(4 * q + 2) * kLd + t] = r[3 + q].z;
          if (4 * q + 3 < C) S.DY[(4 * q + 3) * kLd + t] = r[3 + q].w;
        }
      }
    } else {
      float f[kIn];
      sample_features<LV>(a, uv.x, uv.y, f);
#pragma unroll
      for (int k = 0; k < kIn; ++k) S.X[k * kLd + t] = valid ? f[k] : 0.f;
      // targets (train mode) -> DY rows (turned into dL/dy below); rows >= C stay 0
      if (MODE == kModeTrain) sample_target<TV>(a, uv.x, uv.y, S.DY + t, kLd);
    }
    __syncthreads();
    // ---- H1 = ReLU(W1 x + b1), H2 = ReLU(W2 h1 + b2)
    {
      float2 acc[4][8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float b = S.b1[8 * ng + j];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = make_float2(b, b);
      }
      gemm_8x8<kIn>(S.X, S.W1t, sg, ng, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(fmaxf(acc[i][j].x, 0.f), fmaxf(acc[i][j].y, 0.f));
      store_8x8(S.H1, sg, ng, acc);
    }
    __syncthreads();
    {
      float2 acc[4][8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float b = S.b2[8 * ng + j];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = make_float2(b, b);
      }
      gemm_8x8<kH>(S.H1, S.W2t, sg, ng, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(fmaxf(acc[i][j].x, 0.f), fmaxf(acc[i][j].y, 0.f));
      store_8x8(S.H2, sg, ng, acc);
    }
    __syncthreads();
    // ---- y = W3 h2 + b3 (thread = sample), loss and dL/dy -> DY
    {
      float y[CP];
#pragma unroll
      for (int c = 0; c < CP; ++c) y[c] = S.b3[c];
#pragma unroll 4
      for (int k = 0; k < kH; ++k) {
        const float h = S.H2[k * kLd + t];
        const float4* w = reinterpret_cast<const float4*>(S.W3t + k * kCMax);
#pragma unroll
        for (int q = 0; q < CP / 4; ++q) {
          const float4 wq = w[q];
          y[4 * q + 0] = fmaf(wq.x, h, y[4 * q + 0]);
          y[4 * q + 1] = fmaf(wq.y, h, y[4 * q + 1]);
          y[4 * q + 2] = fmaf(wq.z, h, y[4 * q + 2]);
          y[4 * q + 3] = fmaf(wq.w, h, y[4 * q + 3]);
        }
      }
#pragma unroll
      for (int c = 0; c < CP; ++c) {
        if (c >= C) continue;
        float d = 0.f;
        if (MODE == kModeFwd) {
          if (valid) a.y[sid * C + c] = y[c];
        } else if (MODE == kModeBwd) {
          d = valid ? __ldg(a.dy + sid * C + c) : 0.f;
        } else {
          const float r = y[c] - S.DY[c * kLd + t];
          if (valid) {
            neumaier(loss_s, loss_e, a.loss_l1 ? fabsf(r) : r * r);
            d = a.loss_l1 ? (r > 0.f ? a.scale : (r < 0.f ? -a.scale : 0.f)) : 2.f * r * a.scale;
          }
        }
        if (MODE != kModeFwd) S.DY[c * kLd + t] = d;
      }
    }
    if (MODE == kModeFwd) {
      __syncthreads();
      continue;
    }
    __syncthreads();
    // ---- dW3 += DY H2^T, db3; D2 = (W3^T dy) * [h2 > 0] (into registers, then over H2)
    {
      const int ra[1] = {w3c};
      const int rb[4] = {w2i, w2i + 8, w2i + 16, w2i + 24};
      if (w3c < CP) {  // rows past CP are zero (warps 3 and 7 when CP = 12)
        float d3[1][4];
        sample_dots<1, 4>(S.DY, ra, S.H2, rb, d3);
#pragma unroll
        for (int q = 0; q < 4; ++q) neumaier(g3s[q], g3e[q], d3[0][q]);
      }
    }
    float2 acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(0.f, 0.f);
    gemm_8x8<CP>(S.DY, S.W3, sg, ng, acc);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float2 h[4];
      load_samples(S.H2 + (8 * ng + j) * kLd, sg, h);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        acc[i][j] = make_float2(h[i].x > 0.f ? acc[i][j].x : 0.f, h[i].y > 0.f ? acc[i][j].y : 0.f);
    }
    if (t >= 2 * kH && t < 2 * kH + kCMax) {  // db3
      float s = 0.f;
      const float* row = S.DY + (t - 2 * kH) * kLd;
      for (int i = 0; i < kTS; i += 4) {
        const float4 v = *reinterpret_cast<const float4*>(row + i);
        s += (v.x + v.y) + (v.z + v.w);
      }
      neumaier(gbs, gbe, s);
    }
    __syncthreads();
    store_8x8(S.H2, sg, ng, acc);  // H2 now holds D2
    __syncthreads();
    // ---- dW2 += D2 H1^T, db2; D1 = (W2^T d2) * [h1 > 0] (into registers, then over H1)
    {
      const int ra[4] = {w2o, w2o + 4, w2o + 8, w2o + 12};
      const int rb[4] = {w2i, w2i + 8, w2i + 16, w2i + 24};
      float d2[4][4];
      sample_dots<4, 4>(S.H2, ra, S.H1, rb, d2);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) neumaier(g2s[i][j], g2e[i][j], d2[i][j]);
    }
    if (t >= kH && t < 2 * kH) {  // db2
      float s = 0.f;
      const float* row = S.H2 + (t - kH) * kLd;
      for (int i = 0; i < kTS; i += 4) {
        const float4 v = *reinterpret_cast<const float4*>(row + i);
        s += (v.x + v.y) + (v.z + v.w);
      }
      neumaier(gbs, gbe, s);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(0.f, 0.f);
    gemm_8x8<kH>(S.H2, S.W2, sg, ng, acc);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float2 h[4];
      load_samples(S.H1 + (8 * ng + j) * kLd, sg, h);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        acc[i][j] = make_float2(h[i].x > 0.f ? acc[i][j].x : 0.f, h[i].y > 0.f ? acc[i][j].y : 0.f);
    }
    __syncthreads();
    store_8x8(S.H1, sg, ng, acc);  // H1 now holds D1
    __syncthreads();
    // ---- dW1 += D1 X^T, db1; dx = W1^T d1 (thread = sample) scattered into the latent gradients
    {
      const int ra[1] = {w1o};
      const int rb[3] = {w1i, w1i + 4, w1i + 8};
      float d1[1][3];
      sample_dots<1, 3>(S.H1, ra, S.X, rb, d1);
#pragma unroll
      for (int q = 0; q < 3; ++q) neumaier(g1s[q], g1e[q], d1[0][q]);
    }
    if (t < kH) {  // db1
      float s = 0.f;
      const float* row = S.H1 + t * kLd;
      for (int i = 0; i < kTS; i += 4) {
        const float4 v = *reinterpret_cast<const float4*>(row + i);
        s += (v.x + v.y) + (v.z + v.w);
      }
      neumaier(gbs, gbe, s);
    }
    {
      float dx[kIn];
#pragma unroll
      for (int i = 0; i < kIn; ++i) dx[i] = 0.f;
#pragma unroll 4
      for (int k = 0; k < kH; ++k) {
        const float d = S.H1[k * kLd + t];
        const float4* w = reinterpret_cast<const float4*>(S.W1 + k * kIn);
#pragma unroll
        for (int q = 0; q < kIn / 4; ++q) {
          const float4 wq = w[q];
          dx[4 * q + 0] = fmaf(wq.x, d, dx[4 * q + 0]);
          dx[4 * q + 1] = fmaf(wq.y, d, dx[4 * q + 1]);
          dx[4 * q + 2] = fmaf(wq.z, d, dx[4 * q + 2]);
          dx[4 * q + 3] = fmaf(wq.w, d, dx[4 * q + 3]);
        }
      }
      if (valid) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Taps T = clamp_taps(uv.x, uv.y, a.lw[k], a.lh[k], a.shift[k]);
          check_taps(T, (int64_t)a.lw[k] * a.lh[k], a);
          float* G = a.lgrad[k];
          if constexpr (LV) {
            float4* G4 = reinterpret_cast<float4*>(G);
            const float g0 = dx[3 * k], g1 = dx[3 * k + 1], g2 = dx[3 * k + 2];
            atomicAdd(G4 + T.i00, make_float4(T.w00 * g0, T.w00 * g1, T.w00 * g2, 0.f));
            atomicAdd(G4 + T.i10, make_float4(T.w10 * g0, T.w10 * g1, T.w10 * g2, 0.f));
            atomicAdd(G4 + T.i01, make_float4(T.w01 * g0, T.w01 * g1, T.w01 * g2, 0.f));
            atomicAdd(G4 + T.i11, make_float4(T.w11 * g0, T.w11 * g1, T.w11 * g2, 0.f));
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float g = dx[3 * k + c];
              atomicAdd(G + 3 * T.i00 + c, T.w00 * g);
              atomicAdd(G + 3 * T.i10 + c, T.w10 * g);
              atomicAdd(G + 3 * T.i01 + c, T.w01 * g);
              atomicAdd(G + 3 * T.i11 + c, T.w11 * g);
            }
          }
        }
      }
    }
    __syncthreads();  // X, H1 (D1), H2 (D2), DY are rewritten by the next tile
  }
  if (MODE == kModeFwd) return;
  // ---- per-CTA partials: gradient sums and the loss
  float* part = a.part + (size_t)blockIdx.x * kPart;
  {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int g = kGW2 + (w2o + 4 * i) * kH + w2i + 8 * j;
        part[2 * g] = g2s[i][j];
        part[2 * g + 1] = g2e[i][j];
      }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int g = kGW1 + w1o * kIn + w1i + 4 * q;
      part[2 * g] = g1s[q];
      part[2 * g + 1] = g1e[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int g = kGW3 + w3c * kH + w2i + 8 * q;
      part[2 * g] = g3s[q];
      part[2 * g + 1] = g3e[q];
    }
    if (t < 2 * kH + kCMax) {  // b1 [64], b2 [64], b3 [16] are contiguous slots
      part[2 * (kGB1 + t)] = gbs;
      part[2 * (kGB1 + t) + 1] = gbe;
    }
  }
  // loss: compensated block reduction (warp shuffles, then warps in fixed order)
  float ls = loss_s, le = loss_e;
  for (int off = 16; off; off >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, ls, off), oe = __shfl_xor_sync(0xffffffffu, le, off);
    neumaier(ls, le, os);
    le += oe;
  }
  if ((t & 31) == 0) {
    S.red[2 * (t >> 5)] = ls;
    S.red[2 * (t >> 5) + 1] = le;
  }
  __syncthreads();
  if (t == 0) {
    float s = 0.f, e = 0.f;
    for (int w = 0; w < kTT / 32; ++w) {
      neumaier(s, e, S.red[2 * w]);
      e += S.red[2 * w + 1];
    }
    part[2 * kGN] = s;
    part[2 * kGN + 1] = e;
  }
}

struct AdamHyper {
  float lr, b1, b2, eps, bc1, bc2;  // bc = 1 - beta^t
};

__device__ __forceinline__ void adam_update(float& p, float& m, float& v, float g, const AdamHyper& h) {
  m = h.b1 * m + (1.f - h.b1) * g;
  v = h.b2 * v + (1.f - h.b2) * g * g;
  const float mh = m / h.bc1, vh = v / h.bc2;
  p -= h.lr * mh / (sqrtf(vh) + h.eps);
}

// Sum of the CTA partials of every gradient slot (fixed order, compensated);
// writes the MLP gradients, the loss, and (train mode) the Adam update.
__global__ void k_reduce_adam(const float* __restrict__ part, int nparts, int C, float loss_scale, float* W, float* B,
                              float* gw, float* gb, float* mw, float* vw, float* mb, float* vb, float* loss,
                              int do_adam, AdamHyper h) {
  const int nw = kH * kIn + kH * kH + C * kH;
  const int nb = 2 * kH + C;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= nw + nb; e += gridDim.x * blockDim.x) {
    int slot;
    if (e == nw + nb) slot = kGN;  // the loss
    else if (e < kH * kIn) slot = kGW1 + e;
    else if (e < kH * kIn + kH * kH) slot = kGW2 + (e - kH * kIn);
    else if (e < nw) slot = kGW3 + (e - kH * kIn - kH * kH);
    else slot = kGB1 + (e - nw);  // b1 [64], b2 [64], b3 [C] are contiguous slots
    float s = 0.f, c = 0.f;
    for (int p = 0; p < nparts; ++p) {
      neumaier(s, c, part[(size_t)p * kPart + 2 * slot]);
      c += part[(size_t)p * kPart + 2 * slot + 1];
    }
    const float g = s + c;
    if (e == nw + nb) {
      if (loss) *loss = g * loss_scale;
      continue;
    }
    if (e < nw) {
      gw[e] = g;
      if (do_adam) adam_update(W[e], mw[e], vw[e], g, h);
    } else {
      gb[e - nw] = g;
      if (do_adam) adam_update(B[e - nw], mb[e - nw], vb[e - nw], g, h);
    }
  }
}

// Adam over several parameter arrays in one launch: segment blockIdx.y.
__global__ void k_adam_latent(AdamSegs S, AdamHyper h) {
  const AdamSeg q = S.seg[blockIdx.y];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q.n; i += (int64_t)gridDim.x * blockDim.x) {
    float pp = q.p[i], mm = q.m[i], vv = q.v[i];
    adam_update(pp, mm, vv, q.g[i], h);
    q.p[i] = pp;
    q.m[i] = mm;
    q.v[i] = vv;
  }
}

// Zeroes up to 4 float arrays in one launch: array blockIdx.y.
struct ZeroSeg {
  float* p;
  int64_t n;
};
struct ZeroSegs {
  ZeroSeg seg[4];
};
__global__ void k_zero(ZeroSegs Z) {
  const ZeroSeg z = Z.seg[blockIdx.y];
  float* p = z.p;
  const int64_t n = z.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0.f;
}

// ------------------------------------------------------------------ host

int latent_stride(const nbtc_train_args* A) {
  const int ls = A->latent_stride == 0 ? 3 : A->latent_stride;
  return ls == 3 || ls == 4 ? ls : 0;
}

nbtc_status launch_adam(nbtc_context* ctx, const nbtc_train_args* A, float lr, const AdamSegs& S, cudaStream_t s) {
  AdamHyper h;
  h.b1 = A->beta1;
  h.b2 = A->beta2;
  h.eps = A->eps;
  h.bc1 = (float)(1.0 - pow((double)A->beta1, (double)A->step));
  h.bc2 = (float)(1.0 - pow((double)A->beta2, (double)A->step));
  h.lr = lr;
  int64_t nmax = 0;
  for (int i = 0; i < S.count; ++i) nmax = S.seg[i].n > nmax ? S.seg[i].n : nmax;
  if (nmax <= 0) return NBTC_OK;
  int64_t gx = (nmax + 255) / 256;
  if (gx > ctx->sm_count * 16) gx = ctx->sm_count * 16;
  k_adam_latent<<<dim3((unsigned)gx, (unsigned)S.count), 256, 0, s>>>(S, h);
  return cuda_check(cudaGetLastError(), "launch k_adam_latent");
}

// The latent-gradient scatter of a training step alone: per sample, the four
// bilinear taps of every level receive the atomic adds k_train makes (16-byte
// vector adds with 4-float texels), of a constant gradient, with no other work.
// Timed by the caller, it measures the step's L2-atomic co-bound.
template <bool LV>
__global__ void __launch_bounds__(256) k_scatter_probe(TrainDev a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.batch) return;
  const float2 uv = __ldg(reinterpret_cast<const float2*>(a.uv) + i);
  const float g = 1e-3f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Taps T = clamp_taps(uv.x, uv.y, a.lw[k], a.lh[k], a.shift[k]);
    check_taps(T, (int64_t)a.lw[k] * a.lh[k], a);
    float* G = a.lgrad[k];
    if constexpr (LV) {
      float4* G4 = reinterpret_cast<float4*>(G);
      atomicAdd(G4 + T.i00, make_float4(T.w00 * g, T.w00 * g, T.w00 * g, 0.f));
      atomicAdd(G4 + T.i10, make_float4(T.w10 * g, T.w10 * g, T.w10 * g, 0.f));
      atomicAdd(G4 + T.i01, make_float4(T.w01 * g, T.w01 * g, T.w01 * g, 0.f));
      atomicAdd(G4 + T.i11, make_float4(T.w11 * g, T.w11 * g, T.w11 * g, 0.f));
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        atomicAdd(G + 3 * T.i00 + c, T.w00 * g);
        atomicAdd(G + 3 * T.i10 + c, T.w10 * g);
        atomicAdd(G + 3 * T.i01 + c, T.w01 * g);
        atomicAdd(G + 3 * T.i11 + c, T.w11 * g);
      }
    }
  }
}

static nbtc_status check_train(const nbtc_train_args* A, bool need_target, bool need_adam, bool need_latent_adam) {
  if (!A) return fail(NBTC_ERR_INVALID_ARG, "train args NULL");
  if (A->num_levels != 4) return fail(NBTC_ERR_UNSUPPORTED, "training takes 4 latent levels");
  const nbtc_mlp& m = A->mlp;
  if (m.num_layers != 3 || m.dims[0] != kIn || m.dims[1] != kH || m.dims[2] != kH || m.dims[3] < 1 ||
      m.dims[3] > kCMax)
    return fail(NBTC_ERR_UNSUPPORTED, "training takes an MLP [12, 64, 64, C], C <= 16");
  if (!m.weights || !m.biases) return fail(NBTC_ERR_INVALID_ARG, "mlp weights/biases NULL");
  const int ls = latent_stride(A);
  if (!ls) return fail(NBTC_ERR_INVALID_ARG, "latent_stride must be 3 or 4 (0 means 3)");
  for (int k = 0; k < 4; ++k) {
    if (!A->latents[k] || !A->latent_grads[k]) return fail(NBTC_ERR_INVALID_ARG, "latent or gradient NULL");
    if (ls == 4 && (!aligned(A->latents[k], 16) || !aligned(A->latent_grads[k], 16)))
      return fail(NBTC_ERR_INVALID_ARG, "latent_stride 4 wants 16-byte aligned latents and gradients");
    if (A->widths[k] < 1 || A->heights[k] < 1 || A->widths[k] > (1 << 15) || A->heights[k] > (1 << 15))
      return fail(NBTC_ERR_INVALID_ARG, "latent size out of range");
    if (need_latent_adam && (!A->latent_m[k] || !A->latent_v[k]))
      return fail(NBTC_ERR_INVALID_ARG, "latent moments NULL");
  }
  if (!A->grad_w || !A->grad_b) return fail(NBTC_ERR_INVALID_ARG, "grad_w / grad_b NULL");
  if (need_adam && (!A->m_w || !A->v_w || !A->m_b || !A->v_b)) return fail(NBTC_ERR_INVALID_ARG, "MLP moments NULL");
  if (need_adam && A->step < 1) return fail(NBTC_ERR_INVALID_ARG, "step must be >= 1");
  if (need_target && (!A->target || A->target_w < 1 || A->target_h < 1))
    return fail(NBTC_ERR_INVALID_ARG, "target missing");
  if (need_target && A->target_stride != 0 && A->target_stride < m.dims[3])
    return fail(NBTC_ERR_INVALID_ARG, "target_stride < C");
  if (A->batch < 0) return fail(NBTC_ERR_INVALID_ARG, "batch < 0");
  if (A->batch > 0 && (!A->uv || !aligned(A->uv, 8))) return fail(NBTC_ERR_INVALID_ARG, "uv NULL or not 8-byte aligned");
  if (A->loss != NBTC_LOSS_MSE && A->loss != NBTC_LOSS_L1) return fail(NBTC_ERR_INVALID_ARG, "unknown loss");
  // pointer kinds: every buffer the kernels touch is device memory or pinned host memory
  nbtc_status pk;
  for (int k = 0; k < 4; ++k) {
    // the gradients take atomic adds: device memory only
    if ((pk = need_readable(A->latents[k], "latents")) || (pk = need_device(A->latent_grads[k], "latent_grads")))
      return pk;
    if (need_latent_adam &&
        ((pk = need_readable(A->latent_m[k], "latent_m")) || (pk = need_readable(A->latent_v[k], "latent_v"))))
      return pk;
  }
  if ((pk = need_readable(m.weights, "mlp weights")) || (pk = need_readable(m.biases, "mlp biases")) ||
      (pk = need_readable(A->grad_w, "grad_w")) || (pk = need_readable(A->grad_b, "grad_b")))
    return pk;
  if (need_adam && ((pk = need_readable(A->m_w, "m_w")) || (pk = need_readable(A->v_w, "v_w")) ||
                    (pk = need_readable(A->m_b, "m_b")) || (pk = need_readable(A->v_b, "v_b"))))
    return pk;
  if (need_target && (pk = need_readable(A->target, "target"))) return pk;
  if (A->batch > 0 && (pk = need_readable(A->uv, "uv"))) return pk;
  return NBTC_OK;
}

static int train_grid(nbtc_context* ctx, int64_t batch) {
  int64_t tiles = (batch + kTS - 1) / kTS;
  int64_t g = tiles < ctx->sm_count ? tiles : ctx->sm_count;
  return g < 1 ? 1 : (int)g;
}

// Workspace: the per-CTA partial sums, then (from a 256-byte boundary) one
// pre-gathered record per sample.  A workspace that only holds the partials is
// accepted too; the step then gathers inside k_train.
static size_t partials_bytes(int grid) { return ((size_t)grid * kPart * sizeof(float) + 255) & ~(size_t)255; }

size_t train_workspace(nbtc_context* ctx, const nbtc_train_args* A) {
  const int C = A->mlp.num_layers == 3 ? A->mlp.dims[3] : kCMax;
  return partials_bytes(train_grid(ctx, A->batch)) +
         (size_t)(A->batch > 0 ? A->batch : 0) * gathered_floats(C, true) * sizeof(float);
}

static TrainDev make_dev(const nbtc_train_args* A, void* workspace) {
  TrainDev d;
  d.status = nullptr;
  d.plant = 0;
  for (int k = 0; k < 4; ++k) {
    d.lat[k] = A->latents[k];
    d.lgrad[k] = A->latent_grads[k];
    d.lw[k] = A->widths[k];
    d.lh[k] = A->heights[k];
    d.shift[k] = A->shifts[k];
  }
  d.W = A->mlp.weights;
  d.B = A->mlp.biases;
  d.target = A->target;
  d.tw = A->target_w;
  d.th = A->target_h;
  d.ts = A->target_stride ? A->target_stride : A->mlp.dims[3];
  d.uv = A->uv;
  d.batch = A->batch;
  d.C = A->mlp.dims[3];
  d.scale = A->batch > 0 ? (float)(1.0 / ((double)A->batch * d.C)) : 0.f;
  d.loss_l1 = A->loss == NBTC_LOSS_L1;
  d.dy = nullptr;
  d.y = nullptr;
  d.part = static_cast<float*>(workspace);
  d.xt = nullptr;
  d.rs = 0;
  return d;
}

template <bool LV, bool TV>
static nbtc_status launch_k_gather(nbtc_context* ctx, const TrainDev& d, float* xt, int with_target, cudaStream_t s) {
  int64_t g = (d.batch + 255) / 256;
  if (g > (int64_t)ctx->sm_count * 8) g = (int64_t)ctx->sm_count * 8;
  k_gather<LV, TV><<<(int)g, 256, 0, s>>>(d, xt, with_target);
  return cuda_check(cudaGetLastError(), "launch k_gather");
}

// Pre-gathers the batch's samples into the workspace when it has room for them.
static nbtc_status pre_gather(nbtc_context* ctx, const nbtc_train_args* A, TrainDev& d, int grid, bool target,
                              void* workspace, size_t workspace_bytes, cudaStream_t s) {
  const int rs = gathered_floats(d.C, target);
  const size_t off = partials_bytes(grid);
  if (A->batch <= 0 || workspace_bytes < off + (size_t)A->batch * rs * sizeof(float)) return NBTC_OK;
  float* xt = reinterpret_cast<float*>(static_cast<char*>(workspace) + off);
  d.rs = rs;
  const bool lv = latent_stride(A) == 4, tv = target && d.ts % 4 == 0 && aligned(d.target, 16);
  nbtc_status st = lv ? (tv ? launch_k_gather<true, true>(ctx, d, xt, target, s)
                            : launch_k_gather<true, false>(ctx, d, xt, target, s))
                      : (tv ? launch_k_gather<false, true>(ctx, d, xt, target, s)
                            : launch_k_gather<false, false>(ctx, d, xt, target, s));
  if (st) return st;
  d.xt = xt;
  return NBTC_OK;
}

template <int MODE, bool LV, bool TV>
static nbtc_status launch_k_train(const TrainDev& d, int grid, cudaStream_t s) {
  auto kern = d.C <= 12 ? k_train<MODE, LV, TV, 12> : k_train<MODE, LV, TV, 16>;
  nbtc_status st = cuda_check(
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)), "smem attr");
  if (st) return st;
  kern<<<grid, kTT, sizeof(TrainSmem), s>>>(d);
  return cuda_check(cudaGetLastError(), "launch k_train");
}

// lv: 4-float latent texels; the 16-byte target path needs a target stride that
// is a multiple of 4 floats and a 16-byte aligned target (train mode only).
template <int MODE>
static nbtc_status launch_train_kernel(const nbtc_train_args* A, const TrainDev& d, int grid, cudaStream_t s) {
  const bool lv = latent_stride(A) == 4;
  if constexpr (MODE == kModeTrain) {
    const bool tv = d.ts % 4 == 0 && aligned(d.target, 16);
    if (lv) return tv ? launch_k_train<MODE, true, true>(d, grid, s) : launch_k_train<MODE, true, false>(d, grid, s);
    return tv ? launch_k_train<MODE, false, true>(d, grid, s) : launch_k_train<MODE, false, false>(d, grid, s);
  } else {
    return lv ? launch_k_train<MODE, true, false>(d, grid, s) : launch_k_train<MODE, false, false>(d, grid, s);
  }
}

// Zeroes the latent gradients (this batch's gradient, not an accumulation).
static nbtc_status zero_latent_grads(nbtc_context* ctx, const nbtc_train_args* A, cudaStream_t s) {
  ZeroSegs Z;
  int64_t nmax = 0;
  for (int k = 0; k < 4; ++k) {
    Z.seg[k] = ZeroSeg{A->latent_grads[k], latent_stride(A) * (int64_t)A->widths[k] * A->heights[k]};
    nmax = Z.seg[k].n > nmax ? Z.seg[k].n : nmax;
  }
  int64_t gx = (nmax + 255) / 256;
  if (gx > ctx->sm_count * 16) gx = ctx->sm_count * 16;
  k_zero<<<dim3((unsigned)gx, 4u), 256, 0, s>>>(Z);
  return cuda_check(cudaGetLastError(), "launch k_zero");
}

nbtc_status train_step_impl(nbtc_context* ctx, const nbtc_train_args* A, float* loss, cudaStream_t s, int mode,
                            const float* dy, float* y, void* workspace, size_t workspace_bytes) {
  // mode 3: the full step without the latent Adam (the QAT step updates its raw parameters itself)
  const bool latent_adam = mode == kModeTrain;
  if (mode == 3) mode = kModeTrain;
  nbtc_status st = check_train(A, mode == kModeTrain, mode == kModeTrain, latent_adam);
  if (st) return st;
  const int grid = train_grid(ctx, A->batch);
  TrainDev d = make_dev(A, workspace);
  d.status = ctx->status_dev;
  d.plant = ctx->check_plant;
  if (mode == kModeFwd) {
    if (A->batch == 0) return NBTC_OK;
    if (!y) return fail(NBTC_ERR_INVALID_ARG, "y is NULL");
    if ((st = need_readable(y, "y"))) return st;
    d.y = y;
    return launch_train_kernel<kModeFwd>(A, d, grid, s);
  }
  if (!workspace || !aligned(workspace, 16) || workspace_bytes < (size_t)grid * kPart * sizeof(float))
    return fail(NBTC_ERR_INVALID_ARG, "workspace NULL, misaligned or too small");
  if ((st = need_device(workspace, "workspace"))) return st;
  if (loss && (st = need_readable(loss, "loss"))) return st;
  if (mode == kModeBwd && dy && (st = need_readable(dy, "dy"))) return st;
  if ((st = zero_latent_grads(ctx, A, s))) return st;
  if ((st = pre_gather(ctx, A, d, grid, mode == kModeTrain, workspace, workspace_bytes, s))) return st;
  if (mode == kModeBwd) {
    if (!dy && A->batch > 0) return fail(NBTC_ERR_INVALID_ARG, "dy is NULL");
    d.dy = dy;
    if ((st = launch_train_kernel<kModeBwd>(A, d, grid, s))) return st;
  } else if (d.xt && ctx->train_tc) {
    // pre-gathered records: the tensor-core kernel (two 128-sample warpgroups per CTA)
    auto kern = latent_stride(A) == 4 ? k_train_tc<true> : k_train_tc<false>;
    if ((st = cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, ttc::kSmem),
                         "smem attr")))
      return st;
    kern<<<grid, ttc::kWG * 160, ttc::kSmem, s>>>(d);
    if ((st = cuda_check(cudaGetLastError(), "launch k_train_tc"))) return st;
  } else {
    if ((st = launch_train_kernel<kModeTrain>(A, d, grid, s))) return st;
  }
  const int C = A->mlp.dims[3];
  AdamHyper h;
  h.b1 = A->beta1;
  h.b2 = A->beta2;
  h.eps = A->eps;
  h.bc1 = (float)(1.0 - pow((double)A->beta1, (double)A->step));
  h.bc2 = (float)(1.0 - pow((double)A->beta2, (double)A->step));
  h.lr = A->lr_mlp;
  const float loss_scale = A->batch > 0 ? (float)(1.0 / ((double)A->batch * C)) : 0.f;
  float* W = const_cast<float*>(A->mlp.weights);
  float* Bv = const_cast<float*>(A->mlp.biases);
  const int np = kH * kIn + kH * kH + C * kH + 2 * kH + C + 1;
  k_reduce_adam<<<(np + 255) / 256, 256, 0, s>>>(static_cast<float*>(workspace), grid, C, loss_scale, W, Bv, A->grad_w,
                                                 A->grad_b, A->m_w, A->v_w, A->m_b, A->v_b, loss,
                                                 mode == kModeTrain ? 1 : 0, h);
  if ((st = cuda_check(cudaGetLastError(), "launch k_reduce_adam"))) return st;
  if (latent_adam) {  // all four levels in one launch
    AdamSegs S;
    S.count = 4;
    for (int k = 0; k < 4; ++k)
      S.seg[k] = AdamSeg{A->latents[k], A->latent_grads[k], A->latent_m[k], A->latent_v[k],
                         latent_stride(A) * (int64_t)A->widths[k] * A->heights[k]};
    if ((st = launch_adam(ctx, A, A->lr_latent, S, s))) return st;
  }
  return NBTC_OK;
}

}  // namespace nbtc

// ------------------------------------------------------------------ allocation-free training step
//
// nbtc_train_step_noalloc is for callers that must not allocate device memory
// themselves and cannot let a library do it either: renderers and engines that
// reserve their whole GPU memory budget up front and sub-allocate it
// themselves, plugin hosts whose execute callbacks forbid allocation, and
// real-time loops where cudaMalloc / cudaFree may synchronise the device and
// stall a frame.  Such callers cannot provide the training workspace, and
// cannot create an nbtc_context either (nbtc_create allocates its status word).
//
// The step's only scratch -- the per-CTA partial gradient sums that the
// reduction kernel adds up -- lives instead in the file-scope device array
// below, which every GPU that loads this library holds until the process
// exits.  It is sized for kNoAllocMaxCtas CTAs (one per SM); a device with more
// SMs than that is rejected.  Every kernel writes each slot it later reads, so
// nothing in the array needs clearing between calls.  All calls share the one
// array: two of these steps in flight on the GPU at the same time (different
// streams, or different host threads) race on it and corrupt each other's
// gradients, so callers must order them.
namespace nbtc {
namespace {
constexpr int kNoAllocMaxCtas = 160;
constexpr int kNoAllocMaxDevices = 64;
__device__ __align__(256) float g_noalloc_partials[kNoAllocMaxCtas * kPart];  // 7.72 MB
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};
}  // namespace

}  // namespace nbtc

extern "C" nbtc_status nbtc_train_step_noalloc(const nbtc_train_args* args, float* loss_dev, void* stream) {
  NBTC_RANGE();
  using namespace nbtc;
  if (!args) return fail(NBTC_ERR_INVALID_ARG, "args NULL");
  int dev = 0;
  nbtc_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st) return st;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(NBTC_ERR_UNSUPPORTED, "device index beyond 63");
  void* scratch = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name of
    // the array is not a device address; ask the runtime for it
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if ((st = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_partials), "cudaGetSymbolAddress(scratch)"))) return st;
      g_noalloc_addr[dev] = p;
    }
    scratch = g_noalloc_addr[dev];
  }
  int sms = 0;
  if ((st = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count"))) return st;
  nbtc_context local;  // on the stack: device and SM count only, no status word
  local.device = dev;
  local.sm_count = sms;
  const int64_t tiles = (args->batch + kTS - 1) / kTS;
  const int64_t grid = tiles < sms ? tiles : sms;
  if (grid > kNoAllocMaxCtas)
    return fail(NBTC_ERR_UNSUPPORTED, "nbtc_train_step_noalloc: the device has " + std::to_string(sms) +
                                          " SMs; its fixed scratch holds partial sums for at most 160");
  return train_step_impl(&local, args, loss_dev, (cudaStream_t)stream, 2, nullptr, nullptr, scratch,
                         sizeof(g_noalloc_partials));
}

extern "C" nbtc_status nbtc_probe_scatter(nbtc_context* ctx, const nbtc_train_args* args, void* stream) {
  NBTC_RANGE();
  using namespace nbtc;
  nbtc_status st;
  if ((st = enter(ctx))) return st;
  if ((st = check_train(args, false, false, false))) return st;
  if (args->batch == 0) return NBTC_OK;
  TrainDev d = make_dev(args, nullptr);
  d.status = ctx->status_dev;
  d.plant = ctx->check_plant;
  const unsigned grid = (unsigned)((args->batch + 255) / 256);
  if (latent_stride(args) == 4)
    k_scatter_probe<true><<<grid, 256, 0, (cudaStream_t)stream>>>(d);
  else
    k_scatter_probe<false><<<grid, 256, 0, (cudaStream_t)stream>>>(d);
  return cuda_check(cudaGetLastError(), "launch k_scatter_probe");
}
