// Training step of the decoder on continuous latents (Sec. 3.2): forward
// (bilinear latent sampling + MLP 12-64-64-C), loss against the bilinearly
// sampled target, backward through the MLP into every latent texel, Adam.
//
// k_train: persistent CTAs of 256 threads walk 64-sample tiles.  Per tile all
// activations live in shared memory, feature-major ([k][sample], samples
// contiguous), and every dense product is a register-blocked SIMT FP32 GEMM
// (true FP32 FFMA; activations are recomputed per call, never stored to HBM).
// Weight/bias gradients: per-tile sums added into per-CTA running sums with
// Neumaier compensation, written to the workspace at the end; k_reduce_adam
// adds the CTA partials in a fixed order (compensated), writes the gradients
// and applies Adam.  Latent gradients: FP32 atomics (red.global.add).
#include <mutex>
#include <string>

#include "host.h"

namespace nbtc {

constexpr int kTS = 64;         // samples per tile
constexpr int kTT = 256;        // threads per CTA
constexpr int kH = 64;          // hidden width
constexpr int kIn = 12;         // features
constexpr int kCMax = 16;       // output channels (padded)
constexpr int kLd = kTS + 4;    // row stride of feature-major activations (16-byte rows, bank shift 4)

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
  const float* uv;
  int64_t batch;
  int C;
  float scale;      // 1 / (batch * C)
  int loss_l1;
  const float* dy;  // backward mode
  float* y;         // forward mode
  float* part;      // [gridDim.x][kPart]
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

struct TrainSmem {
  float W1[kH * kIn], W1t[kIn * kH], W2[kH * kH], W2t[kH * kH], W3[kCMax * kH], W3t[kH * kCMax];
  float b1[kH], b2[kH], b3[kCMax];
  float X[kIn * kLd], H1[kH * kLd], H2[kH * kLd], D2[kH * kLd], D1[kH * kLd], DY[kCMax * kLd];
  float gs[kGN], ge[kGN];  // running gradient sums (sum, compensation), owned per thread
  float red[2 * (kTT / 32)];
};

// [64 samples x 64 outputs] = A^T-products over K: acc[i][j] for samples 4sg+i,
// outputs 4ng+j, A feature-major [K][kLd], B [K][64] row-major.
template <int K>
__device__ __forceinline__ void gemm_4x4(const float* __restrict__ A, const float* __restrict__ Bm, int sg, int ng,
                                         float (&acc)[4][4]) {
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(A + k * kLd + 4 * sg);
    const float4 b = *reinterpret_cast<const float4*>(Bm + k * kH + 4 * ng);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}

__device__ __forceinline__ void store_4x4(float* __restrict__ Out, int sg, int ng, const float (&acc)[4][4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j)
    *reinterpret_cast<float4*>(Out + (4 * ng + j) * kLd + 4 * sg) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
}

template <int MODE>
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
  for (int e = t; e < kGN; e += kTT) S.gs[e] = S.ge[e] = 0.f;
  for (int e = t; e < kCMax * kLd; e += kTT) S.DY[e] = 0.f;
  __syncthreads();

  const int sg = t & 15, ng = t >> 4;  // GEMM blocking: samples 4sg.., outputs 4ng..
  const int ts = t & 63, tp = t >> 6;  // per-sample work: sample ts, part tp (0..3)
  float loss_s = 0.f, loss_e = 0.f;
  const int64_t ntiles = (a.batch + kTS - 1) / kTS;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t s0 = tile * kTS;
    const int64_t sid = s0 + ts;
    const bool valid = sid < a.batch;
    const float2 uv = valid ? __ldg(reinterpret_cast<const float2*>(a.uv) + sid) : make_float2(0.f, 0.f);
    // ---- features: part tp = latent level tp
    {
      const Taps T = clamp_taps(uv.x, uv.y, a.lw[tp], a.lh[tp], a.shift[tp]);
      const float* L = a.lat[tp];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float f = T.w00 * __ldg(L + 3 * T.i00 + c) + T.w10 * __ldg(L + 3 * T.i10 + c) +
                        T.w01 * __ldg(L + 3 * T.i01 + c) + T.w11 * __ldg(L + 3 * T.i11 + c);
        S.X[(3 * tp + c) * kLd + ts] = valid ? f : 0.f;
      }
    }
    // ---- targets (train mode), channels tp, tp+4, ...  -> DY rows (turned into dY below)
    if (MODE == kModeTrain) {
      const Taps T = clamp_taps(uv.x, uv.y, a.tw, a.th, 0.f);
      for (int c = tp; c < C; c += 4) {
        const float v = T.w00 * __ldg(a.target + (size_t)T.i00 * C + c) + T.w10 * __ldg(a.target + (size_t)T.i10 * C + c) +
                        T.w01 * __ldg(a.target + (size_t)T.i01 * C + c) + T.w11 * __ldg(a.target + (size_t)T.i11 * C + c);
        S.DY[c * kLd + ts] = v;
      }
    }
    __syncthreads();
    // ---- H1 = ReLU(W1 x + b1)
    {
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = S.b1[4 * ng + j];
      gemm_4x4<kIn>(S.X, S.W1t, sg, ng, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaxf(acc[i][j], 0.f);
      store_4x4(S.H1, sg, ng, acc);
    }
    __syncthreads();
    // ---- H2 = ReLU(W2 h1 + b2)
    {
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = S.b2[4 * ng + j];
      gemm_4x4<kH>(S.H1, S.W2t, sg, ng, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaxf(acc[i][j], 0.f);
      store_4x4(S.H2, sg, ng, acc);
    }
    __syncthreads();
    // ---- y = W3 h2 + b3 (channels tp, tp+4, ...), then dL/dy
    {
      float y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) y[q] = S.b3[tp + 4 * q];
#pragma unroll 8
      for (int k = 0; k < kH; ++k) {
        const float h = S.H2[k * kLd + ts];
#pragma unroll
        for (int q = 0; q < 4; ++q) y[q] = fmaf(S.W3t[k * kCMax + tp + 4 * q], h, y[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = tp + 4 * q;
        if (c >= C) continue;
        float d = 0.f;
        if (MODE == kModeFwd) {
          if (valid) a.y[sid * C + c] = y[q];
        } else if (MODE == kModeBwd) {
          d = valid ? __ldg(a.dy + sid * C + c) : 0.f;
        } else {
          const float r = y[q] - S.DY[c * kLd + ts];
          if (valid) {
            neumaier(loss_s, loss_e, a.loss_l1 ? fabsf(r) : r * r);
            d = a.loss_l1 ? (r > 0.f ? a.scale : (r < 0.f ? -a.scale : 0.f)) : 2.f * r * a.scale;
          }
        }
        if (MODE != kModeFwd) S.DY[c * kLd + ts] = d;
      }
    }
    if (MODE == kModeFwd) {
      __syncthreads();
      continue;
    }
    __syncthreads();
    // ---- D2 = (W3^T dy) * [h2 > 0]
    {
      float acc[4][4] = {};
#pragma unroll 4
      for (int k = 0; k < kCMax; ++k) {
        const float4 dv = *reinterpret_cast<const float4*>(S.DY + k * kLd + 4 * sg);
        const float4 w = *reinterpret_cast<const float4*>(S.W3 + k * kH + 4 * ng);
        const float av[4] = {dv.x, dv.y, dv.z, dv.w}, bv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 h = *reinterpret_cast<const float4*>(S.H2 + (4 * ng + j) * kLd + 4 * sg);
        acc[0][j] = h.x > 0.f ? acc[0][j] : 0.f;
        acc[1][j] = h.y > 0.f ? acc[1][j] : 0.f;
        acc[2][j] = h.z > 0.f ? acc[2][j] : 0.f;
        acc[3][j] = h.w > 0.f ? acc[3][j] : 0.f;
      }
      store_4x4(S.D2, sg, ng, acc);
    }
    __syncthreads();
    // ---- D1 = (W2^T d2) * [h1 > 0]
    {
      float acc[4][4] = {};
      gemm_4x4<kH>(S.D2, S.W2, sg, ng, acc);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 h = *reinterpret_cast<const float4*>(S.H1 + (4 * ng + j) * kLd + 4 * sg);
        acc[0][j] = h.x > 0.f ? acc[0][j] : 0.f;
        acc[1][j] = h.y > 0.f ? acc[1][j] : 0.f;
        acc[2][j] = h.z > 0.f ? acc[2][j] : 0.f;
        acc[3][j] = h.w > 0.f ? acc[3][j] : 0.f;
      }
      store_4x4(S.D1, sg, ng, acc);
    }
    __syncthreads();
    // ---- dx (level tp's 3 features) = W1^T d1, scattered into the latent gradient
    {
      float dx[3] = {0.f, 0.f, 0.f};
#pragma unroll 8
      for (int k = 0; k < kH; ++k) {
        const float d = S.D1[k * kLd + ts];
#pragma unroll
        for (int c = 0; c < 3; ++c) dx[c] = fmaf(S.W1[k * kIn + 3 * tp + c], d, dx[c]);
      }
      if (valid) {
        const Taps T = clamp_taps(uv.x, uv.y, a.lw[tp], a.lh[tp], a.shift[tp]);
        float* G = a.lgrad[tp];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          atomicAdd(G + 3 * T.i00 + c, T.w00 * dx[c]);
          atomicAdd(G + 3 * T.i10 + c, T.w10 * dx[c]);
          atomicAdd(G + 3 * T.i01 + c, T.w01 * dx[c]);
          atomicAdd(G + 3 * T.i11 + c, T.w11 * dx[c]);
        }
      }
    }
    // ---- weight gradients of this tile (sums over its samples), into the running sums
    {
      // dW2[j][i] += sum_s d2[j][s] h1[i][s]: thread owns j = 4 (t>>4).., i = 4 (t&15)..
      float acc[4][4] = {};
      const int jg = t >> 4, ig = t & 15;
#pragma unroll 4
      for (int s = 0; s < kTS; ++s) {
        float dv[4], hv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          dv[q] = S.D2[(4 * jg + q) * kLd + s];
          hv[q] = S.H1[(4 * ig + q) * kLd + s];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(dv[i], hv[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int g = kGW2 + (4 * jg + i) * kH + 4 * ig + j;
          neumaier(S.gs[g], S.ge[g], acc[i][j]);
        }
    }
    {
      // dW1[j][i] += sum_s d1[j][s] x[i][s]: thread owns j = t>>2, i = 3 (t&3) .. +2
      const int j = t >> 2, i0 = 3 * (t & 3);
      float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll 4
      for (int s = 0; s < kTS; ++s) {
        const float d = S.D1[j * kLd + s];
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[q] = fmaf(d, S.X[(i0 + q) * kLd + s], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) neumaier(S.gs[kGW1 + j * kIn + i0 + q], S.ge[kGW1 + j * kIn + i0 + q], acc[q]);
    }
    {
      // dW3[c][i] += sum_s dy[c][s] h2[i][s]: thread owns c = t>>4, i = 4 (t&15) .. +3
      const int c = t >> 4, i0 = 4 * (t & 15);
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
      for (int s = 0; s < kTS; ++s) {
        const float d = S.DY[c * kLd + s];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fmaf(d, S.H2[(i0 + q) * kLd + s], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) neumaier(S.gs[kGW3 + c * kH + i0 + q], S.ge[kGW3 + c * kH + i0 + q], acc[q]);
    }
    if (t < 2 * kH + kCMax) {
      // biases: db1 (t < 64), db2 (64 <= t < 128), db3 (t >= 128)
      const float* src = t < kH ? S.D1 + t * kLd : t < 2 * kH ? S.D2 + (t - kH) * kLd : S.DY + (t - 2 * kH) * kLd;
      float acc = 0.f;
#pragma unroll 8
      for (int s = 0; s < kTS; ++s) acc += src[s];
      neumaier(S.gs[kGB1 + t], S.ge[kGB1 + t], acc);
    }
    __syncthreads();
  }
  if (MODE == kModeFwd) return;
  // ---- per-CTA partials: gradient sums and the loss
  float* part = a.part + (size_t)blockIdx.x * kPart;
  for (int e = t; e < kGN; e += kTT) {
    part[2 * e] = S.gs[e];
    part[2 * e + 1] = S.ge[e];
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

__global__ void k_adam_latent(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                              float* __restrict__ v, int64_t n, AdamHyper h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float pp = p[i], mm = m[i], vv = v[i];
    adam_update(pp, mm, vv, g[i], h);
    p[i] = pp;
    m[i] = mm;
    v[i] = vv;
  }
}

// ------------------------------------------------------------------ host

nbtc_status launch_adam(nbtc_context* ctx, const nbtc_train_args* A, float lr, float* p, const float* g, float* m,
                        float* v, int64_t n, cudaStream_t s) {
  AdamHyper h;
  h.b1 = A->beta1;
  h.b2 = A->beta2;
  h.eps = A->eps;
  h.bc1 = (float)(1.0 - pow((double)A->beta1, (double)A->step));
  h.bc2 = (float)(1.0 - pow((double)A->beta2, (double)A->step));
  h.lr = lr;
  if (n <= 0) return NBTC_OK;
  int grid = (int)((n + 255) / 256);
  if (grid > ctx->sm_count * 16) grid = ctx->sm_count * 16;
  k_adam_latent<<<grid, 256, 0, s>>>(p, g, m, v, n, h);
  return cuda_check(cudaGetLastError(), "launch k_adam_latent");
}

static nbtc_status check_train(const nbtc_train_args* A, bool need_target, bool need_adam, bool need_latent_adam) {
  if (!A) return fail(NBTC_ERR_INVALID_ARG, "train args NULL");
  if (A->num_levels != 4) return fail(NBTC_ERR_UNSUPPORTED, "training takes 4 latent levels");
  const nbtc_mlp& m = A->mlp;
  if (m.num_layers != 3 || m.dims[0] != kIn || m.dims[1] != kH || m.dims[2] != kH || m.dims[3] < 1 ||
      m.dims[3] > kCMax)
    return fail(NBTC_ERR_UNSUPPORTED, "training takes an MLP [12, 64, 64, C], C <= 16");
  if (!m.weights || !m.biases) return fail(NBTC_ERR_INVALID_ARG, "mlp weights/biases NULL");
  for (int k = 0; k < 4; ++k) {
    if (!A->latents[k] || !A->latent_grads[k]) return fail(NBTC_ERR_INVALID_ARG, "latent or gradient NULL");
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
  if (A->batch < 0) return fail(NBTC_ERR_INVALID_ARG, "batch < 0");
  if (A->batch > 0 && (!A->uv || !aligned(A->uv, 8))) return fail(NBTC_ERR_INVALID_ARG, "uv NULL or not 8-byte aligned");
  if (A->loss != NBTC_LOSS_MSE && A->loss != NBTC_LOSS_L1) return fail(NBTC_ERR_INVALID_ARG, "unknown loss");
  return NBTC_OK;
}

static int train_grid(nbtc_context* ctx, int64_t batch) {
  int64_t tiles = (batch + kTS - 1) / kTS;
  int64_t g = tiles < ctx->sm_count ? tiles : ctx->sm_count;
  return g < 1 ? 1 : (int)g;
}

size_t train_workspace(nbtc_context* ctx, const nbtc_train_args* A) {
  return (size_t)train_grid(ctx, A->batch) * kPart * sizeof(float);
}

static TrainDev make_dev(const nbtc_train_args* A, void* workspace) {
  TrainDev d;
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
  d.uv = A->uv;
  d.batch = A->batch;
  d.C = A->mlp.dims[3];
  d.scale = A->batch > 0 ? (float)(1.0 / ((double)A->batch * d.C)) : 0.f;
  d.loss_l1 = A->loss == NBTC_LOSS_L1;
  d.dy = nullptr;
  d.y = nullptr;
  d.part = static_cast<float*>(workspace);
  return d;
}

template <int MODE>
static nbtc_status launch_train_kernel(nbtc_context* ctx, const TrainDev& d, int grid, cudaStream_t s) {
  auto kern = k_train<MODE>;
  nbtc_status st = cuda_check(
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)), "smem attr");
  if (st) return st;
  kern<<<grid, kTT, sizeof(TrainSmem), s>>>(d);
  return cuda_check(cudaGetLastError(), "launch k_train");
}

// Zeroes the latent gradients (this batch's gradient, not an accumulation).
static nbtc_status zero_latent_grads(const nbtc_train_args* A, cudaStream_t s) {
  for (int k = 0; k < 4; ++k) {
    nbtc_status st = cuda_check(
        cudaMemsetAsync(A->latent_grads[k], 0, sizeof(float) * 3 * (size_t)A->widths[k] * A->heights[k], s),
        "memset latent grads");
    if (st) return st;
  }
  return NBTC_OK;
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
  if (mode == kModeFwd) {
    if (A->batch == 0) return NBTC_OK;
    if (!y) return fail(NBTC_ERR_INVALID_ARG, "y is NULL");
    d.y = y;
    return launch_train_kernel<kModeFwd>(ctx, d, grid, s);
  }
  if (!workspace || !aligned(workspace, 16) || workspace_bytes < (size_t)grid * kPart * sizeof(float))
    return fail(NBTC_ERR_INVALID_ARG, "workspace NULL, misaligned or too small");
  if ((st = zero_latent_grads(A, s))) return st;
  if (mode == kModeBwd) {
    if (!dy && A->batch > 0) return fail(NBTC_ERR_INVALID_ARG, "dy is NULL");
    d.dy = dy;
    if ((st = launch_train_kernel<kModeBwd>(ctx, d, grid, s))) return st;
  } else {
    if ((st = launch_train_kernel<kModeTrain>(ctx, d, grid, s))) return st;
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
  if (latent_adam) {
    h.lr = A->lr_latent;
    for (int k = 0; k < 4; ++k) {
      const int64_t n = 3 * (int64_t)A->widths[k] * A->heights[k];
      int g = (int)((n + 255) / 256);
      if (g > ctx->sm_count * 16) g = ctx->sm_count * 16;
      k_adam_latent<<<g, 256, 0, s>>>(A->latents[k], A->latent_grads[k], A->latent_m[k], A->latent_v[k], n, h);
      if ((st = cuda_check(cudaGetLastError(), "launch k_adam_latent"))) return st;
    }
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
