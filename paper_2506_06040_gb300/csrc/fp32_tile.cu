// FP32 SIMT form of the fused decode as a tiled GEMM (hidden width D = 16, 32
// or 64).
//
// A CTA of 256 threads decodes tiles of 256 consecutive output texels of one
// row: the footprint feature stage (features.cuh) writes the 12 features of the
// tile feature-major into shared memory, then every layer is a register-blocked
// FP32 GEMM over the tile -- each thread owns D / 8 texels x 8 neurons (at
// D = 64: 64 FFMA per k step from two 128-bit activation loads and two
// broadcast 128-bit weight loads), hidden activations are rewritten in place
// between layers, and the output layer's rows are staged for coalesced 128-bit
// stores.  True FP32 FFMA
// throughout (the plain FP32 form of the method, Sec. 5 "software FMA").
#include "features.cuh"
#include "host.h"

namespace nbtc {

namespace {

constexpr int kT = 256;      // texels per tile = threads per CTA
constexpr int kIn = 12;
constexpr int kOutMax = 16;

template <int D, int NHID>
struct TileSmem {
  float w1t[kIn * D];                       // [k][n]
  float wht[(NHID > 1 ? NHID - 1 : 1) * D * D];  // hidden->hidden, [k][n] per layer
  float wot[D * kOutMax];                   // [k][c]
  float b[NHID * D + kOutMax];
  float x[kOutMax * kT];                    // features [k][texel]; reused as output staging [texel][c]
  float h[D * kT];                          // activations [n][texel]; also the column buffer
};
static_assert(16 * kT >= 4 * kColCap * 4, "the column buffer fits the smallest activation buffer");

// Thread (sg, ng) owns neurons 8 ng + {0..7} and TPT = D / 8 texels of the
// tile, laid out so each activation load is contiguous across the warp (no
// bank conflicts): TPT = 8 -> texels 4 sg + {0..3} and 128 + 4 sg + {0..3};
// TPT = 4 -> 4 sg + {0..3}; TPT = 2 -> 2 sg + {0, 1}.  Accumulators are texel
// pairs (FP32x2): acc[i][j] holds texels (2i, 2i+1) of the thread's TPT for
// neuron 8 ng + j, so every multiply-add is one packed FMA (two IEEE FP32 FMAs)
// and a weight feeds two texels per instruction.
template <int TPT>
__device__ __forceinline__ void load_pairs(const float* __restrict__ row, int sg, float2 (&av)[TPT / 2]) {
  if constexpr (TPT == 8) {
    const float4 a0 = *reinterpret_cast<const float4*>(row + 4 * sg);
    const float4 a1 = *reinterpret_cast<const float4*>(row + kT / 2 + 4 * sg);
    av[0] = make_float2(a0.x, a0.y);
    av[1] = make_float2(a0.z, a0.w);
    av[2] = make_float2(a1.x, a1.y);
    av[3] = make_float2(a1.z, a1.w);
  } else if constexpr (TPT == 4) {
    const float4 a0 = *reinterpret_cast<const float4*>(row + 4 * sg);
    av[0] = make_float2(a0.x, a0.y);
    av[1] = make_float2(a0.z, a0.w);
  } else {
    av[0] = *reinterpret_cast<const float2*>(row + 2 * sg);
  }
}

template <int TPT>
__device__ __forceinline__ void store_pairs(float* __restrict__ row, int sg, const float2 (&v)[TPT / 2]) {
  if constexpr (TPT == 8) {
    *reinterpret_cast<float4*>(row + 4 * sg) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    *reinterpret_cast<float4*>(row + kT / 2 + 4 * sg) = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
  } else if constexpr (TPT == 4) {
    *reinterpret_cast<float4*>(row + 4 * sg) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  } else {
    *reinterpret_cast<float2*>(row + 2 * sg) = v[0];
  }
}

template <int K, int D, int TPT>
__device__ __forceinline__ void gemm_block(const float* __restrict__ A, const float* __restrict__ Bt, int sg, int ng,
                                           float2 (&acc)[TPT / 2][8]) {
#pragma unroll 2
  for (int k = 0; k < K; ++k) {
    float2 av[TPT / 2];
    load_pairs<TPT>(A + k * kT, sg, av);
    const float4 b0 = *reinterpret_cast<const float4*>(Bt + k * D + 8 * ng);
    const float4 b1 = *reinterpret_cast<const float4*>(Bt + k * D + 8 * ng + 4);
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float2 w = make_float2(bv[j], bv[j]);
#pragma unroll
      for (int i = 0; i < TPT / 2; ++i) acc[i][j] = __ffma2_rn(av[i], w, acc[i][j]);
    }
  }
}

template <int TPT>
__device__ __forceinline__ void init_bias(const float* __restrict__ b, int ng, float2 (&acc)[TPT / 2][8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float v = b[8 * ng + j];
#pragma unroll
    for (int i = 0; i < TPT / 2; ++i) acc[i][j] = make_float2(v, v);
  }
}

template <int TPT>
__device__ __forceinline__ void store_relu(float* __restrict__ H, int sg, int ng, const float2 (&acc)[TPT / 2][8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float2 v[TPT / 2];
#pragma unroll
    for (int i = 0; i < TPT / 2; ++i) v[i] = make_float2(fmaxf(acc[i][j].x, 0.f), fmaxf(acc[i][j].y, 0.f));
    store_pairs<TPT>(H + (8 * ng + j) * kT, sg, v);
  }
}

template <int D, int NHID, int NO>
__global__ void __launch_bounds__(kT, 2) k_decode_fp32_tile(DecodeArgs a, const float* __restrict__ gW,
                                                           const float* __restrict__ gB, int nout, int footprint) {
  constexpr int TPT = D / 8;           // texels per thread
  constexpr int TG = kT / TPT;         // texel groups = threads per neuron group
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<D, NHID>& S = *reinterpret_cast<TileSmem<D, NHID>*>(smem_raw);
  const int t = threadIdx.x;
  // ---- weights: global [out][in] per layer -> shared [in][out]
  {
    int off = 0;
    for (int e = t; e < D * kIn; e += kT) {
      const int n = e / kIn, k = e - n * kIn;
      S.w1t[k * D + n] = gW[e];
    }
    off += D * kIn;
    for (int l = 0; l < NHID - 1; ++l) {
      for (int e = t; e < D * D; e += kT) {
        const int n = e / D, k = e - n * D;
        S.wht[l * D * D + k * D + n] = gW[off + e];
      }
      off += D * D;
    }
    for (int e = t; e < D * kOutMax; e += kT) {
      const int c = e / D, k = e - c * D;
      S.wot[k * kOutMax + c] = c < nout ? gW[off + c * D + k] : 0.f;
    }
    for (int e = t; e < NHID * D + kOutMax; e += kT) S.b[e] = e < NHID * D + nout ? gB[e] : 0.f;
  }
  __syncthreads();
  const int sg = t % TG, ng = t / TG;  // warp-uniform neuron group (weights broadcast), lane = texel group
  const int64_t tiles = (a.n + kT - 1) / kT;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t t0 = tile * kT;
    // ---- features -> x [k][texel]
    float f[12];
    if (footprint) {
      footprint_features<kT>(a, t0, t, reinterpret_cast<float4*>(S.h), 1, f);
    } else {
      const int64_t tex = t0 + t;
      direct_features(a, tex < a.n ? tex : a.n - 1, f);
    }
#pragma unroll
    for (int k = 0; k < kIn; ++k) S.x[k * kT + t] = f[k];
    __syncthreads();
    // ---- layer 1
    {
      float2 acc[TPT / 2][8];
      init_bias<TPT>(S.b, ng, acc);
      gemm_block<kIn, D, TPT>(S.x, S.w1t, sg, ng, acc);
      store_relu<TPT>(S.h, sg, ng, acc);
    }
    __syncthreads();
    // ---- hidden layers, in place
#pragma unroll 1
    for (int l = 0; l < NHID - 1; ++l) {
      float2 acc[TPT / 2][8];
      init_bias<TPT>(S.b + (l + 1) * D, ng, acc);
      gemm_block<D, D, TPT>(S.h, S.wht + l * D * D, sg, ng, acc);
      __syncthreads();
      store_relu<TPT>(S.h, sg, ng, acc);
      __syncthreads();
    }
    // ---- output layer: thread t -> texel t, NO (padded) channels as FP32x2 pairs; staged in x
    {
      float2 y[NO / 2];
#pragma unroll
      for (int c = 0; c < NO / 2; ++c) y[c] = make_float2(S.b[NHID * D + 2 * c], S.b[NHID * D + 2 * c + 1]);
#pragma unroll 4
      for (int k = 0; k < D; ++k) {
        const float hv = S.h[k * kT + t];
        const float2 h2 = make_float2(hv, hv);
        const float2* w = reinterpret_cast<const float2*>(S.wot + k * kOutMax);
#pragma unroll
        for (int c = 0; c < NO / 2; ++c) y[c] = __ffma2_rn(w[c], h2, y[c]);
      }
      // x (features) is free: every thread passed the layer-1 barrier
#pragma unroll
      for (int c = 0; c < NO / 2; ++c) {
        if (2 * c < nout) S.x[t * nout + 2 * c] = y[c].x;
        if (2 * c + 1 < nout) S.x[t * nout + 2 * c + 1] = y[c].y;
      }
    }
    __syncthreads();
    {
      float* out = reinterpret_cast<float*>(a.out);
      const int64_t valid = a.n - t0 < kT ? a.n - t0 : kT;
      if (valid == kT) {  // whole tile: 256 * nout contiguous floats, 16-byte aligned
        const float4* src = reinterpret_cast<const float4*>(S.x);
        float4* dst = reinterpret_cast<float4*>(out + t0 * nout);
        for (int e = t; e < kT * nout / 4; e += kT) dst[e] = src[e];
      } else {
        for (int e = t; e < valid * nout; e += kT) out[t0 * nout + e] = S.x[e];
      }
    }
    __syncthreads();
  }
}

template <int D, int NHID>
nbtc_status launch_tile(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, int footprint, cudaStream_t s) {
  const size_t smem = sizeof(TileSmem<D, NHID>);
  auto kern = mlp->dims[mlp->num_layers] <= 10 ? k_decode_fp32_tile<D, NHID, 10> : k_decode_fp32_tile<D, NHID, 16>;
  nbtc_status st =
      cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
  if (st) return st;
  int per_sm = 0;
  if ((st = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, smem), "occupancy")))
    return st;
  const int64_t tiles = (a.n + kT - 1) / kT;
  int64_t grid = (int64_t)ctx->sm_count * (per_sm > 0 ? per_sm : 1);
  if (grid > tiles) grid = tiles;
  kern<<<(int)grid, kT, smem, s>>>(a, mlp->weights, mlp->biases, mlp->dims[mlp->num_layers], footprint);
  return cuda_check(cudaGetLastError(), "launch k_decode_fp32_tile");
}

// ---- wide variant (hidden width 64, two hidden layers): one 512-thread CTA per
// SM on 512-texel tiles, which leaves shared memory for a pair-swapped copy of
// every weight row.  A thread's products then pair two texels with two neurons
// in "diagonal" and "anti-diagonal" packed FMAs -- (a0, a1) x (w0, w1) and
// (a0, a1) x (w1, w0) -- so no operand needs a broadcast register pair (no
// register moves in the inner loops).
constexpr int kTW = 512;   // texels per tile = threads per CTA
constexpr int kD = 64;     // hidden width of the wide kernel

template <int NHID>
struct WideSmem {
  float w1n[kIn * kD], w1s[kIn * kD];                                  // [k][n], pair-swapped copy
  float whn[(NHID > 1 ? NHID - 1 : 1) * kD * kD], whs[(NHID > 1 ? NHID - 1 : 1) * kD * kD];
  float won[kD * kOutMax], wos[kD * kOutMax];                          // output layer [k][c], swapped copy
  float b[NHID * kD + kOutMax], bs[NHID * kD + kOutMax];               // biases and their swapped pairs
  float x[kOutMax * kTW];                                              // features [k][texel]; output staging
  float h[kD * kTW];                                                   // activations [n][texel]; column buffer
};

// Thread (sg, ng) of a group tiling TW texels: texels 4 sg + {0..3} and
// TW / 2 + 4 sg + {0..3} (texel pairs i = 0..3), neurons 8 ng + {0..7} (neuron
// pairs p = 0..3).  dg[i][p] holds (t_i0 x n_p0, t_i1 x n_p1), ad[i][p] holds
// (t_i0 x n_p1, t_i1 x n_p0).
template <int K, int TW>
__device__ __forceinline__ void gemm_diag(const float* __restrict__ A, const float* __restrict__ Bn,
                                          const float* __restrict__ Bs, int sg, int ng, float2 (&dg)[4][4],
                                          float2 (&ad)[4][4]) {
#pragma unroll 2
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(A + k * TW + 4 * sg);
    const float4 a1 = *reinterpret_cast<const float4*>(A + k * TW + TW / 2 + 4 * sg);
    const float4 n0 = *reinterpret_cast<const float4*>(Bn + k * kD + 8 * ng);
    const float4 n1 = *reinterpret_cast<const float4*>(Bn + k * kD + 8 * ng + 4);
    const float4 s0 = *reinterpret_cast<const float4*>(Bs + k * kD + 8 * ng);
    const float4 s1 = *reinterpret_cast<const float4*>(Bs + k * kD + 8 * ng + 4);
    const float2 av[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                          make_float2(a1.z, a1.w)};
    const float2 wn[4] = {make_float2(n0.x, n0.y), make_float2(n0.z, n0.w), make_float2(n1.x, n1.y),
                          make_float2(n1.z, n1.w)};
    const float2 ws[4] = {make_float2(s0.x, s0.y), make_float2(s0.z, s0.w), make_float2(s1.x, s1.y),
                          make_float2(s1.z, s1.w)};
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        dg[i][p] = __ffma2_rn(av[i], wn[p], dg[i][p]);
        ad[i][p] = __ffma2_rn(av[i], ws[p], ad[i][p]);
      }
  }
}

__device__ __forceinline__ void init_diag(const float* __restrict__ b, const float* __restrict__ bs, int ng,
                                          float2 (&dg)[4][4], float2 (&ad)[4][4]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float2 bn = *reinterpret_cast<const float2*>(b + 8 * ng + 2 * p);
    const float2 bw = *reinterpret_cast<const float2*>(bs + 8 * ng + 2 * p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      dg[i][p] = bn;
      ad[i][p] = bw;
    }
  }
}

// ReLU and store: neuron n_p0 of texels (t_i0, t_i1) = (dg.x, ad.y); n_p1 = (ad.x, dg.y).
template <int TW>
__device__ __forceinline__ void store_diag(float* __restrict__ H, int sg, int ng, const float2 (&dg)[4][4],
                                           const float2 (&ad)[4][4]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float* r0 = H + (8 * ng + 2 * p) * TW;
    float* r1 = r0 + TW;
    *reinterpret_cast<float4*>(r0 + 4 * sg) = make_float4(fmaxf(dg[0][p].x, 0.f), fmaxf(ad[0][p].y, 0.f),
                                                          fmaxf(dg[1][p].x, 0.f), fmaxf(ad[1][p].y, 0.f));
    *reinterpret_cast<float4*>(r0 + TW / 2 + 4 * sg) = make_float4(fmaxf(dg[2][p].x, 0.f), fmaxf(ad[2][p].y, 0.f),
                                                                    fmaxf(dg[3][p].x, 0.f), fmaxf(ad[3][p].y, 0.f));
    *reinterpret_cast<float4*>(r1 + 4 * sg) = make_float4(fmaxf(ad[0][p].x, 0.f), fmaxf(dg[0][p].y, 0.f),
                                                          fmaxf(ad[1][p].x, 0.f), fmaxf(dg[1][p].y, 0.f));
    *reinterpret_cast<float4*>(r1 + TW / 2 + 4 * sg) = make_float4(fmaxf(ad[2][p].x, 0.f), fmaxf(dg[2][p].y, 0.f),
                                                                    fmaxf(ad[3][p].x, 0.f), fmaxf(dg[3][p].y, 0.f));
  }
}

// GR independent groups of kTW / GR threads, each on its own tiles of kTW / GR
// texels with its own activation / feature buffers and its own named barrier
// (id 1 + group): the groups drift out of phase, so one group's feature stage
// (integer BC1 decode, loads, blends) overlaps the other's FMA-bound layers.
// GR = 1 is one 512-texel group with block-wide barriers.
template <int NHID, int GR>
__global__ void __launch_bounds__(kTW, 1) k_decode_fp32_wide(DecodeArgs a, const float* __restrict__ gW,
                                                            const float* __restrict__ gB, int nout, int footprint) {
  constexpr int TW = kTW / GR;  // texels per tile = threads per group
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WideSmem<NHID>& S = *reinterpret_cast<WideSmem<NHID>*>(smem_raw);
  const int t = threadIdx.x;
  // ---- weights: global [out][in] per layer -> shared [in][out] and the pair-swapped copy
  {
    auto put = [](float* n, float* sw, int idx, float v) {
      n[idx] = v;
      sw[idx ^ 1] = v;
    };
    int off = 0;
    for (int e = t; e < kD * kIn; e += kTW) {
      const int nn = e / kIn, k = e - nn * kIn;
      put(S.w1n, S.w1s, k * kD + nn, gW[e]);
    }
    off += kD * kIn;
    for (int l = 0; l < NHID - 1; ++l) {
      for (int e = t; e < kD * kD; e += kTW) {
        const int nn = e / kD, k = e - nn * kD;
        put(S.whn + l * kD * kD, S.whs + l * kD * kD, k * kD + nn, gW[off + e]);
      }
      off += kD * kD;
    }
    for (int e = t; e < kD * kOutMax; e += kTW) {
      const int c = e / kD, k = e - c * kD;
      put(S.won, S.wos, k * kOutMax + c, c < nout ? gW[off + c * kD + k] : 0.f);
    }
    for (int e = t; e < NHID * kD + kOutMax; e += kTW) put(S.b, S.bs, e, e < NHID * kD + nout ? gB[e] : 0.f);
  }
  __syncthreads();
  const int g = GR == 1 ? 0 : t / TW, lt = GR == 1 ? t : t - g * TW;
  const int bar = 1 + g;
  auto group_sync = [&]() {
    if constexpr (GR == 1) {
      __syncthreads();
    } else {
      sm100::named_bar_sync(bar, TW);
    }
  };
  float* X = S.x + g * (kOutMax * TW);  // features [k][texel]; output staging
  float* Hb = S.h + g * (kD * TW);      // activations [n][texel]; column buffer
  // TW / 8 texel groups x 8 neuron groups (a warp spans one neuron group)
  const int sg = lt % (TW / 8), ng = lt / (TW / 8);
  const int64_t tiles = (a.n + TW - 1) / TW;
  for (int64_t tile = (int64_t)blockIdx.x * GR + g; tile < tiles; tile += (int64_t)gridDim.x * GR) {
    const int64_t t0 = tile * TW;
    // ---- features -> x [k][texel]
    float f[12];
    if (footprint) {
      footprint_features<TW>(a, t0, lt, reinterpret_cast<float4*>(Hb), bar, f);
    } else {
      const int64_t tex = t0 + lt;
      direct_features(a, tex < a.n ? tex : a.n - 1, f);
    }
#pragma unroll
    for (int k = 0; k < kIn; ++k) X[k * TW + lt] = f[k];
    group_sync();
    {
      float2 dg[4][4], ad[4][4];
      init_diag(S.b, S.bs, ng, dg, ad);
      gemm_diag<kIn, TW>(X, S.w1n, S.w1s, sg, ng, dg, ad);
      store_diag<TW>(Hb, sg, ng, dg, ad);
    }
    group_sync();
#pragma unroll 1
    for (int l = 0; l < NHID - 1; ++l) {
      float2 dg[4][4], ad[4][4];
      init_diag(S.b + (l + 1) * kD, S.bs + (l + 1) * kD, ng, dg, ad);
      gemm_diag<kD, TW>(Hb, S.whn + l * kD * kD, S.whs + l * kD * kD, sg, ng, dg, ad);
      group_sync();
      store_diag<TW>(Hb, sg, ng, dg, ad);
      group_sync();
    }
    // ---- output layer: threads lt < TW / 2 take texel pairs (2 lt, 2 lt + 1), 10 channels as 5 pairs
    if (lt < TW / 2) {
      float2 dg[5], ad[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        dg[c] = *reinterpret_cast<const float2*>(S.b + NHID * kD + 2 * c);
        ad[c] = *reinterpret_cast<const float2*>(S.bs + NHID * kD + 2 * c);
      }
#pragma unroll 8
      for (int k = 0; k < kD; ++k) {
        const float2 hv = *reinterpret_cast<const float2*>(Hb + k * TW + 2 * lt);
        const float2* wn = reinterpret_cast<const float2*>(S.won + k * kOutMax);
        const float2* ws = reinterpret_cast<const float2*>(S.wos + k * kOutMax);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          dg[c] = __ffma2_rn(hv, wn[c], dg[c]);
          ad[c] = __ffma2_rn(hv, ws[c], ad[c]);
        }
      }
      // texel 2 lt: channels (2c, 2c+1) = (dg.x, ad.x); texel 2 lt + 1: (ad.y, dg.y); staged in x
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        if (2 * c < nout) {
          X[(2 * lt) * nout + 2 * c] = dg[c].x;
          X[(2 * lt + 1) * nout + 2 * c] = ad[c].y;
        }
        if (2 * c + 1 < nout) {
          X[(2 * lt) * nout + 2 * c + 1] = ad[c].x;
          X[(2 * lt + 1) * nout + 2 * c + 1] = dg[c].y;
        }
      }
    }
    group_sync();
    {
      float* out = reinterpret_cast<float*>(a.out);
      const int64_t valid = a.n - t0 < TW ? a.n - t0 : TW;
      if (valid == TW) {  // whole tile: TW * nout contiguous floats, 16-byte aligned
        const float4* src = reinterpret_cast<const float4*>(X);
        float4* dst = reinterpret_cast<float4*>(out + t0 * nout);
        for (int e = lt; e < TW * nout / 4; e += TW) dst[e] = src[e];
      } else {
        for (int e = lt; e < valid * nout; e += TW) out[t0 * nout + e] = X[e];
      }
    }
    group_sync();
  }
}

template <int NHID, int GR>
nbtc_status launch_wide(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, int footprint, cudaStream_t s) {
  static_assert(NHID == 2, "the wide kernel is instantiated for two hidden layers");
  const size_t smem = sizeof(WideSmem<NHID>);
  auto kern = k_decode_fp32_wide<NHID, GR>;
  nbtc_status st =
      cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
  if (st) return st;
  const int64_t tiles = (a.n + kTW / GR - 1) / (kTW / GR);
  int64_t grid = ctx->sm_count;
  if (grid > (tiles + GR - 1) / GR) grid = (tiles + GR - 1) / GR;
  kern<<<(int)grid, kTW, smem, s>>>(a, mlp->weights, mlp->biases, mlp->dims[mlp->num_layers], footprint);
  return cuda_check(cudaGetLastError(), "launch k_decode_fp32_wide");
}

}  // namespace

// Tiled FP32 decode for MLPs [12, D, .., D, C <= 16] with D in {16, 32, 64}
// and 1-3 hidden layers; returns NBTC_ERR_UNSUPPORTED (without launching) for
// other shapes.
nbtc_status launch_decode_fp32_tile(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, cudaStream_t s) {
  const int L = mlp->num_layers;
  const int D = mlp->dims[1];
  if (mlp->dims[0] != kIn || L < 2 || L > 4 || mlp->dims[L] > kOutMax) return NBTC_ERR_UNSUPPORTED;
  if (D != 16 && D != 32 && D != 64) return NBTC_ERR_UNSUPPORTED;
  for (int l = 1; l < L; ++l)
    if (mlp->dims[l] != D) return NBTC_ERR_UNSUPPORTED;
  // footprint stage: tiles inside one output row, every level's span within the column buffer
  bool fp = a.uv == nullptr && (a.grid_w % kT) == 0;
  for (int k = 0; k < 4; ++k) fp = fp && (int64_t)(kT - 1) * a.lv[k].w / a.grid_w + 3 <= kColCap;
#define NBTC_TILE(DD)                                           \
  if (D == DD) {                                                \
    switch (L - 1) {                                            \
      case 1: return launch_tile<DD, 1>(ctx, a, mlp, fp, s);    \
      case 2: return launch_tile<DD, 2>(ctx, a, mlp, fp, s);    \
      default: return launch_tile<DD, 3>(ctx, a, mlp, fp, s);   \
    }                                                           \
  }
  // hidden width 64 with 2 hidden layers and at most 10 outputs: the wide kernel
  // (measured faster there; with one hidden layer the 256-texel tiles win)
  if (D == 64 && L - 1 == 2 && mlp->dims[L] <= 10) {
    const int gr = ctx->fp32_groups == 1 ? 1 : 2;
    const int tw = kTW / gr;
    bool fpw = a.uv == nullptr && (a.grid_w % tw) == 0;
    for (int k = 0; k < 4; ++k) fpw = fpw && (int64_t)(tw - 1) * a.lv[k].w / a.grid_w + 3 <= kColCap;
    if (fpw || !fp) return gr == 1 ? launch_wide<2, 1>(ctx, a, mlp, fpw, s) : launch_wide<2, 2>(ctx, a, mlp, fpw, s);
  }
  NBTC_TILE(16)
  NBTC_TILE(32)
  NBTC_TILE(64)
#undef NBTC_TILE
  return NBTC_ERR_UNSUPPORTED;
}

}  // namespace nbtc
