// FP32 SIMT form of the fused decode (template; instantiated in
// decode_fp32.cu and calib_fp32.cu).
//
// The paper's "software FMA" path (Sec. 5, Table 2): BC1 fetch + decode +
// bilinear sampling of the 4 latent levels, then the MLP with true FP32 fused
// multiply-adds.  Each thread decodes TPT texels at once; with TPT = 2 every
// multiply-add is a packed FP32x2 FMA whose weight operand (duplicated in
// shared memory) is shared by the texel pair.
#pragma once

#include "host.h"

namespace nbtc {

template <int TPT>
struct Vec;

template <>
struct Vec<1> {
  using T = float;
  static __device__ __forceinline__ T fma(T a, T b, T c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ T relu(T x) { return fmaxf(x, 0.f); }
  static __device__ __forceinline__ T splat(float x) { return x; }
  static __device__ __forceinline__ float absmax(T x) { return fabsf(x); }
  static __device__ __forceinline__ float lane(T x, int) { return x; }
  static __device__ __forceinline__ void set(T& x, int, float v) { x = v; }
};

template <>
struct Vec<2> {
  using T = float2;
  static __device__ __forceinline__ T fma(T a, T b, T c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ T relu(T x) { return make_float2(fmaxf(x.x, 0.f), fmaxf(x.y, 0.f)); }
  static __device__ __forceinline__ T splat(float x) { return make_float2(x, x); }
  static __device__ __forceinline__ float absmax(T x) { return fmaxf(fabsf(x.x), fabsf(x.y)); }
  static __device__ __forceinline__ float lane(T x, int q) { return q ? x.y : x.x; }
  static __device__ __forceinline__ void set(T& x, int q, float v) {
    if (q) x.y = v; else x.x = v;
  }
};

constexpr int kNin = 12;

// Shared-memory image of the network: per layer W as [in][out] (input-major,
// so one input's weights for consecutive outputs are contiguous), then biases.
template <int D, int NHID, int NOUT>
struct Fp32Layout {
  static constexpr int nlayers = NHID + 1;
  static __host__ __device__ constexpr int in_dim(int l) { return l == 0 ? kNin : D; }
  static __host__ __device__ constexpr int out_dim(int l) { return l == NHID ? NOUT : D; }
  static __host__ __device__ constexpr int w_off(int l) {
    int o = 0;
    for (int k = 0; k < l; ++k) o += in_dim(k) * out_dim(k);
    return o;
  }
  static constexpr int w_total = w_off(nlayers);
  static __host__ __device__ constexpr int b_off(int l) {
    int o = w_total;
    for (int k = 0; k < l; ++k) o += out_dim(k);
    return o;
  }
  static constexpr int total = b_off(nlayers);
};

// y = ReLU(W x + b), all outputs at once (input-outer loop: OUT independent chains).
template <int IN, int OUT, class VV>
__device__ __forceinline__ void dense_relu(const typename VV::T* __restrict__ W,
                                           const typename VV::T* __restrict__ b,
                                           const typename VV::T (&x)[IN], typename VV::T (&y)[OUT]) {
#pragma unroll
  for (int j = 0; j < OUT; ++j) y[j] = b[j];
#pragma unroll
  for (int i = 0; i < IN; ++i) {
#pragma unroll
    for (int j = 0; j < OUT; ++j) y[j] = VV::fma(W[i * OUT + j], x[i], y[j]);
  }
#pragma unroll
  for (int j = 0; j < OUT; ++j) y[j] = VV::relu(y[j]);
}

// out = Wo ReLU(Wh x + bh) + bo, the hidden layer produced CH outputs at a time
// and consumed at once by the linear output layer (keeps registers low).
template <int IN, int DH, int NOUT, int CH, class VV>
__device__ __forceinline__ void dense_relu_out(const typename VV::T* __restrict__ Wh,
                                               const typename VV::T* __restrict__ bh,
                                               const typename VV::T* __restrict__ Wo,
                                               const typename VV::T* __restrict__ bo,
                                               const typename VV::T (&x)[IN],
                                               typename VV::T (&out)[NOUT], float& amax_h) {
  using T = typename VV::T;
#pragma unroll
  for (int k = 0; k < NOUT; ++k) out[k] = bo[k];
#pragma unroll 1
  for (int j0 = 0; j0 < DH; j0 += CH) {
    T acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = bh[j0 + c];
#pragma unroll
    for (int i = 0; i < IN; ++i) {
#pragma unroll
      for (int c = 0; c < CH; ++c) acc[c] = VV::fma(Wh[i * DH + j0 + c], x[i], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      acc[c] = VV::relu(acc[c]);
      amax_h = fmaxf(amax_h, VV::absmax(acc[c]));
#pragma unroll
      for (int k = 0; k < NOUT; ++k) out[k] = VV::fma(Wo[(j0 + c) * NOUT + k], acc[c], out[k]);
    }
  }
}

template <int D, int NHID, int NOUT, int TPT, bool CALIB>
__global__ void __launch_bounds__(256, 1)
    k_decode_fp32(DecodeArgs a, const float* __restrict__ gW, const float* __restrict__ gB,
                  int calib_step, float* __restrict__ absmax) {
  using VV = Vec<TPT>;
  using T = typename VV::T;
  using Lay = Fp32Layout<D, NHID, NOUT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);

  // Stage the weights: global W_l is [out][in]; shared is [in][out], each value
  // replicated TPT times.
  for (int l = 0; l < Lay::nlayers; ++l) {
    const int in = Lay::in_dim(l), out = Lay::out_dim(l);
    const float* src = gW + Lay::w_off(l);
    for (int e = threadIdx.x; e < in * out; e += blockDim.x) {
      const int j = e / in, i = e - j * in;
      sm[Lay::w_off(l) + i * out + j] = VV::splat(src[e]);
    }
  }
  for (int e = threadIdx.x; e < Lay::total - Lay::w_total; e += blockDim.x)
    sm[Lay::w_total + e] = VV::splat(gB[e]);
  __syncthreads();

  int64_t nunits = a.n, cw = 0;
  if (CALIB) {
    cw = (a.grid_w + calib_step - 1) / calib_step;
    nunits = cw * ((a.grid_h + calib_step - 1) / calib_step);
  }
  float amax[NHID + 1];
#pragma unroll
  for (int l = 0; l <= NHID; ++l) amax[l] = 0.f;

  const int64_t ngroups = (nunits + TPT - 1) / TPT;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    int64_t tex[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      int64_t k = g * TPT + q;
      if (k >= nunits) k = nunits - 1;
      if (CALIB) k = (k / cw) * calib_step * a.grid_w + (k % cw) * calib_step;
      tex[q] = k;
    }
    T x[kNin];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const float2 uv = texel_uv(a, tex[q]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float3 c = sample_bilinear(a.lv[k], uv.x, uv.y, a.wrap);
        VV::set(x[3 * k + 0], q, c.x);
        VV::set(x[3 * k + 1], q, c.y);
        VV::set(x[3 * k + 2], q, c.z);
      }
    }
    if (CALIB) {
#pragma unroll
      for (int i = 0; i < kNin; ++i) amax[0] = fmaxf(amax[0], VV::absmax(x[i]));
    }
    T out[NOUT];
    const T* W = sm;
    const T* B = sm + Lay::w_total;
    if constexpr (NHID == 1) {
      dense_relu_out<kNin, D, NOUT, 8, VV>(W + Lay::w_off(0), B + Lay::b_off(0) - Lay::w_total,
                                           W + Lay::w_off(1), B + Lay::b_off(1) - Lay::w_total, x, out,
                                           amax[1]);
    } else if constexpr (NHID == 2) {
      T h1[D];
      dense_relu<kNin, D, VV>(W + Lay::w_off(0), B + Lay::b_off(0) - Lay::w_total, x, h1);
      if (CALIB) {
#pragma unroll
        for (int i = 0; i < D; ++i) amax[1] = fmaxf(amax[1], VV::absmax(h1[i]));
      }
      dense_relu_out<D, D, NOUT, 8, VV>(W + Lay::w_off(1), B + Lay::b_off(1) - Lay::w_total,
                                        W + Lay::w_off(2), B + Lay::b_off(2) - Lay::w_total, h1, out,
                                        amax[2]);
    } else {
      static_assert(NHID == 3, "1..3 hidden layers");
      T h1[D], h2[D];
      dense_relu<kNin, D, VV>(W + Lay::w_off(0), B + Lay::b_off(0) - Lay::w_total, x, h1);
      dense_relu<D, D, VV>(W + Lay::w_off(1), B + Lay::b_off(1) - Lay::w_total, h1, h2);
      if (CALIB) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
          amax[1] = fmaxf(amax[1], VV::absmax(h1[i]));
          amax[2] = fmaxf(amax[2], VV::absmax(h2[i]));
        }
      }
      dense_relu_out<D, D, NOUT, 8, VV>(W + Lay::w_off(2), B + Lay::b_off(2) - Lay::w_total,
                                        W + Lay::w_off(3), B + Lay::b_off(3) - Lay::w_total, h2, out,
                                        amax[3]);
    }
    if (!CALIB) {
      float* o = reinterpret_cast<float*>(a.out);
#pragma unroll
      for (int q = 0; q < TPT; ++q) {
        if (g * TPT + q < nunits) {
#pragma unroll
          for (int k = 0; k < NOUT; ++k) o[tex[q] * NOUT + k] = VV::lane(out[k], q);
        }
      }
    }
  }
  if (CALIB) {
    // non-negative floats order like their bit patterns
#pragma unroll
    for (int l = 0; l <= NHID; ++l) {
      float m = amax[l];
      for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
      if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(absmax) + l, __float_as_int(m));
    }
  }
}

template <int D, int NHID, bool CALIB>
static nbtc_status launch_t(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, int step,
                            float* absmax, cudaStream_t s) {
  constexpr int TPT = (NHID >= 3) ? 1 : 2;
  using Lay = Fp32Layout<D, NHID, 9>;
  const size_t smem = sizeof(typename Vec<TPT>::T) * Lay::total;
  auto kern = k_decode_fp32<D, NHID, 9, TPT, CALIB>;
  nbtc_status st = cuda_check(
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attribute");
  if (st) return st;
  int64_t units = a.n;
  if (CALIB) units = (int64_t)((a.grid_w + step - 1) / step) * ((a.grid_h + step - 1) / step);
  const int64_t groups = (units + TPT - 1) / TPT;
  int64_t grid = (groups + 255) / 256;
  if (grid > ctx->sm_count) grid = ctx->sm_count;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, 256, smem, s>>>(a, mlp->weights, mlp->biases, step, absmax);
  return cuda_check(cudaGetLastError(), "launch k_decode_fp32");
}

template <bool CALIB>
static nbtc_status dispatch(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, int step,
                            float* absmax, cudaStream_t s) {
  const int L = mlp->num_layers;
  const int D = mlp->dims[1];
  for (int l = 1; l < L; ++l)
    if (mlp->dims[l] != D) return fail(NBTC_ERR_UNSUPPORTED, "hidden layers must share one width");
  if (mlp->dims[0] != kNin) return fail(NBTC_ERR_UNSUPPORTED, "decode kernels take 12 input features");
  if (mlp->dims[L] != 9) return fail(NBTC_ERR_UNSUPPORTED, "FP32 decode kernels output 9 channels");
#define NBTC_CASE(DD, HH) \
  if (D == DD && L - 1 == HH) return launch_t<DD, HH, CALIB>(ctx, a, mlp, step, absmax, s);
  NBTC_CASE(16, 1) NBTC_CASE(32, 1) NBTC_CASE(64, 1)
  NBTC_CASE(32, 2) NBTC_CASE(64, 2)
  NBTC_CASE(64, 3)
#undef NBTC_CASE
  return fail(NBTC_ERR_UNSUPPORTED, "no FP32 kernel for this MLP shape");
}

}  // namespace nbtc
