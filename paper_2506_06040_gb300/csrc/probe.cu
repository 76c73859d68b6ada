// Measurement probe: a kernel with a known amount of FP32 FFMA work, timed by
// the caller, which gives the FP32 SIMT roofline that the FP32 decode and the
// training step are reported against (a measured peak instead of one derived
// from unit counts and the clock).
#include "host.h"

namespace nbtc {

// 16 independent multiply-add chains per thread (8 packed FP32x2 FMAs when
// PACKED): x <- a x + b, iterated; with 0 < a < 1 the values stay bounded.
template <bool PACKED>
__global__ void __launch_bounds__(256) k_ffma_probe(float* out, int iters, float a, float b) {
  float x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = 1e-3f * (float)threadIdx.x + (float)i;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
    if constexpr (PACKED) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 r = __ffma2_rn(make_float2(x[2 * j], x[2 * j + 1]), make_float2(a, a), make_float2(b, b));
        x[2 * j] = r.x;
        x[2 * j + 1] = r.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) x[i] = fmaf(x[i], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += x[i];
  if (s == -1.f) out[0] = s;  // never true (every x stays positive); keeps the chains live
}

}  // namespace nbtc

extern "C" nbtc_status nbtc_probe_ffma(nbtc_context* ctx, int32_t ctas, int32_t iters, int32_t packed,
                                       float* out_dev, double* flop, void* stream) {
  NBTC_RANGE();
  using namespace nbtc;
  nbtc_status st;
  if ((st = enter(ctx))) return st;
  if (ctas < 1 || iters < 1 || !flop || !out_dev) return fail(NBTC_ERR_INVALID_ARG, "ctas, iters, flop or out_dev");
  if ((st = need_device(out_dev, "out_dev"))) return st;
  *flop = (double)ctas * 256.0 * iters * 16.0 * 2.0;
  if (packed)
    k_ffma_probe<true><<<ctas, 256, 0, (cudaStream_t)stream>>>(out_dev, iters, 0.999f, 1e-3f);
  else
    k_ffma_probe<false><<<ctas, 256, 0, (cudaStream_t)stream>>>(out_dev, iters, 0.999f, 1e-3f);
  return cuda_check(cudaGetLastError(), "launch k_ffma_probe");
}
