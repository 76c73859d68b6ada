// BC1 level decode to RGB8 (parity and debugging): one thread per texel.
#include "host.h"

namespace nbtc {

__global__ void k_bc1_decode_level(LevelView v, uint8_t* __restrict__ out) {
  const int64_t n = (int64_t)v.w * v.h;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(t / v.w), x = (int)(t - (int64_t)y * v.w);
    const uint32_t rgb = fetch_texel(v, x, y);
    out[3 * t + 0] = (uint8_t)(rgb & 255u);
    out[3 * t + 1] = (uint8_t)((rgb >> 8) & 255u);
    out[3 * t + 2] = (uint8_t)((rgb >> 16) & 255u);
  }
}

nbtc_status launch_bc1_decode(nbtc_context* ctx, const LevelView& v, uint8_t* out, cudaStream_t s) {
  const int64_t n = (int64_t)v.w * v.h;
  int grid = (int)((n + 255) / 256);
  if (grid > ctx->sm_count * 8) grid = ctx->sm_count * 8;
  k_bc1_decode_level<<<grid, 256, 0, s>>>(v, out);
  return cuda_check(cudaGetLastError(), "launch k_bc1_decode_level");
}

}  // namespace nbtc
