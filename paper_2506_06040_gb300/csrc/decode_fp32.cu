// FP32 SIMT decode: instantiations of the decode kernel (see fp32_kernel.cuh).
#include "fp32_kernel.cuh"

namespace nbtc {

nbtc_status launch_decode_fp32_tile(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, cudaStream_t s);

nbtc_status launch_decode_fp32(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, cudaStream_t s) {
  // hidden width 64: the tiled GEMM kernel; other shapes: the per-texel kernel
  const nbtc_status st = launch_decode_fp32_tile(ctx, a, mlp, s);
  if (st != NBTC_ERR_UNSUPPORTED) return st;
  return dispatch<false>(ctx, a, mlp, 1, nullptr, s);
}


}  // namespace nbtc
