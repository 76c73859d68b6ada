// FP32 SIMT decode: instantiations of the decode kernel (see fp32_kernel.cuh).
#include "fp32_kernel.cuh"

namespace nbtc {

nbtc_status launch_decode_fp32(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, cudaStream_t s) {
  return dispatch<false>(ctx, a, mlp, 1, nullptr, s);
}


}  // namespace nbtc
