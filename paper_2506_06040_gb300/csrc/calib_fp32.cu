// FP8 calibration: the FP32 decode kernel recording each layer's input absmax
// (instantiations of fp32_kernel.cuh).
#include "fp32_kernel.cuh"

namespace nbtc {

nbtc_status launch_calibrate_fp32(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, int step,
                                  float* absmax, cudaStream_t s) {
  nbtc_status st = cuda_check(cudaMemsetAsync(absmax, 0, sizeof(float) * mlp->num_layers, s), "memset absmax");
  if (st) return st;
  return dispatch<true>(ctx, a, mlp, step, absmax, s);
}

}  // namespace nbtc
