// Instantiation unit of the tensor-core decode kernel, batched materials / frame: 2 hidden layer(s), FP16 operands.
#include "tc_kernel.cuh"

namespace nbtc {

nbtc_status launch_tc_h2_f16_batch(const TcArgs& p, int W, int grid, cudaStream_t s) {
  return W == 3 ? launch_tc_w<2, false, 3, kModeBatch>(p, grid, s) : launch_tc_w<2, false, 4, kModeBatch>(p, grid, s);
}

}  // namespace nbtc
