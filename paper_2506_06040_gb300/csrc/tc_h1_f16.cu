// Instantiation unit of the tensor-core decode kernel: 1 hidden layer(s), FP16 operands.
#include "tc_kernel.cuh"

namespace nbtc {

nbtc_status launch_tc_h1_f16(const TcArgs& p, int W, int grid, cudaStream_t s) {
  return W == 3 ? launch_tc_w<1, false, 3, kModeSingle>(p, grid, s) : launch_tc_w<1, false, 4, kModeSingle>(p, grid, s);
}

}  // namespace nbtc
