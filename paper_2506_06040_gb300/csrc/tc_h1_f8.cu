// Instantiation unit of the tensor-core decode kernel: 1 hidden layer(s), E4M3 operands.
#include "tc_kernel.cuh"

namespace nbtc {

nbtc_status launch_tc_h1_f8(const TcArgs& p, int W, int grid, cudaStream_t s) {
  return W == 3 ? launch_tc_w<1, true, 3, kModeSingle>(p, grid, s) : launch_tc_w<1, true, 4, kModeSingle>(p, grid, s);
}

}  // namespace nbtc
