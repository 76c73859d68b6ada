// Instantiation unit of the tensor-core decode kernel: 1 hidden layer(s), E4M3 operands.
#include "tc_kernel.cuh"

namespace nbtc {

nbtc_status launch_tc_h1_f8(const TcArgs& p, int W, int slots, int grid, cudaStream_t s) {
  if (p.tmem_a && W == 5 && slots == 1)  // A operands in TMEM: 5 warpgroups x 1 slot
    return launch_tc_w<1, kF8, 5, kModeSingle, 1, true>(p, grid, s);
  if (slots != 2) return fail(NBTC_ERR_UNSUPPORTED, "this form runs two tile slots per warpgroup");
  return W == 3 ? launch_tc_w<1, kF8, 3, kModeSingle, 2>(p, grid, s) : launch_tc_w<1, kF8, 4, kModeSingle, 2>(p, grid, s);
}

}  // namespace nbtc
