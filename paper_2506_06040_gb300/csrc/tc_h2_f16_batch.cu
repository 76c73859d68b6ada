// Instantiation unit of the tensor-core decode kernel, batched materials / frame: 2 hidden layer(s), FP16 operands.
#include "tc_kernel.cuh"

namespace nbtc {

nbtc_status launch_tc_h2_f16_batch(const TcArgs& p, int W, int slots, int grid, cudaStream_t s) {
  if (p.tmem_a) {  // A operands in TMEM: 4 warpgroups x 1 slot
    if (W == 4 && slots == 1) return launch_tc_w<2, kF16, 4, kModeBatch, 1, true>(p, grid, s);
    return fail(NBTC_ERR_UNSUPPORTED, "TMEM operands: 4 warpgroups x 1 slot");
  }
  if (slots != 2) return fail(NBTC_ERR_UNSUPPORTED, "the batched decode runs two tile slots per warpgroup");
  return W == 3 ? launch_tc_w<2, kF16, 3, kModeBatch, 2>(p, grid, s) : launch_tc_w<2, kF16, 4, kModeBatch, 2>(p, grid, s);
}

}  // namespace nbtc
