// Instantiation unit of the tensor-core decode kernel: 1 hidden layer(s), split FP16 operands (hi + lo pairs).
#include "tc_kernel.cuh"

namespace nbtc {

nbtc_status launch_tc_h1_f16s(const TcArgs& p, int W, int slots, int grid, cudaStream_t s) {
  if (p.tmem_a && W == 4 && slots == 1)  // A operands in TMEM
    return launch_tc_w<1, kF16Split, 4, kModeSingle, 1, true>(p, grid, s);
  if (W == 4 && slots == 1) return launch_tc_w<1, kF16Split, 4, kModeSingle, 1>(p, grid, s);
  return fail(NBTC_ERR_UNSUPPORTED, "split FP16 decode runs 4 warpgroups x 1 slot");
}

}  // namespace nbtc
