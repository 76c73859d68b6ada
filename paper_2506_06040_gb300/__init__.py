"""GB300-native neural block texture decode (arXiv 2506.06040).

Python face of the C-ABI library `libnbtc.so` (include/nbtc.h): PyTorch holds
device memory and streams; every step of the decode, training and batching
paths runs in the library's CUDA kernels.  Build the library with
`paper_2506_06040_gb300.build.build()` (or `__graft_entry__.build()`).
"""
from ._abi import (CLAMP, FP8_E4M3, FP8_E4M3_SPLIT, FP16, FP16_SPLIT, FP32, FP32_TC, LOSS_L1, LOSS_MSE,  # noqa: F401
                   WRAP, NbtcError,
                   load)
from .api import (Batch, Context, Material, bc1_decode_level, decode, decode_to_host, fp8_calibrate,  # noqa: F401
                  pack_mlp)
