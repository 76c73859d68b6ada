"""ctypes view of include/nbtc.h: struct layouts and function prototypes.

Argument marshalling only; every step of the decode runs in the CUDA library.
Loading fails loudly when `libnbtc.so` has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_float, c_int, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnbtc.so")

MAX_LEVELS, MAX_LAYERS, MAX_MIPS = 8, 4, 16
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT, ERR_BOUNDS = range(6)
FP32, FP16, FP8_E4M3 = 0, 1, 2
CLAMP, WRAP = 0, 1
LOSS_MSE, LOSS_L1 = 0, 1


class Level(ctypes.Structure):
    _fields_ = [("blocks", c_void_p), ("width", c_int32), ("height", c_int32),
                ("num_mips", c_int32), ("shift", c_float)]


class Latents(ctypes.Structure):
    _fields_ = [("num_levels", c_int32), ("address", c_int32), ("levels", Level * MAX_LEVELS)]


class Mlp(ctypes.Structure):
    _fields_ = [("num_layers", c_int32), ("dims", c_int32 * (MAX_LAYERS + 1)),
                ("weights", c_void_p), ("biases", c_void_p)]


# name -> (restype, argtypes)
PROTOTYPES = {
    "nbtc_create": (c_int, [c_int, POINTER(c_void_p)]),
    "nbtc_destroy": (c_int, [c_void_p]),
    "nbtc_status_sync": (c_int, [c_void_p, c_void_p]),
    "nbtc_status_string": (c_char_p, [c_int]),
    "nbtc_last_error": (c_char_p, []),
    "nbtc_set_wait_budget": (c_int, [c_void_p, c_int64]),
    "nbtc_bc1_decode_level": (c_int, [c_void_p, POINTER(Level), c_int32, c_void_p, c_void_p]),
    "nbtc_packed_mlp_bytes": (c_int, [POINTER(Mlp), c_int32, POINTER(c_size_t)]),
    "nbtc_pack_mlp": (c_int, [c_void_p, POINTER(Mlp), c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "nbtc_fp8_calibrate": (c_int, [c_void_p, POINTER(Latents), POINTER(Mlp), c_int32, c_int32, c_int32,
                                   c_void_p, c_void_p]),
    "nbtc_decode": (c_int, [c_void_p, POINTER(Latents), POINTER(Mlp), c_int32, c_void_p, c_void_p, c_int64,
                            c_int32, c_int32, c_void_p, c_void_p]),
}

_lib = None


class NbtcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"nbtc error {code}: {msg}")
        self.code = code


def load() -> ctypes.CDLL:
    """Loads libnbtc.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _lib = lib
    return _lib


def check(code: int) -> None:
    if code != OK:
        msg = load().nbtc_last_error().decode(errors="replace")
        raise NbtcError(code, msg)
