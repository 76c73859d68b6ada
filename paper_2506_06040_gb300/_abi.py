"""ctypes view of include/nbtc.h: struct layouts and function prototypes.

Argument marshalling only; every step of the decode runs in the CUDA library.
Loading fails loudly when `libnbtc.so` has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnbtc.so")
# the same library built with per-access bounds checks (NBTC_CHECKED)
LIB_CHECKED_PATH = os.path.join(HERE, "libnbtc_checked.so")

MAX_LEVELS, MAX_LAYERS, MAX_MIPS = 8, 4, 16
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT, ERR_BOUNDS = range(6)
FP32, FP16, FP8_E4M3, FP16_SPLIT, FP8_E4M3_SPLIT, FP32_TC = 0, 1, 2, 3, 4, 5
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


class TrainArgs(ctypes.Structure):
    _fields_ = [("num_levels", c_int32), ("widths", c_int32 * MAX_LEVELS), ("heights", c_int32 * MAX_LEVELS),
                ("shifts", c_float * MAX_LEVELS), ("latents", c_void_p * MAX_LEVELS),
                ("latent_grads", c_void_p * MAX_LEVELS), ("latent_m", c_void_p * MAX_LEVELS),
                ("latent_v", c_void_p * MAX_LEVELS), ("mlp", Mlp), ("grad_w", c_void_p), ("grad_b", c_void_p),
                ("m_w", c_void_p), ("v_w", c_void_p), ("m_b", c_void_p), ("v_b", c_void_p), ("target", c_void_p),
                ("target_w", c_int32), ("target_h", c_int32), ("uv", c_void_p), ("batch", c_int64),
                ("step", c_int32), ("lr_mlp", c_float), ("lr_latent", c_float), ("beta1", c_float),
                ("beta2", c_float), ("eps", c_float), ("loss", c_int32), ("workspace", c_void_p),
                ("workspace_bytes", c_size_t), ("latent_stride", c_int32), ("target_stride", c_int32)]


class QatLevel(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("e0", c_void_p), ("e1", c_void_p), ("alpha", c_void_p),
                ("g_e0", c_void_p), ("g_e1", c_void_p), ("g_alpha", c_void_p), ("m_e0", c_void_p),
                ("v_e0", c_void_p), ("m_e1", c_void_p), ("v_e1", c_void_p), ("m_alpha", c_void_p),
                ("v_alpha", c_void_p)]


class BatchMaterial(ctypes.Structure):
    _fields_ = [("latents", Latents), ("mlp", Mlp), ("out_w", c_int32), ("out_h", c_int32), ("out", c_void_p)]


class Frame(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("mat_id", c_void_p), ("uv", c_void_p),
                ("lod", c_void_p), ("out", c_void_p), ("duv", c_void_p), ("max_aniso", c_int32),
                ("shaded", c_void_p), ("light_dir", c_float * 3), ("light_rgb", c_float * 3),
                ("view_dir", c_float * 3), ("sky", c_float * 3), ("ground", c_float * 3)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("warpgroups", c_int32), ("chunk_tiles", c_int32), ("tile_w", c_int32), ("tile_h", c_int32),
                ("decode_tiles", c_int64), ("frame_uniform_tiles", c_int64), ("frame_mixed_tiles", c_int64),
                ("frame_packed_tiles", c_int64), ("tuned_decode_ms", c_float), ("tuned_render_ms", c_float),
                ("render_warpgroups", c_int32), ("decode_tmem_operands", c_int32),
                ("render_tmem_operands", c_int32)]


BATCH_AUTOTUNE = 1


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
    "nbtc_decode_rows": (c_int, [c_void_p, POINTER(Latents), POINTER(Mlp), c_int32, c_void_p, c_int32, c_int32,
                                 c_int32, c_int32, c_void_p, c_void_p]),
    "nbtc_train_workspace_bytes": (c_int, [c_void_p, POINTER(TrainArgs), POINTER(c_size_t)]),
    "nbtc_train_step": (c_int, [c_void_p, POINTER(TrainArgs), c_void_p, c_void_p]),
    "nbtc_forward_continuous": (c_int, [c_void_p, POINTER(TrainArgs), c_void_p, c_void_p]),
    "nbtc_backward_continuous": (c_int, [c_void_p, POINTER(TrainArgs), c_void_p, c_void_p]),
    "nbtc_train_step_noalloc": (c_int, [POINTER(TrainArgs), c_void_p, c_void_p]),
    "nbtc_qat_decode": (c_int, [c_void_p, POINTER(QatLevel), c_void_p, c_void_p]),
    "nbtc_qat_encode": (c_int, [c_void_p, POINTER(QatLevel), c_void_p, c_void_p]),
    "nbtc_train_step_qat": (c_int, [c_void_p, POINTER(TrainArgs), POINTER(QatLevel), c_void_p, c_void_p]),
    "nbtc_batch_create": (c_int, [c_void_p, POINTER(BatchMaterial), c_int32, POINTER(Frame), c_int32,
                                  POINTER(c_void_p), c_void_p]),
    "nbtc_decode_batched": (c_int, [c_void_p, c_void_p, c_void_p]),
    "nbtc_render_frame": (c_int, [c_void_p, c_void_p, c_void_p]),
    "nbtc_batch_info_get": (c_int, [c_void_p, POINTER(BatchInfo)]),
    "nbtc_batch_destroy": (c_int, [c_void_p]),
    "nbtc_probe_ffma": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, POINTER(c_double), c_void_p]),
    "nbtc_probe_scatter": (c_int, [c_void_p, POINTER(TrainArgs), c_void_p]),
    "nbtc_set_check_plant": (c_int, [c_void_p, c_int32]),
}

_lib = None
_lib_checked = None


class NbtcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"nbtc error {code}: {msg}")
        self.code = code


def _open(path: str) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


def load(checked: bool = False) -> ctypes.CDLL:
    """Loads libnbtc.so, or with checked=True its bounds-checked build
    libnbtc_checked.so (raises if it is missing: there is no fallback path)."""
    global _lib, _lib_checked
    if checked:
        if _lib_checked is None:
            _lib_checked = _open(LIB_CHECKED_PATH)
        return _lib_checked
    if _lib is None:
        _lib = _open(LIB_PATH)
    return _lib


def check(code: int) -> None:
    if code != OK:
        msg = load().nbtc_last_error().decode(errors="replace")
        if not msg and _lib_checked is not None:
            msg = _lib_checked.nbtc_last_error().decode(errors="replace")
        raise NbtcError(code, msg)
