"""Thin torch-facing wrappers over the C ABI (argument marshalling only)."""
from __future__ import annotations

import ctypes
from ctypes import byref, c_size_t, c_void_p

import numpy as np
import torch

from . import _abi
from ._abi import check


def _stream(stream) -> c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def _ptr(t) -> c_void_p:
    return c_void_p(0 if t is None else t.data_ptr())


class Context:
    """A library context on one CUDA device (owns the device status word).
    checked=True runs every call of this context through the bounds-checked
    build of the library (libnbtc_checked.so)."""

    def __init__(self, device: int = 0, checked: bool = False):
        self.lib = _abi.load(checked)
        self.checked = checked
        self.device = device
        h = c_void_p()
        check(self.lib.nbtc_create(device, byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            self.lib.nbtc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        """Waits for the stream and raises if a kernel recorded a fault."""
        check(self.lib.nbtc_status_sync(self.handle, _stream(stream)))

    def status(self, stream=None) -> int:
        return self.lib.nbtc_status_sync(self.handle, _stream(stream))

    def set_wait_budget(self, spins: int):
        check(self.lib.nbtc_set_wait_budget(self.handle, spins))

    def set_check_plant(self, offset: int):
        """Checked build, tests only: offset added to every gather index, so that
        the bounds checks fire (NBTC_ERR_UNSUPPORTED in the default build)."""
        check(self.lib.nbtc_set_check_plant(self.handle, offset))


class Material:
    """Device copy of a material: BC1 latent levels (with mips) and an FP32 MLP.

    levels: list of (blocks: uint64 array of all mips back to back, width, height,
    num_mips, shift); weights[l]: [out, in] FP32; biases[l]: [out] FP32."""

    def __init__(self, levels, weights, biases, address: int = _abi.CLAMP, device="cuda"):
        self.device = torch.device(device)
        self.blocks, self.level_meta = [], []
        for blocks, w, h, mips, shift in levels:
            b = np.ascontiguousarray(np.asarray(blocks, dtype=np.uint64)).view(np.int64)
            self.blocks.append(torch.from_numpy(b).to(self.device))
            self.level_meta.append((int(w), int(h), int(mips), float(shift)))
        self.dims = [int(weights[0].shape[1])] + [int(w.shape[0]) for w in weights]
        self.weights = torch.from_numpy(np.concatenate([np.asarray(w, np.float32).ravel() for w in weights])).to(self.device)
        self.biases = torch.from_numpy(np.concatenate([np.asarray(b, np.float32).ravel() for b in biases])).to(self.device)
        self.address = address

    @classmethod
    def from_synth(cls, mat, device="cuda"):
        levels = [(lv.packed(), lv.width, lv.height, lv.num_mips, lv.shift) for lv in mat.levels]
        addr = _abi.WRAP if mat.address == "wrap" else _abi.CLAMP
        return cls(levels, mat.mlp.weights, mat.mlp.biases, addr, device)

    @property
    def n_out(self) -> int:
        return self.dims[-1]

    def latents_struct(self) -> _abi.Latents:
        s = _abi.Latents()
        s.num_levels = len(self.blocks)
        s.address = self.address
        for k, (b, (w, h, mips, shift)) in enumerate(zip(self.blocks, self.level_meta)):
            s.levels[k] = _abi.Level(b.data_ptr(), w, h, mips, shift)
        return s

    def level_struct(self, k: int) -> _abi.Level:
        w, h, mips, shift = self.level_meta[k]
        return _abi.Level(self.blocks[k].data_ptr(), w, h, mips, shift)

    def mlp_struct(self) -> _abi.Mlp:
        s = _abi.Mlp()
        s.num_layers = len(self.dims) - 1
        for i, d in enumerate(self.dims):
            s.dims[i] = d
        s.weights = self.weights.data_ptr()
        s.biases = self.biases.data_ptr()
        return s


def bc1_decode_level(ctx: Context, mat: Material, k: int, mip: int = 0, stream=None) -> torch.Tensor:
    w, h, _, _ = mat.level_meta[k]
    for _ in range(mip):
        w, h = max(4, w // 2), max(4, h // 2)
    out = torch.empty((h, w, 3), dtype=torch.uint8, device=mat.device)
    lv = mat.level_struct(k)
    check(ctx.lib.nbtc_bc1_decode_level(ctx.handle, byref(lv), mip, _ptr(out), _stream(stream)))
    return out


def packed_mlp_bytes(mat: Material, precision: int) -> int:
    n = c_size_t()
    m = mat.mlp_struct()
    check(_abi.load().nbtc_packed_mlp_bytes(byref(m), precision, byref(n)))
    return n.value


def fp8_calibrate(ctx: Context, mat: Material, grid_w: int, grid_h: int, step: int = 16,
                  stream=None) -> torch.Tensor:
    absmax = torch.empty(len(mat.dims) - 1, dtype=torch.float32, device=mat.device)
    lat, m = mat.latents_struct(), mat.mlp_struct()
    check(ctx.lib.nbtc_fp8_calibrate(ctx.handle, byref(lat), byref(m), grid_w, grid_h, step,
                                     _ptr(absmax), _stream(stream)))
    return absmax


def pack_mlp(ctx: Context, mat: Material, precision: int, act_absmax=None, stream=None) -> torch.Tensor:
    nbytes = packed_mlp_bytes(mat, precision)
    packed = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=mat.device)
    m = mat.mlp_struct()
    check(ctx.lib.nbtc_pack_mlp(ctx.handle, byref(m), precision, _ptr(act_absmax), _ptr(packed), nbytes,
                                _stream(stream)))
    return packed


def decode(ctx: Context, mat: Material, precision: int = _abi.FP32, packed=None, uv=None, grid=None,
           out=None, stream=None, rows=None) -> torch.Tensor:
    """Decodes n texels: grid=(w, h) texel centres, or uv [n, 2] FP32 on the device.
    rows=(row0, count) with a grid decodes only those rows of it.
    Returns [n, N] FP32 (FP32 form) or FP16 (tensor-core forms)."""
    if rows is not None:
        gw, gh = grid
        r0, nr = rows
        dt = torch.float32 if precision in (_abi.FP32, _abi.FP32_TC) else torch.float16
        if out is None:
            out = torch.empty((nr * gw, mat.n_out), dtype=dt, device=mat.device)
        lat, m = mat.latents_struct(), mat.mlp_struct()
        check(ctx.lib.nbtc_decode_rows(ctx.handle, byref(lat), byref(m), precision, _ptr(packed), gw, gh, r0, nr,
                                       _ptr(out), _stream(stream)))
        return out
    if uv is not None:
        assert uv.dtype == torch.float32 and uv.is_contiguous() and uv.dim() == 2 and uv.shape[1] == 2
        n, gw, gh = uv.shape[0], 0, 0
    else:
        gw, gh = grid
        n = gw * gh
    dt = torch.float32 if precision in (_abi.FP32, _abi.FP32_TC) else torch.float16
    if out is None:
        out = torch.empty((n, mat.n_out), dtype=dt, device=mat.device)
    lat, m = mat.latents_struct(), mat.mlp_struct()
    check(ctx.lib.nbtc_decode(ctx.handle, byref(lat), byref(m), precision, _ptr(packed), _ptr(uv), n, gw, gh,
                              _ptr(out), _stream(stream)))
    return out


def decode_to_host(ctx: Context, mat: Material, host_out: torch.Tensor, grid, precision: int = _abi.FP32,
                   packed=None, bands: int = 8, stream=None, copy_stream=None) -> torch.Tensor:
    """Grid decode into a pinned host tensor host_out [w*h, N].  FP32: one decode
    whose kernel stores the texels straight into host_out over the host link (no
    device buffer, no copy; done when `stream` is).  FP16 / FP8: the grid is
    decoded in `bands` row bands on `stream`, each band's device-to-host copy on
    `copy_stream` overlapping the next band's decode (two device band buffers);
    done when copy_stream is.  Returns host_out once the work is enqueued."""
    if host_out.device.type != "cpu" or not host_out.is_pinned():
        raise ValueError("host_out must be a pinned host tensor")
    gw, gh = grid
    stream = stream or torch.cuda.current_stream()
    if precision == _abi.FP32:
        return decode(ctx, mat, precision, packed, grid=grid, out=host_out, stream=stream)
    copy_stream = copy_stream or torch.cuda.Stream()
    per = -(-gh // bands)
    dt = torch.float32 if precision in (_abi.FP32, _abi.FP32_TC) else torch.float16
    bufs = [torch.empty((per * gw, mat.n_out), dtype=dt, device=mat.device) for _ in range(2)]
    done = [torch.cuda.Event(), torch.cuda.Event()]     # band decoded
    freed = [torch.cuda.Event(), torch.cuda.Event()]    # band buffer copied out
    for b, r0 in enumerate(range(0, gh, per)):
        nr = min(per, gh - r0)
        k = b & 1
        if b >= 2:
            stream.wait_event(freed[k])
        decode(ctx, mat, precision, packed, grid=grid, rows=(r0, nr), out=bufs[k][:nr * gw], stream=stream)
        done[k].record(stream)
        copy_stream.wait_event(done[k])
        with torch.cuda.stream(copy_stream):
            host_out[r0 * gw:(r0 + nr) * gw].copy_(bufs[k][:nr * gw], non_blocking=True)
        freed[k].record(copy_stream)
    return host_out


class Batch:
    """A batched-decode plan: many materials (each with its own BC1 pyramid and
    FP32 MLP, decoded in FP16 on tensor cores) decoded in one persistent
    graph-captured launch, and optionally a frame rendered through the tile
    classification / binning pipeline.

    materials: list of Material; outs: list of (tensor FP16 [h*w, C], w, h) or
    None per material; frame: dict(mat_id int32 [h, w], uv FP32 [h, w, 2],
    lod FP32 [h, w], out FP16 [h, w, C], and optionally duv FP32 [h, w, 4] with
    max_aniso for the anisotropic latent filter -- lod is then the mip bias -- and
    shaded FP32 [h, w, 4] with light=dict(light_dir, light_rgb, view_dir, sky,
    ground) for the fused lighting pass) or None."""

    def __init__(self, ctx: Context, materials, outs=None, frame=None, autotune=True, stream=None):
        self.ctx = ctx
        self.materials = list(materials)
        self.outs = list(outs) if outs is not None else [None] * len(self.materials)
        self.frame = frame
        arr = (_abi.BatchMaterial * len(self.materials))()
        for i, (m, o) in enumerate(zip(self.materials, self.outs)):
            arr[i].latents = m.latents_struct()
            arr[i].mlp = m.mlp_struct()
            if o is not None:
                t, w, h = o
                arr[i].out, arr[i].out_w, arr[i].out_h = t.data_ptr(), w, h
        fr = None
        if frame is not None:
            fr = _abi.Frame()
            fr.height, fr.width = int(frame["mat_id"].shape[0]), int(frame["mat_id"].shape[1])
            fr.mat_id, fr.uv, fr.lod, fr.out = (frame["mat_id"].data_ptr(), frame["uv"].data_ptr(),
                                                frame["lod"].data_ptr(), frame["out"].data_ptr())
            if frame.get("duv") is not None:
                fr.duv, fr.max_aniso = frame["duv"].data_ptr(), int(frame.get("max_aniso", 16))
            if frame.get("shaded") is not None:
                fr.shaded = frame["shaded"].data_ptr()
                lt = frame.get("light", {})
                for name, default in (("light_dir", (0.3, 0.4, 1.0)), ("light_rgb", (3.0, 3.0, 3.0)),
                                      ("view_dir", (0.0, 0.0, 1.0)), ("sky", (0.6, 0.7, 0.9)),
                                      ("ground", (0.15, 0.12, 0.1))):
                    getattr(fr, name)[:] = [float(x) for x in lt.get(name, default)]
        h = c_void_p()
        flags = _abi.BATCH_AUTOTUNE if autotune else 0
        check(ctx.lib.nbtc_batch_create(ctx.handle, arr, len(self.materials), byref(fr) if fr is not None else None,
                                        flags, byref(h), _stream(stream)))
        self.handle = h

    def decode(self, stream=None):
        check(self.ctx.lib.nbtc_decode_batched(self.ctx.handle, self.handle, _stream(stream)))

    def render(self, stream=None):
        check(self.ctx.lib.nbtc_render_frame(self.ctx.handle, self.handle, _stream(stream)))

    def info(self) -> dict:
        i = _abi.BatchInfo()
        check(self.ctx.lib.nbtc_batch_info_get(self.handle, byref(i)))
        return {f: getattr(i, f) for f, _ in i._fields_}

    def close(self):
        if self.handle:
            self.ctx.lib.nbtc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
