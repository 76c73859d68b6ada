"""Checkpoint / resume of a training state (host side): the latents, the MLP,
every Adam moment and the step counter -- for QAT models also the raw BC1
parameters (endpoints, blend factors) and their moments.

File layout: the 8 bytes b"NBTCCKPT", a little-endian uint64 header length, a
UTF-8 JSON header (model kind, shifts, MLP dims, step, latent texel stride and
one entry per array: name, shape, byte offset), then the arrays as
little-endian FP32, each starting on a 64-byte boundary.  Latents and their
moments are stored as [h, w, 3] whatever their texel stride in memory.
Loading rebuilds the model on a device with the same state, so the next step
runs from exactly the saved values."""
from __future__ import annotations

import json
import struct

import numpy as np
import torch

from .train import ContinuousModel, QatModel

MAGIC = b"NBTCCKPT"
_ALIGN = 64


def _arrays(model: ContinuousModel) -> dict:
    out = {"weights": model.weights, "biases": model.biases, "m_w": model.m_w, "v_w": model.v_w,
           "m_b": model.m_b, "v_b": model.v_b}
    if isinstance(model, QatModel):
        names = ("e0", "e1", "alpha", "m_e0", "v_e0", "m_e1", "v_e1", "m_alpha", "v_alpha")
    else:
        names = ("latents", "latent_m", "latent_v")
    for n in names:
        for k, t in enumerate(getattr(model, n)):
            out[f"{n}.{k}"] = t
    return out


def save(model: ContinuousModel, path: str) -> None:
    """Writes the model's training state to `path` (synchronises with the device)."""
    arrays = {n: np.ascontiguousarray(t.detach().float().cpu().numpy()) for n, t in _arrays(model).items()}
    entries, off = [], 0
    for n, a in arrays.items():
        off = -(-off // _ALIGN) * _ALIGN
        entries.append({"name": n, "shape": list(a.shape), "offset": off})
        off += a.nbytes
    header = {"version": 1, "kind": "qat" if isinstance(model, QatModel) else "continuous",
              "shifts": model.shifts, "dims": model.dims, "step": model.step_count,
              "latent_stride": model.latent_stride, "arrays": entries}
    hb = json.dumps(header).encode()
    with open(path, "wb") as f:
        f.write(MAGIC + struct.pack("<Q", len(hb)) + hb)
        base = f.tell()
        for e, a in zip(entries, arrays.values()):
            f.seek(base + e["offset"])
            f.write(a.astype("<f4").tobytes())


def load(path: str, device="cuda") -> ContinuousModel:
    """Rebuilds the model saved in `path` on `device`."""
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError(f"{path}: not an nbtc checkpoint")
        (n,) = struct.unpack("<Q", f.read(8))
        header = json.loads(f.read(n).decode())
        base = f.tell()
        arrays = {}
        for e in header["arrays"]:
            f.seek(base + e["offset"])
            count = int(np.prod(e["shape"])) if e["shape"] else 1
            arrays[e["name"]] = np.frombuffer(f.read(4 * count), dtype="<f4").reshape(e["shape"]).astype(np.float32)
    if header["version"] != 1:
        raise ValueError(f"{path}: checkpoint version {header['version']}")
    dims = header["dims"]
    offs = np.cumsum([0] + [dims[i] * dims[i + 1] for i in range(len(dims) - 1)])
    boffs = np.cumsum([0] + dims[1:])
    weights = [arrays["weights"][offs[i]:offs[i + 1]].reshape(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]
    biases = [arrays["biases"][boffs[i]:boffs[i + 1]] for i in range(len(dims) - 1)]
    levels = len(header["shifts"])
    pick = lambda name: [arrays[f"{name}.{k}"] for k in range(levels)]
    if header["kind"] == "qat":
        model = QatModel(pick("e0"), pick("e1"), pick("alpha"), header["shifts"], weights, biases, device,
                         header["latent_stride"])
        for name in ("m_e0", "v_e0", "m_e1", "v_e1", "m_alpha", "v_alpha"):
            for dst, src in zip(getattr(model, name), pick(name)):
                dst.copy_(torch.from_numpy(src))
    else:
        model = ContinuousModel(pick("latents"), header["shifts"], weights, biases, device, header["latent_stride"])
        for name in ("latent_m", "latent_v"):
            for dst, src in zip(getattr(model, name), pick(name)):
                dst.copy_(torch.from_numpy(src))
    for name in ("m_w", "v_w", "m_b", "v_b"):
        getattr(model, name).copy_(torch.from_numpy(arrays[name]))
    model.step_count = int(header["step"])
    return model
