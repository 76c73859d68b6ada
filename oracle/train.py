"""Training step of the decoder on continuous latents, FP64.

Paper Sec. 3.2: the compressor decodes latents with a replica of the texture
unit (bilinear sampling, Sec. 3.1 features), runs the MLP, compares with the
reference texture sampled with the same filter, and lets Adam update both the
MLP (lr 1e-3) and every latent texel (lr 1e-2), gradients flowing through the
MLP and the filter into the latents.  This is the continuous (pre-BC1) form:
latents are plain FP32 textures, no sigmoid, no quantisation.

Readings fixed here: the loss is the mean over batch and channels of (y - t)^2
(MSE; an L1 variant, mean |y - t|, is the paper's own choice and kept as an
option); Adam uses PyTorch's defaults beta = (0.9, 0.999), eps = 1e-8 with
bias correction; targets are sampled bilinearly with clamp, shift 0; ReLU'(0) = 0.
"""
from __future__ import annotations

import numpy as np

from .sample import axis_taps, bilinear


def _taps(h: int, w: int, u, v, shift: float):
    """Clamp-addressed bilinear taps: four (row, col, weight) triples per sample."""
    xa, xb, fx = axis_taps(u, w, shift, "clamp")
    ya, yb, fy = axis_taps(v, h, shift, "clamp")
    return [(ya, xa, (1 - fx) * (1 - fy)), (ya, xb, fx * (1 - fy)),
            (yb, xa, (1 - fx) * fy), (yb, xb, fx * fy)]


def forward(latents: list, shifts, weights: list, biases: list, uv: np.ndarray):
    """Returns (y [B, N], cache) with every layer's input and pre-activation."""
    u, v = uv[:, 0].astype(np.float64), uv[:, 1].astype(np.float64)
    x = np.concatenate([bilinear(t, u, v, s, "clamp") for t, s in zip(latents, shifts)], axis=-1)
    ins, pre = [x], []
    h = x
    n = len(weights)
    for l, (w, b) in enumerate(zip(weights, biases)):
        z = h @ np.asarray(w, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
        pre.append(z)
        h = np.maximum(z, 0.0) if l < n - 1 else z
        if l < n - 1:
            ins.append(h)
    return h, {"inputs": ins, "pre": pre, "u": u, "v": v}


def target_sample(target: np.ndarray, uv: np.ndarray) -> np.ndarray:
    return bilinear(target, uv[:, 0].astype(np.float64), uv[:, 1].astype(np.float64), 0.0, "clamp")


def loss_and_dy(y: np.ndarray, t: np.ndarray, kind: str = "mse"):
    n = y.size
    d = y - t
    if kind == "mse":
        return float(np.sum(d * d) / n), 2.0 * d / n
    if kind == "l1":
        return float(np.sum(np.abs(d)) / n), np.sign(d) / n
    raise ValueError(kind)


def backward(dy: np.ndarray, cache: dict, latents: list, shifts, weights: list):
    """Gradients (dW list, db list, dlatents list) of the loss given dL/dy."""
    n = len(weights)
    dW, db = [None] * n, [None] * n
    g = dy
    for l in range(n - 1, -1, -1):
        dW[l] = g.T @ cache["inputs"][l]
        db[l] = g.sum(axis=0)
        g = g @ np.asarray(weights[l], dtype=np.float64)
        if l > 0:
            g = g * (cache["pre"][l - 1] > 0)
    dx = g  # [B, 3L]
    dlat = []
    for k, (t, s) in enumerate(zip(latents, shifts)):
        h, w = t.shape[:2]
        acc = np.zeros(h * w * 3)
        for (yy, xx, wt) in _taps(h, w, cache["u"], cache["v"], s):
            for c in range(3):
                # dL/dT_k[texel, c] += tap weight * dL/dx_k,c  (weighted histogram over texels)
                acc[c::3] += np.bincount(yy * w + xx, weights=wt * dx[:, 3 * k + c], minlength=h * w)
        dlat.append(acc.reshape(h, w, 3))
    return dW, db, dlat


def adam(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (PyTorch form); returns (p, m, v) as new FP64 arrays."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def loss_fn(latents, shifts, weights, biases, target, uv, kind="mse") -> float:
    y, _ = forward(latents, shifts, weights, biases, uv)
    return loss_and_dy(y, target_sample(target, uv), kind)[0]


def train_step(state: dict, shifts, target: np.ndarray, uv: np.ndarray, lr_mlp: float = 1e-3,
               lr_latent: float = 1e-2, kind: str = "mse") -> dict:
    """state: latents, weights, biases, and Adam moments m_*/v_* and step t (t = number of
    updates done so far).  Returns the new state plus 'loss' and the gradients."""
    y, cache = forward(state["latents"], shifts, state["weights"], state["biases"], uv)
    loss, dy = loss_and_dy(y, target_sample(target, uv), kind)
    dW, db, dlat = backward(dy, cache, state["latents"], shifts, state["weights"])
    t = state["t"] + 1
    new = {"t": t, "loss": loss, "grad_w": dW, "grad_b": db, "grad_lat": dlat}
    for name, grads, lr in (("weights", dW, lr_mlp), ("biases", db, lr_mlp), ("latents", dlat, lr_latent)):
        ps, ms, vs = [], [], []
        for p, g, m, v in zip(state[name], grads, state["m_" + name], state["v_" + name]):
            p2, m2, v2 = adam(np.asarray(p, dtype=np.float64), g, m, v, t, lr)
            ps.append(p2); ms.append(m2); vs.append(v2)
        new[name], new["m_" + name], new["v_" + name] = ps, ms, vs
    return new


def init_state(latents, weights, biases) -> dict:
    st = {"t": 0}
    for name, arrs in (("latents", latents), ("weights", weights), ("biases", biases)):
        st[name] = [np.asarray(a, dtype=np.float64) for a in arrs]
        st["m_" + name] = [np.zeros_like(a, dtype=np.float64) for a in arrs]
        st["v_" + name] = [np.zeros_like(a, dtype=np.float64) for a in arrs]
    return st
