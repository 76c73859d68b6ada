"""Quantisation-aware BC1 latents (paper Sec. 3.2, Eqs. 1-3) -- TEST INFRASTRUCTURE ONLY.

The compressor keeps every BC1 latent level as floating-point parameters: per
4x4 block two endpoints e0, e1 (RGB) and per texel a blend factor alpha.  Each
goes through a sigmoid and is quantised to its BC1 bit width -- alpha to 2
bits, the endpoints to the [5, 6, 5] pattern -- and the decoded texel is the
Sec. 3.1 interpolation (1 - a) E0 + a E1 of the quantised values.  The
quantiser's gradient is passed through unchanged (straight-through), so the
backward sees only the sigmoid's derivative.  Eqs. 1-3 are garbled in the text
(all three read sigmoid(alpha)); the reading here applies each to its own
parameter.

Reading of quant(x, b): x in [0, 1] maps to the nearest of the 2^b levels
k / (2^b - 1).  The level is decided on the raw parameter p (x = sigmoid(p)):
k = #{j : p >= logit((j + 1/2) / n)}, n = 2^b - 1, with the thresholds
rounded to FP32 and p compared in FP32.  This is the nearest level of
sigmoid(p) (ties go up) computed without an exp, so an integer code never
depends on which exp implementation evaluated the sigmoid.

Encoding to real BC1 blocks (the closing step from trained parameters to the
decoder's input): endpoint codes c = R << 11 | G << 5 | B from the quantised
levels; the 2-bit level q of alpha (a = q / 3) selects palette entry
0 -> c0 (q = 0), 1 -> c1 (q = 3), 2 -> (2 c0 + c1) / 3 (q = 1),
3 -> (c0 + 2 c1) / 3 (q = 2), which is the four-colour mode and needs
c0 > c1.  If c0 < c1 the endpoints are swapped and q -> 3 - q; if c0 == c1
every index is 0 (all four levels decode to the same colour, and index 3 of
the then-selected three-colour mode would be black).
"""
from __future__ import annotations

import numpy as np

BITS = (5, 6, 5)


def sigmoid(p):
    return 1.0 / (1.0 + np.exp(-np.asarray(p, dtype=np.float64)))


def thresholds(bits: int) -> np.ndarray:
    """FP32 logits of the midpoints (j + 1/2) / n, j = 0 .. n-1, n = 2^bits - 1."""
    n = (1 << bits) - 1
    m = (np.arange(n, dtype=np.float64) + 0.5) / n
    return np.log(m / (1.0 - m)).astype(np.float32)


def level(p, bits: int) -> np.ndarray:
    """Integer level k in 0 .. 2^bits - 1 of raw parameters p (FP32 compares)."""
    p32 = np.asarray(p, dtype=np.float32)
    t = thresholds(bits)
    return np.sum(p32[..., None] >= t, axis=-1).astype(np.int64)


def quant_value(p, bits: int) -> np.ndarray:
    """quant(sigmoid(p), bits) as a value in [0, 1] (FP64)."""
    return level(p, bits) / float((1 << bits) - 1)


def endpoint_values(e: np.ndarray) -> np.ndarray:
    """[..., 3] raw endpoints -> quantised RGB in [0, 1] on the [5, 6, 5] levels."""
    return np.stack([quant_value(e[..., c], BITS[c]) for c in range(3)], axis=-1)


def decode(e0: np.ndarray, e1: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """Decoded latent texture T [h, w, 3] (FP64) of one level: e0, e1 [h/4, w/4, 3],
    alpha [h, w] (Sec. 3.1 interpolation of the quantised parameters)."""
    h, w = alpha.shape
    E0 = np.repeat(np.repeat(endpoint_values(e0), 4, axis=0), 4, axis=1)
    E1 = np.repeat(np.repeat(endpoint_values(e1), 4, axis=0), 4, axis=1)
    a = quant_value(alpha, 2)[..., None]
    assert E0.shape == (h, w, 3)
    return (1.0 - a) * E0 + a * E1


def backward(e0: np.ndarray, e1: np.ndarray, alpha: np.ndarray, dT: np.ndarray):
    """Straight-through gradients (g_e0, g_e1, g_alpha) of a loss given dL/dT [h, w, 3]."""
    h, w = alpha.shape
    E0 = np.repeat(np.repeat(endpoint_values(e0), 4, axis=0), 4, axis=1)
    E1 = np.repeat(np.repeat(endpoint_values(e1), 4, axis=0), 4, axis=1)
    a = quant_value(alpha, 2)[..., None]
    dT = np.asarray(dT, dtype=np.float64)

    def block_sum(x):  # [h, w, 3] -> [h/4, w/4, 3]
        return x.reshape(h // 4, 4, w // 4, 4, 3).sum(axis=(1, 3))

    s0, s1, sa = sigmoid(e0), sigmoid(e1), sigmoid(alpha)
    g_e0 = block_sum(dT * (1.0 - a)) * s0 * (1.0 - s0)
    g_e1 = block_sum(dT * a) * s1 * (1.0 - s1)
    g_alpha = np.sum(dT * (E1 - E0), axis=-1) * sa * (1.0 - sa)
    return g_e0, g_e1, g_alpha


def codes(e: np.ndarray) -> np.ndarray:
    """RGB565 words of raw endpoints [..., 3]."""
    return (level(e[..., 0], 5) << 11) | (level(e[..., 1], 6) << 5) | level(e[..., 2], 5)


def encode(e0: np.ndarray, e1: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """BC1 blocks (uint64, block row-major) of one level from its raw parameters."""
    h, w = alpha.shape
    c0, c1 = codes(e0), codes(e1)                  # [h/4, w/4]
    q = level(alpha, 2).reshape(h // 4, 4, w // 4, 4).transpose(0, 2, 1, 3)  # [bh, bw, ty, tx]
    swap = (c0 < c1)[..., None, None]
    q = np.where(swap, 3 - q, q)
    to_index = np.array([0, 2, 3, 1], dtype=np.int64)   # level q -> palette index
    idx = to_index[q]
    idx = np.where((c0 == c1)[..., None, None], 0, idx)
    first, second = np.maximum(c0, c1), np.minimum(c0, c1)   # four-colour mode: first > second
    shifts = 2 * (4 * np.arange(4)[:, None] + np.arange(4)[None, :])  # [ty, tx]
    word = np.sum(idx << shifts, axis=(-2, -1))
    blocks = (first.astype(np.uint64) | (second.astype(np.uint64) << np.uint64(16)) |
              (word.astype(np.uint64) << np.uint64(32)))
    return blocks.reshape(-1)


def train_step(state: dict, shifts, target: np.ndarray, uv: np.ndarray, lr_mlp: float = 1e-3,
               lr_latent: float = 1e-2, kind: str = "mse") -> dict:
    """One QAT training step (Sec. 3.2): decode every level from its raw
    parameters, run the continuous-latent forward / loss / backward on the
    decoded textures (oracle.train), carry dL/dT back to the raw parameters
    straight through the quantisers, and update MLP and raw parameters with Adam.
    state: e0, e1, alpha (lists over levels), weights, biases, their m_/v_
    moments and t (updates done so far).  Returns the new state with 'loss', the
    decoded textures 'T' and every gradient."""
    from . import train as tr
    T = [decode(a, b, c) for a, b, c in zip(state["e0"], state["e1"], state["alpha"])]
    y, cache = tr.forward(T, shifts, state["weights"], state["biases"], uv)
    loss, dy = tr.loss_and_dy(y, tr.target_sample(target, uv), kind)
    dW, db, dT = tr.backward(dy, cache, T, shifts, state["weights"])
    g = [backward(a, b, c, d) for a, b, c, d in zip(state["e0"], state["e1"], state["alpha"], dT)]
    t = state["t"] + 1
    new = {"t": t, "loss": loss, "T": T, "grad_w": dW, "grad_b": db, "grad_T": dT,
           "grad_e0": [x[0] for x in g], "grad_e1": [x[1] for x in g], "grad_alpha": [x[2] for x in g]}
    for name, grads, lr in (("weights", dW, lr_mlp), ("biases", db, lr_mlp), ("e0", new["grad_e0"], lr_latent),
                            ("e1", new["grad_e1"], lr_latent), ("alpha", new["grad_alpha"], lr_latent)):
        ps, ms, vs = [], [], []
        for p, gr, m, v in zip(state[name], grads, state["m_" + name], state["v_" + name]):
            p2, m2, v2 = tr.adam(np.asarray(p, dtype=np.float64), gr, m, v, t, lr)
            ps.append(p2); ms.append(m2); vs.append(v2)
        new[name], new["m_" + name], new["v_" + name] = ps, ms, vs
    return new


def init_state(e0, e1, alpha, weights, biases) -> dict:
    st = {"t": 0}
    for name, arrs in (("e0", e0), ("e1", e1), ("alpha", alpha), ("weights", weights), ("biases", biases)):
        st[name] = [np.asarray(a, dtype=np.float64) for a in arrs]
        st["m_" + name] = [np.zeros_like(a, dtype=np.float64) for a in arrs]
        st["v_" + name] = [np.zeros_like(a, dtype=np.float64) for a in arrs]
    return st
