"""MLP decoder f(x), FP64.

Paper Sec. 3.1: the concatenated latent vector is fed to a multi-layer
perceptron that outputs the material channels.  Hidden layers apply ReLU; the
output layer is linear.  Layer l has weight W_l [out, in] and bias b_l:
h_{l+1} = ReLU(W_l h_l + b_l).
"""
from __future__ import annotations

import numpy as np


def forward(x: np.ndarray, weights: list, biases: list) -> np.ndarray:
    h = np.asarray(x, dtype=np.float64)
    n = len(weights)
    for l, (w, b) in enumerate(zip(weights, biases)):
        h = h @ np.asarray(w, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
        if l < n - 1:
            h = np.maximum(h, 0.0)
    return h


def hidden_activations(x: np.ndarray, weights: list, biases: list) -> list:
    """Inputs of every layer: [x, h_1, ..., h_{L-1}] (FP64)."""
    acts = [np.asarray(x, dtype=np.float64)]
    h = acts[0]
    for w, b in zip(weights[:-1], biases[:-1]):
        h = np.maximum(h @ np.asarray(w, dtype=np.float64).T + np.asarray(b, dtype=np.float64), 0.0)
        acts.append(h)
    return acts
