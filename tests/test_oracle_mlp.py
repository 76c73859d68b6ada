"""Pins of the oracle's MLP (Sec. 3.1 f(x): ReLU hidden layers, linear output)."""
import numpy as np
import torch

from oracle import mlp


def _brute(x, ws, bs):
    out = []
    for row in x:
        h = list(row)
        for l, (w, b) in enumerate(zip(ws, bs)):
            nh = []
            for j in range(len(b)):
                s = b[j]
                for i in range(len(h)):
                    s += w[j][i] * h[i]
                if l < len(ws) - 1 and s < 0:
                    s = 0.0
                nh.append(s)
            h = nh
        out.append(h)
    return np.array(out)


def test_tiny_brute_force():
    rng = np.random.default_rng(7)
    for dims in ([3, 2, 2], [12, 4, 9], [12, 5, 3, 9]):
        ws = [rng.normal(size=(dims[i + 1], dims[i])) for i in range(len(dims) - 1)]
        bs = [rng.normal(size=dims[i + 1]) for i in range(len(dims) - 1)]
        x = rng.random((17, dims[0]))
        np.testing.assert_allclose(mlp.forward(x, ws, bs), _brute(x, ws, bs), rtol=1e-13, atol=1e-13)


def test_against_torch_float64():
    rng = np.random.default_rng(8)
    dims = [12, 64, 64, 64, 9]
    ws = [rng.normal(size=(dims[i + 1], dims[i])) * np.sqrt(2 / dims[i]) for i in range(4)]
    bs = [rng.normal(size=dims[i + 1]) * 0.01 for i in range(4)]
    x = rng.random((1000, 12))
    h = torch.tensor(x)
    for l in range(4):
        h = torch.nn.functional.linear(h, torch.tensor(ws[l]), torch.tensor(bs[l]))
        if l < 3:
            h = torch.relu(h)
    np.testing.assert_allclose(mlp.forward(x, ws, bs), h.numpy(), rtol=1e-12, atol=1e-12)


def test_relu_signs():
    # hidden pre-activations (+2, -3): only the first survives; output = 5 * 2 + 7 * 0 + 1
    ws = [np.array([[1.0], [-1.0]]), np.array([[5.0, 7.0]])]
    bs = [np.array([1.0, -2.0]), np.array([1.0])]
    np.testing.assert_allclose(mlp.forward(np.array([[1.0]]), ws, bs), [[11.0]])
    # output layer is linear: negative outputs pass
    ws2 = [np.array([[1.0]]), np.array([[-4.0]])]
    np.testing.assert_allclose(mlp.forward(np.array([[2.0]]), ws2, [np.zeros(1), np.zeros(1)]), [[-8.0]])
    acts = mlp.hidden_activations(np.array([[1.0]]), ws, bs)
    np.testing.assert_allclose(acts[1], [[2.0, 0.0]])
