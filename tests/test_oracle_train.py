"""Pins of the oracle's training step (Sec. 3.2): analytic gradients against
central finite differences in FP64 and against torch float64 autograd; Adam
against its closed form at t = 1."""
import numpy as np
import pytest
import torch

import synth
from oracle import train


@pytest.fixture(scope="module")
def reduced():
    wl = synth.train_workload(full=False)
    return wl, wl.uv(0)


def _grads(wl, uv, kind="mse"):
    y, cache = train.forward(wl.latents, wl.shifts, wl.mlp.weights, wl.mlp.biases, uv)
    loss, dy = train.loss_and_dy(y, train.target_sample(wl.target, uv), kind)
    return loss, train.backward(dy, cache, wl.latents, wl.shifts, wl.mlp.weights)


def _fd(f, arrs, idx, base_mask, h=1e-6):
    """Central difference; None when the +-h evaluations cross a ReLU kink (the
    activation pattern differs from the unperturbed one)."""
    a = arrs[idx[0]]
    old = a[idx[1:]]
    a[idx[1:]] = old + h
    fp, mp = f()
    a[idx[1:]] = old - h
    fm, mm = f()
    a[idx[1:]] = old
    if not (np.array_equal(mp, base_mask) and np.array_equal(mm, base_mask)):
        return None
    return (fp - fm) / (2 * h)


def test_finite_differences(reduced):
    wl, uv = reduced
    lat = [l.astype(np.float64) for l in wl.latents]
    ws = [w.astype(np.float64) for w in wl.mlp.weights]
    bs = [b.astype(np.float64) for b in wl.mlp.biases]
    def f():
        y, c = train.forward(lat, wl.shifts, ws, bs, uv)
        mask = np.concatenate([(z > 0).ravel() for z in c["pre"][:-1]])
        return train.loss_and_dy(y, train.target_sample(wl.target, uv))[0], mask
    y, cache = train.forward(lat, wl.shifts, ws, bs, uv)
    base = np.concatenate([(z > 0).ravel() for z in cache["pre"][:-1]])
    _, dy = train.loss_and_dy(y, train.target_sample(wl.target, uv))
    dW, db, dlat = train.backward(dy, cache, lat, wl.shifts, ws)
    scale = max(np.abs(g).max() for g in dW + db + dlat)
    errs, skipped = [], 0

    def check(arrs, idx, analytic):
        nonlocal skipped
        d = _fd(f, arrs, idx, base)
        if d is None:
            skipped += 1
        else:
            errs.append(d - analytic)
    for k in range(4):                                   # every latent coordinate
        for idx in np.ndindex(lat[k].shape):
            check(lat, (k,) + idx, dlat[k][idx])
    for l in range(3):                                   # every bias
        for j in range(bs[l].shape[0]):
            check(bs, (l, j), db[l][j])
    rng = np.random.default_rng(15)
    for _ in range(512):                                 # 512 random weights
        l = int(rng.integers(0, 3))
        j, i = int(rng.integers(0, ws[l].shape[0])), int(rng.integers(0, ws[l].shape[1]))
        check(ws, (l, j, i), dW[l][j, i])
    assert skipped <= 0.01 * (len(errs) + skipped)
    assert np.abs(errs).max() <= 1e-6 * scale


def test_against_torch_autograd(reduced):
    wl, uv = reduced
    for kind in ("mse", "l1"):
        loss, (dW, db, dlat) = _grads(wl, uv, kind)
        lat = [torch.tensor(l.astype(np.float64), requires_grad=True) for l in wl.latents]
        ws = [torch.tensor(w.astype(np.float64), requires_grad=True) for w in wl.mlp.weights]
        bs = [torch.tensor(b.astype(np.float64), requires_grad=True) for b in wl.mlp.biases]
        u = torch.tensor(uv[:, 0].astype(np.float64))
        v = torch.tensor(uv[:, 1].astype(np.float64))
        feats = []
        for t, s in zip(lat, wl.shifts):
            h, w = t.shape[:2]
            # grid_sample with align_corners=False uses the same texel-centre convention
            g = torch.stack([u * 2 - 1 + 2 * s / w, v * 2 - 1 + 2 * s / h], -1)[None, None]
            smp = torch.nn.functional.grid_sample(t.permute(2, 0, 1)[None], g, mode="bilinear",
                                                  padding_mode="border", align_corners=False)
            feats.append(smp[0, :, 0, :].T)
        x = torch.cat(feats, -1)
        hh = x
        for l in range(3):
            hh = torch.nn.functional.linear(hh, ws[l], bs[l])
            if l < 2:
                hh = torch.relu(hh)
        tt = torch.tensor(train.target_sample(wl.target, uv))
        tl = ((hh - tt) ** 2).mean() if kind == "mse" else (hh - tt).abs().mean()
        tl.backward()
        assert abs(tl.item() - loss) < 1e-12
        for a, b in zip(dW + db + dlat, [t.grad for t in ws + bs + lat]):
            np.testing.assert_allclose(a, b.numpy(), rtol=1e-9, atol=1e-14)


def test_latent_grad_partition_of_unity(reduced):
    wl, uv = reduced
    y, cache = train.forward(wl.latents, wl.shifts, wl.mlp.weights, wl.mlp.biases, uv)
    _, dy = train.loss_and_dy(y, train.target_sample(wl.target, uv))
    g = dy
    for l in range(2, -1, -1):
        g = g @ wl.mlp.weights[l].astype(np.float64)
        if l > 0:
            g = g * (cache["pre"][l - 1] > 0)
    _, _, dlat = train.backward(dy, cache, wl.latents, wl.shifts, wl.mlp.weights)
    for k in range(4):
        np.testing.assert_allclose(dlat[k].sum(axis=(0, 1)), g[:, 3 * k:3 * k + 3].sum(axis=0), atol=1e-13)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(16)
    p, g = rng.normal(size=1000), rng.normal(size=1000) * 10.0 ** rng.uniform(-9, 0, 1000)
    z = np.zeros(1000)
    p2, m, v = train.adam(p, g, z, z, 1, 1e-2)
    np.testing.assert_allclose(p2, p - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
    p3, _, _ = train.adam(p, np.zeros(1000), z, z, 1, 1e-2)
    np.testing.assert_array_equal(p3, p)


def test_train_step_reduces_loss(reduced):
    wl, uv = reduced
    st = train.init_state(wl.latents, wl.mlp.weights, wl.mlp.biases)
    losses = []
    for _ in range(5):
        st = train.train_step(st, wl.shifts, wl.target, uv)
        losses.append(st["loss"])
    assert losses[-1] < losses[0]
    assert st["t"] == 5
