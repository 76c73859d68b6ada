"""Host-only: the batch gradient is the sum of the gradients of its shards
(each shard's loss weighted by its share), the decomposition a data-parallel
training run would all-reduce."""
import numpy as np

import synth
from oracle import train


def test_shard_gradients_sum_to_batch_gradient():
    wl = synth.train_workload(full=False)
    uv = wl.uv(3)
    full = train.forward(wl.latents, wl.shifts, wl.mlp.weights, wl.mlp.biases, uv)
    _, dy = train.loss_and_dy(full[0], train.target_sample(wl.target, uv))
    gW, gb, gl = train.backward(dy, full[1], wl.latents, wl.shifts, wl.mlp.weights)
    R = 4
    acc = None
    for r in range(R):
        part = uv[r::R]
        y, cache = train.forward(wl.latents, wl.shifts, wl.mlp.weights, wl.mlp.biases, part)
        _, d = train.loss_and_dy(y, train.target_sample(wl.target, part))
        d = d * (len(part) / len(uv))   # shard mean -> share of the batch mean
        g = train.backward(d, cache, wl.latents, wl.shifts, wl.mlp.weights)
        flat = np.concatenate([x.ravel() for grp in g for x in grp])
        acc = flat if acc is None else acc + flat
    ref = np.concatenate([x.ravel() for grp in (gW, gb, gl) for x in grp])
    np.testing.assert_allclose(acc, ref, rtol=1e-10, atol=1e-14)
