"""The allocation-free training step, for callers that cannot allocate device
memory (no workspace, no context), gives the same step as nbtc_train_step.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  It creates its own models and context, so it
passes alone in a fresh process as well as after the other tests."""
import ctypes
from ctypes import byref, c_void_p

import numpy as np
import pytest
import torch

import synth
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu
REL = 1e-4   # the gradient tolerance of the training parity tests


def _rel_ok(got, ref):
    got = got.double().cpu().numpy().ravel()
    ref = ref.double().cpu().numpy().ravel()
    nrm = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) <= REL * nrm and np.abs(got - ref).max() <= REL * np.abs(ref).max()


@pytest.mark.parametrize("batch", [3000 + 7, 30000 + 11])
def test_no_alloc_step_matches_workspace_step_twice(batch):
    """batch 3,007: partial sums and gather records both fit the fixed array (the
    step gathers first and runs the tensor-core kernel, as the workspace step
    does); batch 30,011: only the partial sums fit (the step gathers inside the
    SIMT kernel), so the workspace step it is held to runs on a context that
    selects the SIMT kernel too -- the two kernels may take the other side of a
    ReLU kink for a sample whose pre-activation is within rounding of 0, which
    moves that sample's latent gradient by far more than the tolerance."""
    require_gpu()
    import os
    import paper_2506_06040_gb300 as nb
    from paper_2506_06040_gb300 import _abi
    from paper_2506_06040_gb300.train import ContinuousModel

    rng = synth.Rng(91, 1)
    sides = [128, 64, 32, 16]
    lat = [rng.normal(s * s * 3, 0.1).reshape(s, s, 3).astype(np.float32) for s in sides]
    mlp = synth.he_mlp(synth.Rng(91, 2), [12, 64, 64, 9])
    target = synth.sinusoid_target(synth.Rng(91, 3), 256)
    wl = synth.TrainWorkload("no-alloc", sides, synth.SHIFTS, lat, mlp, target, batch, 91)

    simt = batch > 3000 + 7
    if simt:
        os.environ["NBTC_TRAIN_SIMT"] = "1"
    try:
        ctx = nb.Context(0)
    finally:
        os.environ.pop("NBTC_TRAIN_SIMT", None)
    lib = _abi.load()
    ref = ContinuousModel.from_synth(wl)   # nbtc_train_step with a caller workspace
    na = ContinuousModel.from_synth(wl)    # nbtc_train_step_noalloc
    tgt = torch.from_numpy(wl.target).cuda()
    for step in range(2):                  # two calls in a row share the fixed scratch
        uv = torch.from_numpy(wl.uv(step)).cuda()
        loss_ref = ref.train_step(ctx, uv, tgt)
        a = na.args(uv, tgt)
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        rc = lib.nbtc_train_step_noalloc(byref(a), c_void_p(loss.data_ptr()),
                                         c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == _abi.OK, lib.nbtc_last_error()
        na.step_count += 1
        torch.cuda.synchronize()
        assert abs(loss.item() - loss_ref.item()) <= REL * abs(loss_ref.item())
        assert _rel_ok(na.grad_w, ref.grad_w) and _rel_ok(na.grad_b, ref.grad_b)
        for k in range(4):
            assert _rel_ok(na.latent_grads[k], ref.latent_grads[k])
            assert (na.latents[k] - ref.latents[k]).abs().max().item() <= 1e-2 * 1e-3
        assert (na.weights - ref.weights).abs().max().item() <= 1e-3 * 1e-3
    ctx.close()
