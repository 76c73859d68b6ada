"""GPU parity of the training path (continuous latents, Sec. 3.2) against the
FP64 oracle: forward outputs, loss, MLP and latent gradients (relative error
1e-4), and the Adam update; plus the autograd.Function."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu
REL = 1e-4


@pytest.fixture(scope="module")
def nb():
    require_gpu()
    import paper_2506_06040_gb300 as nb
    return nb


@pytest.fixture(scope="module")
def ctx(nb):
    c = nb.Context(0)
    yield c
    c.close()


def _check_grad(got, ref, name):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    nrm = np.linalg.norm(ref)
    assert np.linalg.norm(got - ref) <= REL * nrm, (name, np.linalg.norm(got - ref) / nrm)
    assert np.abs(got - ref).max() <= REL * np.abs(ref).max(), (name, np.abs(got - ref).max() / np.abs(ref).max())


def kink_free(wl, uv, margin=1e-5):
    """Drops samples with a hidden pre-activation within `margin` of 0: there the
    ReLU subgradient flips with the last bit of the arithmetic (FP32 vs FP64), a
    difference in which side of the kink is taken, not in the arithmetic."""
    _, cache = oracle.train.forward(wl.latents, wl.shifts, wl.mlp.weights, wl.mlp.biases, uv)
    keep = np.ones(len(uv), dtype=bool)
    for z in cache["pre"][:-1]:
        keep &= np.abs(z).min(axis=1) > margin
    return uv[keep]


def _oracle_grads(wl, uv, kind="mse"):
    y, cache = oracle.train.forward(wl.latents, wl.shifts, wl.mlp.weights, wl.mlp.biases, uv)
    loss, dy = oracle.train.loss_and_dy(y, oracle.train.target_sample(wl.target, uv), kind)
    dW, db, dlat = oracle.train.backward(dy, cache, wl.latents, wl.shifts, wl.mlp.weights)
    return y, loss, dW, db, dlat


def _check_all_grads(model, dW, db, dlat):
    gw, gb = model.grad_w.cpu().numpy(), model.grad_b.cpu().numpy()
    for l, ((w0, w1), (b0, b1)) in enumerate(model.layer_slices()):
        _check_grad(gw[w0:w1], dW[l], f"W{l}")
        _check_grad(gb[b0:b1], db[l], f"b{l}")
    for k in range(4):
        _check_grad(model.latent_grads[k].cpu().numpy(), dlat[k], f"latent{k}")


def _mid_workload(seed=77):
    """Latents 128^2..16^2, target 256^2, batch 20000 (+ a ragged tile)."""
    rng = synth.Rng(seed, 1)
    sides = [128, 64, 32, 16]
    lat = [rng.normal(s * s * 3, 0.1).reshape(s, s, 3).astype(np.float32) for s in sides]
    mlp = synth.he_mlp(synth.Rng(seed, 2), [12, 64, 64, 9])
    target = synth.sinusoid_target(synth.Rng(seed, 3), 256)
    return synth.TrainWorkload("train-mid", sides, synth.SHIFTS, lat, mlp, target, 20000 + 37, seed)


# (latent texel stride, target padded to a multiple of 4 channels): every pairing
# of the 3- and 4-float latent forms with the scalar and 16-byte target reads
@pytest.mark.parametrize("which,kind,layout", [
    ("reduced", "mse", (4, True)), ("reduced", "l1", (3, False)),
    ("mid", "mse", (4, True)), ("mid", "mse", (4, False)), ("mid", "l1", (3, False)), ("mid", "l1", (3, True))])
def test_forward_loss_and_gradients(nb, ctx, which, kind, layout):
    from paper_2506_06040_gb300.train import ContinuousModel, padded
    wl = synth.train_workload(full=False) if which == "reduced" else _mid_workload()
    uv = kink_free(wl, wl.uv(0))
    model = ContinuousModel.from_synth(wl, latent_stride=layout[0])
    uvd = torch.from_numpy(uv).cuda()
    tgt = torch.from_numpy(wl.target).cuda()
    if layout[1]:
        tgt = padded(tgt)
        tgt[..., wl.target.shape[2]:] = float("nan")   # padding channels must never be read into the loss
    y = model.forward(ctx, uvd)
    ctx.sync()
    y_ref, loss_ref, dW, db, dlat = _oracle_grads(wl, uv, kind)
    assert np.abs(y.cpu().numpy() - y_ref).max() <= 1e-5
    loss = model.train_step(ctx, uvd, tgt, loss=nb.LOSS_L1 if kind == "l1" else nb.LOSS_MSE)
    ctx.sync()
    assert abs(float(loss.item()) - loss_ref) <= REL * abs(loss_ref)
    _check_all_grads(model, dW, db, dlat)


def test_adam_updates_three_steps(nb, ctx):
    from paper_2506_06040_gb300.train import ContinuousModel
    wl = synth.train_workload(full=False)
    model = ContinuousModel.from_synth(wl)
    st = oracle.train.init_state(wl.latents, wl.mlp.weights, wl.mlp.biases)
    tgt = torch.from_numpy(wl.target).cuda()
    for step in range(3):
        uv = kink_free(wl, wl.uv(step))
        model.train_step(ctx, torch.from_numpy(uv).cuda(), tgt)
        st = oracle.train.train_step(st, wl.shifts, wl.target, uv)
    ctx.sync()
    # parameters: Adam moves each by about lr per step; compare within lr * 1e-3
    w = model.weights.cpu().numpy()
    for l, ((w0, w1), _) in enumerate(model.layer_slices()):
        assert np.abs(w[w0:w1] - st["weights"][l].ravel()).max() <= 1e-3 * 1e-3
    for k in range(4):
        assert np.abs(model.latents[k].cpu().numpy() - st["latents"][k]).max() <= 1e-2 * 1e-3
        m = model.latent_m[k].cpu().numpy()
        assert np.abs(m - st["m_latents"][k]).max() <= REL * np.abs(st["m_latents"][k]).max() + 1e-12
        # the padding channel of the 4-float texels: zero gradient, untouched by Adam
        for buf in (model.latents[k], model.latent_grads[k], model.latent_m[k], model.latent_v[k]):
            assert buf._base is not None and buf._base.shape[2] == 4
            assert float(buf._base[..., 3].abs().max()) == 0.0


def test_full_size_step(nb, ctx):
    """The benchmark's configuration: latents 1024^2..128^2, target 2048^2 x 9,
    batch 2^20.  MLP gradients and loss against the oracle on the whole batch;
    latent gradients through the full FP64 backward."""
    from paper_2506_06040_gb300.train import ContinuousModel
    wl = synth.train_workload(full=True)
    uv = kink_free(wl, wl.uv(0))
    assert len(uv) > 0.95 * wl.batch
    from paper_2506_06040_gb300.train import padded
    model = ContinuousModel.from_synth(wl)   # the benchmark's layouts: 4-float latents, padded target
    loss = model.train_step(ctx, torch.from_numpy(uv).cuda(), padded(torch.from_numpy(wl.target).cuda()))
    ctx.sync()
    _, loss_ref, dW, db, dlat = _oracle_grads(wl, uv)
    assert abs(float(loss.item()) - loss_ref) <= REL * abs(loss_ref)
    _check_all_grads(model, dW, db, dlat)


@pytest.mark.parametrize("lat_channels", [3, 4])
def test_autograd_function(nb, ctx, lat_channels):
    """Leaf latents [h, w, 3] (read 3 floats per texel) or [h, w, 4] with a padding
    channel (16-byte texels; its gradient is 0)."""
    from paper_2506_06040_gb300.train import ContinuousModel, NbtcDecodeFn
    wl = synth.train_workload(full=False)
    uv = kink_free(wl, wl.uv(1))
    model = ContinuousModel.from_synth(wl)
    lats = [torch.nn.functional.pad(l, (0, lat_channels - 3)).contiguous().requires_grad_(True)
            for l in model.latents]
    w = model.weights.clone().requires_grad_(True)
    b = model.biases.clone().requires_grad_(True)
    uvd = torch.from_numpy(uv).cuda()
    y = NbtcDecodeFn.apply(ctx, model, uvd, *lats, w, b)
    t = torch.from_numpy(oracle.train.target_sample(wl.target, uv)).cuda().float()
    loss = ((y - t) ** 2).mean()
    loss.backward()
    _, loss_ref, dW, db, dlat = _oracle_grads(wl, uv)
    assert abs(float(loss.item()) - loss_ref) <= REL * abs(loss_ref)
    gw, gb = w.grad.cpu().numpy(), b.grad.cpu().numpy()
    for l, ((w0, w1), (b0, b1)) in enumerate(model.layer_slices()):
        _check_grad(gw[w0:w1], dW[l], f"W{l}")
        _check_grad(gb[b0:b1], db[l], f"b{l}")
    for k in range(4):
        assert lats[k].grad.shape == lats[k].shape
        _check_grad(lats[k].grad[..., :3].cpu().numpy(), dlat[k], f"latent{k}")
        if lat_channels == 4:
            assert float(lats[k].grad[..., 3].abs().max()) == 0.0


def test_empty_batch_and_invalid(nb, ctx):
    from paper_2506_06040_gb300.train import ContinuousModel
    wl = synth.train_workload(full=False)
    model = ContinuousModel.from_synth(wl)
    y = model.forward(ctx, torch.empty((0, 2), device="cuda"))
    assert y.shape == (0, 9)
    with pytest.raises(nb.NbtcError):
        model.train_step(ctx, torch.from_numpy(wl.uv(0)).cuda(), None)  # no target
    ctx.sync()


def test_invalid_strides(nb, ctx):
    import ctypes
    from paper_2506_06040_gb300 import _abi
    from paper_2506_06040_gb300.train import ContinuousModel
    wl = synth.train_workload(full=False)
    model = ContinuousModel.from_synth(wl)
    uv = torch.from_numpy(wl.uv(0)).cuda()
    tgt = torch.from_numpy(wl.target).cuda()
    loss = torch.empty(1, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def run(edit):
        a = model.args(uv, tgt)
        model._workspace(ctx, a)
        edit(a)
        return ctx.lib.nbtc_train_step(ctx.handle, ctypes.byref(a), ctypes.c_void_p(loss.data_ptr()), s)

    assert run(lambda a: setattr(a, "latent_stride", 5)) == _abi.ERR_INVALID_ARG
    assert run(lambda a: setattr(a, "target_stride", 8)) == _abi.ERR_INVALID_ARG   # < C = 9
    # 4-float texels must start on a 16-byte boundary
    assert run(lambda a: a.latents.__setitem__(1, a.latents[1] + 4)) == _abi.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        model.train_step(ctx, uv, tgt[..., :8].contiguous())
    # a pageable host target or uv is refused before any launch
    tgt_host = tgt.cpu()
    assert run(lambda a: setattr(a, "target", tgt_host.data_ptr())) == _abi.ERR_INVALID_ARG
    uv_host = uv.cpu()
    assert run(lambda a: setattr(a, "uv", uv_host.data_ptr())) == _abi.ERR_INVALID_ARG
    # the workspace must be device memory; the loss device or pinned host memory;
    # latent gradients (atomic adds) device memory, also when the host's are pinned
    ws_host = torch.empty(64 << 20, dtype=torch.uint8)
    assert run(lambda a: setattr(a, "workspace", ws_host.data_ptr())) == _abi.ERR_INVALID_ARG
    ws_pinned = torch.empty(64 << 20, dtype=torch.uint8).pin_memory()
    assert run(lambda a: setattr(a, "workspace", ws_pinned.data_ptr())) == _abi.ERR_INVALID_ARG
    g_pinned = torch.zeros(model.latent_grads[2].numel(), dtype=torch.float32).pin_memory()
    assert run(lambda a: a.latent_grads.__setitem__(2, g_pinned.data_ptr())) == _abi.ERR_INVALID_ARG
    a = model.args(uv, tgt)
    model._workspace(ctx, a)
    loss_host = torch.empty(1)
    assert ctx.lib.nbtc_train_step(ctx.handle, ctypes.byref(a), ctypes.c_void_p(loss_host.data_ptr()),
                                   s) == _abi.ERR_INVALID_ARG
    y_host = torch.empty((uv.shape[0], 9))
    assert ctx.lib.nbtc_forward_continuous(ctx.handle, ctypes.byref(a), ctypes.c_void_p(y_host.data_ptr()),
                                           s) == _abi.ERR_INVALID_ARG
    dy_host = torch.zeros((uv.shape[0], 9))
    assert ctx.lib.nbtc_backward_continuous(ctx.handle, ctypes.byref(a), ctypes.c_void_p(dy_host.data_ptr()),
                                            s) == _abi.ERR_INVALID_ARG
    # a pinned host loss is written over the host link
    loss_pinned = torch.zeros(1).pin_memory()
    a = model.args(uv, tgt)
    model._workspace(ctx, a)
    assert ctx.lib.nbtc_train_step(ctx.handle, ctypes.byref(a), ctypes.c_void_p(loss_pinned.data_ptr()),
                                   s) == _abi.OK
    ctx.sync()
    assert float(loss_pinned[0]) > 0


def test_layouts_give_the_same_step(nb, ctx):
    """4-float latent texels with a padded target run the 3-float form's arithmetic
    term for term: the same loss and MLP gradients bit for bit; latent gradients
    equal up to the order of the atomic adds."""
    from paper_2506_06040_gb300.train import ContinuousModel, padded
    wl = _mid_workload(seed=78)
    uv = torch.from_numpy(wl.uv(0)).cuda()
    tgt = torch.from_numpy(wl.target).cuda()
    m3 = ContinuousModel.from_synth(wl, latent_stride=3)
    m4 = ContinuousModel.from_synth(wl, latent_stride=4)
    l3 = m3.train_step(ctx, uv, tgt)
    l4 = m4.train_step(ctx, uv, padded(tgt))
    ctx.sync()
    assert torch.equal(l3, l4)
    assert torch.equal(m3.grad_w, m4.grad_w) and torch.equal(m3.grad_b, m4.grad_b)
    assert torch.equal(m3.weights, m4.weights)
    for k in range(4):
        g3, g4 = m3.latent_grads[k], m4.latent_grads[k]
        assert (g3 - g4).abs().max().item() <= 1e-6 * g3.abs().max().item()


@pytest.fixture(scope="module")
def simt_ctx(nb):
    """A context whose steps run every sample on the FP32 SIMT training kernel
    (NBTC_TRAIN_SIMT=1, read when the context is created)."""
    import os
    os.environ["NBTC_TRAIN_SIMT"] = "1"
    try:
        c = nb.Context(0)
    finally:
        del os.environ["NBTC_TRAIN_SIMT"]
    yield c
    c.close()


def _raw_step(ctx, wl, uv, tgt, partials_only):
    """One nbtc_train_step on a fresh model; partials_only: a workspace with room
    for the per-CTA partial sums only (2 x 6033 floats per CTA, one CTA per
    256-sample tile or SM), so the step gathers inside its main kernel."""
    import ctypes
    from paper_2506_06040_gb300.train import ContinuousModel
    m = ContinuousModel.from_synth(wl)
    a = m.args(uv, tgt)
    m._workspace(ctx, a)
    if partials_only:
        grid = min(-(-int(uv.shape[0]) // 256), torch.cuda.get_device_properties(0).multi_processor_count)
        a.workspace_bytes = grid * 2 * 6033 * 4
    loss = torch.empty(1, device="cuda")
    assert ctx.lib.nbtc_train_step(ctx.handle, ctypes.byref(a), ctypes.c_void_p(loss.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    ctx.sync()
    return loss.clone(), m.grad_w.clone(), m.grad_b.clone(), [g.clone() for g in m.latent_grads]


def test_pre_gathered_and_fused_gather_agree(nb, simt_ctx):
    """On the SIMT kernel, a workspace with room for the batch makes the step
    gather every sample's features and target first (k_gather); one that only
    holds the partial sums makes it gather inside the training kernel.  Same
    arithmetic: the same loss and MLP gradients bit for bit."""
    from paper_2506_06040_gb300.train import padded
    wl = _mid_workload(seed=79)
    uv = torch.from_numpy(wl.uv(0)).cuda()
    tgt = padded(torch.from_numpy(wl.target).cuda())
    r = [_raw_step(simt_ctx, wl, uv, tgt, small) for small in (False, True)]
    assert torch.equal(r[0][0], r[1][0])
    assert torch.equal(r[0][1], r[1][1]) and torch.equal(r[0][2], r[1][2])
    for g0, g1 in zip(r[0][3], r[1][3]):
        assert (g0 - g1).abs().max().item() <= 1e-6 * g0.abs().max().item()


@pytest.mark.parametrize("which", ["mid", "full"])
def test_tensor_core_and_simt_steps_agree(nb, ctx, simt_ctx, which):
    """The tensor-core step (pre-gathered samples, split FP16 operands with FP32
    accumulation) against the FP32 SIMT step on the same kink-free batch: loss
    and MLP gradients within 1e-5 relative, latent gradients within 1e-5 of
    their largest magnitude.  The FP64 parity tests above hold each one to the
    oracle at 1e-4; this bounds the two kernels' difference directly."""
    from paper_2506_06040_gb300.train import padded
    wl = _mid_workload(seed=81) if which == "mid" else synth.train_workload(full=True)
    uv = torch.from_numpy(kink_free(wl, wl.uv(0))).cuda()
    tgt = padded(torch.from_numpy(wl.target).cuda())
    tc = _raw_step(ctx, wl, uv, tgt, False)
    ref = _raw_step(simt_ctx, wl, uv, tgt, False)
    tol = 1e-5
    assert abs(tc[0].item() - ref[0].item()) <= tol * abs(ref[0].item())
    for got, want in ((tc[1], ref[1]), (tc[2], ref[2])):
        d = (got - want).double()
        assert d.norm().item() <= tol * want.double().norm().item()
    for g, w in zip(tc[3], ref[3]):
        assert (g - w).abs().max().item() <= tol * w.abs().max().item()


@pytest.mark.parametrize("C,pad", [(3, False), (12, True), (13, True), (16, False), (5, True)])
def test_channel_counts(nb, ctx, C, pad):
    """Output widths either side of the kernels' 12 / 16-channel paddings, with
    plain and padded targets: loss and every gradient against the oracle."""
    from paper_2506_06040_gb300.train import ContinuousModel, padded
    rng = synth.Rng(200 + C, 1)
    sides = [64, 32, 16, 8]
    lat = [rng.normal(s * s * 3, 0.1).reshape(s, s, 3).astype(np.float32) for s in sides]
    mlp = synth.he_mlp(synth.Rng(200 + C, 2), [12, 64, 64, C])
    target = synth.sinusoid_target(synth.Rng(200 + C, 3), 128, channels=C)
    wl = synth.TrainWorkload("train-C", sides, synth.SHIFTS, lat, mlp, target, 5000 + 13, 200 + C)
    uv = kink_free(wl, wl.uv(0))
    model = ContinuousModel.from_synth(wl)
    tgt = torch.from_numpy(wl.target).cuda()
    loss = model.train_step(ctx, torch.from_numpy(uv).cuda(), padded(tgt) if pad else tgt)
    ctx.sync()
    _, loss_ref, dW, db, dlat = _oracle_grads(wl, uv)
    assert abs(float(loss.item()) - loss_ref) <= REL * abs(loss_ref)
    _check_all_grads(model, dW, db, dlat)


def test_resume_from_checkpoint(nb, ctx, tmp_path):
    """Two steps, save, one more step -- against load and one step: the resumed
    step starts from exactly the saved state, so its loss and MLP update are
    bit-identical (deterministic sums); the latent update matches up to the
    order of the gradient's atomic adds."""
    from paper_2506_06040_gb300 import checkpoint
    from paper_2506_06040_gb300.train import ContinuousModel, padded
    wl = _mid_workload(seed=80)
    tgt = padded(torch.from_numpy(wl.target).cuda())
    a = ContinuousModel.from_synth(wl)
    for i in range(2):
        a.train_step(ctx, torch.from_numpy(wl.uv(i)).cuda(), tgt)
    path = str(tmp_path / "state.ckpt")
    checkpoint.save(a, path)
    b = checkpoint.load(path)
    uv = torch.from_numpy(wl.uv(2)).cuda()
    la = a.train_step(ctx, uv, tgt)
    lb = b.train_step(ctx, uv, tgt)
    ctx.sync()
    assert torch.equal(la, lb)
    assert torch.equal(a.weights, b.weights) and torch.equal(a.biases, b.biases)
    assert torch.equal(a.m_w, b.m_w) and torch.equal(a.v_w, b.v_w)
    for k in range(4):
        assert (a.latents[k] - b.latents[k]).abs().max().item() <= 1e-6
    assert a.step_count == b.step_count == 3
