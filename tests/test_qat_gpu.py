"""GPU parity of the quantisation-aware BC1 latents (Sec. 3.2, Eqs. 1-3)
against the FP64 oracle: the decode of raw parameters, the encoder (bit-exact),
and the QAT training step (loss, straight-through gradients, Adam update)."""
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


def _params(seed, sides, scale=2.0):
    rng = synth.Rng(seed, 5)
    e0 = [rng.normal(s * s // 16 * 3, scale).reshape(s // 4, s // 4, 3).astype(np.float32) for s in sides]
    e1 = [rng.normal(s * s // 16 * 3, scale).reshape(s // 4, s // 4, 3).astype(np.float32) for s in sides]
    al = [rng.normal(s * s, scale).reshape(s, s).astype(np.float32) for s in sides]
    return e0, e1, al


def _model(e0, e1, al, mlp_seed=9, C=9, latent_stride=4):
    from paper_2506_06040_gb300.train import QatModel
    mlp = synth.he_mlp(synth.Rng(mlp_seed, 2), [12, 64, 64, C])
    return QatModel(e0, e1, al, synth.SHIFTS, mlp.weights, mlp.biases, latent_stride=latent_stride), mlp


def _check_grad(got, ref, name):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    nrm = np.linalg.norm(ref)
    assert np.linalg.norm(got - ref) <= REL * nrm, (name, np.linalg.norm(got - ref) / nrm)
    assert np.abs(got - ref).max() <= REL * np.abs(ref).max(), (name, np.abs(got - ref).max() / np.abs(ref).max())


def _with_threshold_values(e0, e1, al):
    """Puts some parameters exactly on (and one FP32 step beside) the quantisers'
    decision thresholds, where an exp-based decision would be fragile."""
    t2, t5, t6 = oracle.qat.thresholds(2), oracle.qat.thresholds(5), oracle.qat.thresholds(6)
    a = al[0].reshape(-1)
    for i, t in enumerate(np.concatenate([t2, t2])):
        if 3 * i + 2 >= a.size:
            break
        a[3 * i] = t
        a[3 * i + 1] = np.nextafter(t, np.float32(-np.inf))
        a[3 * i + 2] = np.nextafter(t, np.float32(np.inf))
    e = e0[0].reshape(-1, 3)
    for i in range(min(len(e), 31)):
        e[i, 0], e[i, 1], e[i, 2] = t5[i], t6[2 * i], np.nextafter(t5[i], np.float32(np.inf))


def _expansion_error():
    e = 0.0
    for bits in (5, 6):
        n = (1 << bits) - 1
        k = np.arange(n + 1)
        rep = (k << (8 - bits)) | (k >> (2 * bits - 8))
        e = max(e, float(np.max(np.abs(rep - 255.0 * k / n))))
    return e


def _bc1_decode(ctx, blocks, w, h):
    import ctypes
    from paper_2506_06040_gb300 import _abi
    d = torch.from_numpy(blocks.view(np.int64).copy()).cuda()
    lv = _abi.Level()
    lv.blocks, lv.width, lv.height, lv.num_mips, lv.shift = d.data_ptr(), w, h, 1, 0.0
    out = torch.empty((h, w, 3), dtype=torch.uint8, device="cuda")
    assert ctx.lib.nbtc_bc1_decode_level(ctx.handle, ctypes.byref(lv), 0, ctypes.c_void_p(out.data_ptr()), None) == 0
    ctx.sync()
    return out.cpu().numpy()


@pytest.mark.parametrize("side", [4, 64, 128])
def test_decode_and_encode(nb, ctx, side):
    e0, e1, al = _params(40 + side, [side, side, side, side])
    _with_threshold_values(e0, e1, al)
    model, _ = _model(e0, e1, al)
    for k in (0, 1):
        T = model.decode_level(ctx, k).cpu().numpy().astype(np.float64)
        ref = oracle.qat.decode(e0[k], e1[k], al[k])
        assert np.max(np.abs(T - ref)) <= 1e-6
        blocks = model.encode_level(ctx, k).cpu().numpy().view(np.uint64)
        want = oracle.qat.encode(e0[k], e1[k], al[k])
        assert np.array_equal(blocks, want)
        # the encoded blocks decode (library BC1 decode) to the QAT texture within
        # BC1 rounding: 5/6-bit replication vs k / (2^b - 1), plus 1/3 from the thirds
        rgb = _bc1_decode(ctx, blocks, side, side)
        err = np.abs(rgb.astype(np.float64) - 255.0 * ref).max()
        assert err <= _expansion_error() + 1.0 / 3.0 + 1e-9


def _qat_workload(seed=61):
    sides = [32, 16, 8, 4]
    e0, e1, al = _params(seed, sides, scale=1.5)
    target = synth.sinusoid_target(synth.Rng(seed, 3), 64)
    uv = synth.random_uv(seed, 3000 + 17)
    return sides, e0, e1, al, target, uv


@pytest.mark.parametrize("latent_stride", [3, 4])
def test_qat_step_matches_oracle(nb, ctx, latent_stride):
    sides, e0, e1, al, target, uv = _qat_workload()
    model, mlp = _model(e0, e1, al, latent_stride=latent_stride)
    # kink-free batch on the decoded textures (see the continuous-latent tests)
    T = [oracle.qat.decode(a, b, c) for a, b, c in zip(e0, e1, al)]
    _, cache = oracle.train.forward(T, synth.SHIFTS, mlp.weights, mlp.biases, uv)
    keep = np.ones(len(uv), dtype=bool)
    for z in cache["pre"][:-1]:
        keep &= np.abs(z).min(axis=1) > 1e-5
    uv = uv[keep]
    st = oracle.qat.init_state(e0, e1, al, mlp.weights, mlp.biases)
    ref = oracle.qat.train_step(st, synth.SHIFTS, target, uv)
    loss = model.train_step(ctx, torch.from_numpy(uv).cuda(), torch.from_numpy(target).cuda())
    ctx.sync()
    assert abs(float(loss.item()) - ref["loss"]) <= 1e-5 * ref["loss"]
    for k in range(4):
        _check_grad(model.latent_grads[k].cpu().numpy(), ref["grad_T"][k], f"dT{k}")
        _check_grad(model.g_e0[k].cpu().numpy(), ref["grad_e0"][k], f"e0_{k}")
        _check_grad(model.g_e1[k].cpu().numpy(), ref["grad_e1"][k], f"e1_{k}")
        _check_grad(model.g_alpha[k].cpu().numpy(), ref["grad_alpha"][k], f"alpha{k}")
        for name in ("e0", "e1", "alpha"):
            got = getattr(model, name)[k].cpu().numpy().astype(np.float64)
            want, before, g = ref[name][k], st[name][k], ref["grad_" + name][k]
            # the first Adam step moves a parameter by lr g / (|g| + eps): compare the
            # moves where the gradient is clearly away from 0 (elsewhere its sign is
            # within the FP32 summation noise), and require no move where it is 0
            clear = np.abs(g) > 1e-3 * np.abs(g).max()
            assert clear.mean() > 0.5
            _check_grad((got - before)[clear], (want - before)[clear], f"{name}{k} update")
            assert np.all(got[g == 0] == before[g == 0])
    gw = model.grad_w.cpu().numpy()
    for l, ((w0, w1), _) in enumerate(model.layer_slices()):
        _check_grad(gw[w0:w1], ref["grad_w"][l], f"W{l}")


def test_qat_steps_then_encode(nb, ctx):
    """A few steps on the device, then the trained parameters' decode and
    encoding still agree with the oracle applied to the same parameters."""
    sides, e0, e1, al, target, uv = _qat_workload(seed=62)
    model, _ = _model(e0, e1, al)
    uv_d, tg = torch.from_numpy(uv).cuda(), torch.from_numpy(target).cuda()
    losses = [float(model.train_step(ctx, uv_d, tg).item()) for _ in range(5)]
    ctx.sync()
    assert all(np.isfinite(losses))
    for k in range(4):
        p = [getattr(model, n)[k].cpu().numpy() for n in ("e0", "e1", "alpha")]
        T = model.decode_level(ctx, k).cpu().numpy().astype(np.float64)
        assert np.max(np.abs(T - oracle.qat.decode(*p))) <= 1e-6
        blocks = model.encode_level(ctx, k).cpu().numpy().view(np.uint64)
        assert np.array_equal(blocks, oracle.qat.encode(*p))


def test_invalid_arguments(nb, ctx):
    from paper_2506_06040_gb300 import _abi
    e0, e1, al = _params(3, [8, 8, 8, 8])
    model, _ = _model(e0, e1, al)
    q = model.level(0)
    q.width = 6
    import ctypes
    out = torch.empty(8 * 8 * 3, device="cuda")
    assert ctx.lib.nbtc_qat_decode(ctx.handle, ctypes.byref(q), ctypes.c_void_p(out.data_ptr()), None) == \
        _abi.ERR_INVALID_ARG


def test_qat_full_size_step(nb, ctx):
    """The benchmark's QAT configuration: levels 1024^2..128^2 of raw parameters
    N(0, 1), target 2048^2 x 9, batch 2^20: loss, the straight-through gradients
    and the MLP gradients against the oracle on the whole batch."""
    wl = synth.train_workload(full=True)
    rng = synth.Rng(1003, 9)
    sides = wl.latent_sides
    e0 = [rng.normal(s * s // 16 * 3, 1.0).reshape(s // 4, s // 4, 3).astype(np.float32) for s in sides]
    e1 = [rng.normal(s * s // 16 * 3, 1.0).reshape(s // 4, s // 4, 3).astype(np.float32) for s in sides]
    al = [rng.normal(s * s, 1.0).reshape(s, s).astype(np.float32) for s in sides]
    from paper_2506_06040_gb300.train import QatModel
    model = QatModel(e0, e1, al, wl.shifts, wl.mlp.weights, wl.mlp.biases)
    uv = wl.uv(0)
    T = [oracle.qat.decode(a, b, c) for a, b, c in zip(e0, e1, al)]
    _, cache = oracle.train.forward(T, wl.shifts, wl.mlp.weights, wl.mlp.biases, uv)
    keep = np.ones(len(uv), dtype=bool)
    for z in cache["pre"][:-1]:
        keep &= np.abs(z).min(axis=1) > 1e-5
    uv = uv[keep]
    assert len(uv) > 0.95 * wl.batch
    st = oracle.qat.init_state(e0, e1, al, wl.mlp.weights, wl.mlp.biases)
    ref = oracle.qat.train_step(st, wl.shifts, wl.target, uv)
    from paper_2506_06040_gb300.train import padded
    loss = model.train_step(ctx, torch.from_numpy(uv).cuda(), padded(torch.from_numpy(wl.target).cuda()))
    ctx.sync()
    assert abs(float(loss.item()) - ref["loss"]) <= REL * ref["loss"]
    for k in range(4):
        _check_grad(model.g_e0[k].cpu().numpy(), ref["grad_e0"][k], f"e0_{k}")
        _check_grad(model.g_e1[k].cpu().numpy(), ref["grad_e1"][k], f"e1_{k}")
        _check_grad(model.g_alpha[k].cpu().numpy(), ref["grad_alpha"][k], f"alpha{k}")
    gw = model.grad_w.cpu().numpy()
    for l, ((w0, w1), _) in enumerate(model.layer_slices()):
        _check_grad(gw[w0:w1], ref["grad_w"][l], f"W{l}")
