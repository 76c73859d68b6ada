"""Training on continuous latents through the C ABI (Sec. 3.2): the model's
tensors live in torch device memory; every step of forward, loss, backward and
Adam runs in the library's kernels."""
from __future__ import annotations

import ctypes
from ctypes import byref, c_size_t, c_void_p

import numpy as np
import torch

from . import _abi
from ._abi import check


def _p(t):
    return c_void_p(0 if t is None else t.data_ptr())


def texel_stride(t: torch.Tensor) -> int:
    """Floats per texel of a latent tensor as the library reads it: 3 for a
    contiguous [h, w, 3], 4 for a contiguous [h, w, 4] (channel 3 is padding) or
    for the [h, w, 3] view of one."""
    if t.dim() == 3 and t.shape[2] in (3, 4) and t.is_contiguous():
        return int(t.shape[2])
    if t.dim() == 3 and t.shape[2] == 3 and t.stride() == (4 * t.shape[1], 4, 1):
        return 4
    raise ValueError("latent tensors are [h, w, 3] or [h, w, 4] with contiguous texels")


def padded(t: torch.Tensor, multiple: int = 4) -> torch.Tensor:
    """[..., C] -> [..., C'] with C' the next multiple of `multiple` and zero
    padding channels: a target in this form is read 16 bytes at a time."""
    c = t.shape[-1]
    cp = -(-c // multiple) * multiple
    out = torch.zeros((*t.shape[:-1], cp), dtype=t.dtype, device=t.device)
    out[..., :c] = t
    return out


class ContinuousModel:
    """Latent pyramid (4 FP32 textures [h, w, 3]) + MLP [12, 64, 64, C] with their
    gradients and Adam moments, on one device.  With latent_stride 4 (the
    default) the latents, their gradients and moments are stored [h, w, 4] with
    a zero padding channel, and `latents[k]` etc. are their [h, w, 3] views."""

    def __init__(self, latents, shifts, weights, biases, device="cuda", latent_stride=4):
        dev = torch.device(device)
        self.device = dev
        if latent_stride not in (3, 4):
            raise ValueError("latent_stride is 3 or 4")
        self.latent_stride = latent_stride

        def store(l):
            l = np.asarray(l, dtype=np.float32)
            buf = torch.zeros((l.shape[0], l.shape[1], latent_stride), dtype=torch.float32, device=dev)
            buf[..., :3] = torch.from_numpy(np.ascontiguousarray(l)).to(dev)
            return buf if latent_stride == 3 else buf[..., :3]

        self.latents = [store(l) for l in latents]
        self.shifts = [float(s) for s in shifts]
        self.dims = [int(weights[0].shape[1])] + [int(w.shape[0]) for w in weights]
        self.weights = torch.from_numpy(np.concatenate([np.asarray(w, np.float32).ravel() for w in weights])).to(dev)
        self.biases = torch.from_numpy(np.concatenate([np.asarray(b, np.float32).ravel() for b in biases])).to(dev)
        z = torch.zeros_like
        zl = lambda l: store(np.zeros(l.shape, np.float32))
        self.latent_grads = [zl(l) for l in self.latents]
        self.latent_m = [zl(l) for l in self.latents]
        self.latent_v = [zl(l) for l in self.latents]
        self._alt_grads = {}   # gradient buffers for caller latents of the other texel stride
        self.grad_w, self.grad_b = z(self.weights), z(self.biases)
        self.m_w, self.v_w, self.m_b, self.v_b = z(self.weights), z(self.weights), z(self.biases), z(self.biases)
        self.step_count = 0
        self.workspace = None

    @classmethod
    def from_synth(cls, wl, device="cuda", latent_stride=4):
        return cls(wl.latents, wl.shifts, wl.mlp.weights, wl.mlp.biases, device, latent_stride)

    def grads_for(self, ls):
        """Latent gradient buffers ([h, w, 3] views) for latents of texel stride ls."""
        if ls == self.latent_stride:
            return self.latent_grads
        if ls not in self._alt_grads:
            self._alt_grads[ls] = [torch.zeros((g.shape[0], g.shape[1], ls), dtype=torch.float32,
                                               device=self.device)[..., :3] for g in self.latent_grads]
        return self._alt_grads[ls]

    def layer_slices(self):
        """(weight, bias) offsets of each layer in the packed parameter vectors."""
        out, wo, bo = [], 0, 0
        for i in range(len(self.dims) - 1):
            n_w, n_b = self.dims[i] * self.dims[i + 1], self.dims[i + 1]
            out.append(((wo, wo + n_w), (bo, bo + n_b)))
            wo += n_w
            bo += n_b
        return out

    def args(self, uv, target=None, loss=_abi.LOSS_MSE, lr_mlp=1e-3, lr_latent=1e-2, betas=(0.9, 0.999),
             eps=1e-8, latents=None, weights=None, biases=None) -> _abi.TrainArgs:
        a = _abi.TrainArgs()
        lats = latents if latents is not None else self.latents
        strides = {texel_stride(l) for l in lats}
        if len(strides) != 1:
            raise ValueError("all latent levels need the same texel stride")
        a.latent_stride = ls = strides.pop()
        grads = self.grads_for(ls)
        a.num_levels = len(lats)
        for k, l in enumerate(lats):
            a.heights[k], a.widths[k] = int(l.shape[0]), int(l.shape[1])
            a.shifts[k] = self.shifts[k]
            a.latents[k] = l.data_ptr()
            a.latent_grads[k] = grads[k].data_ptr()
            a.latent_m[k] = self.latent_m[k].data_ptr()
            a.latent_v[k] = self.latent_v[k].data_ptr()
        a.mlp.num_layers = len(self.dims) - 1
        for i, d in enumerate(self.dims):
            a.mlp.dims[i] = d
        a.mlp.weights = (weights if weights is not None else self.weights).data_ptr()
        a.mlp.biases = (biases if biases is not None else self.biases).data_ptr()
        a.grad_w, a.grad_b = self.grad_w.data_ptr(), self.grad_b.data_ptr()
        a.m_w, a.v_w, a.m_b, a.v_b = (self.m_w.data_ptr(), self.v_w.data_ptr(), self.m_b.data_ptr(),
                                      self.v_b.data_ptr())
        if target is not None:
            if target.dim() != 3 or not target.is_contiguous() or target.shape[2] < self.dims[-1]:
                raise ValueError("target is a contiguous [h, w, >= C] tensor (channels beyond C are padding)")
            a.target = target.data_ptr()
            a.target_h, a.target_w = int(target.shape[0]), int(target.shape[1])
            a.target_stride = int(target.shape[2])
        a.uv = 0 if uv is None or uv.numel() == 0 else uv.data_ptr()
        a.batch = 0 if uv is None else int(uv.shape[0])
        a.step = self.step_count + 1
        a.lr_mlp, a.lr_latent = lr_mlp, lr_latent
        a.beta1, a.beta2, a.eps = betas[0], betas[1], eps
        a.loss = loss
        return a

    def _workspace(self, ctx, a):
        n = c_size_t()
        check(ctx.lib.nbtc_train_workspace_bytes(ctx.handle, byref(a), byref(n)))
        if self.workspace is None or self.workspace.numel() < n.value:
            self.workspace = torch.empty(max(n.value, 16), dtype=torch.uint8, device=self.device)
        a.workspace, a.workspace_bytes = self.workspace.data_ptr(), self.workspace.numel()

    def train_step(self, ctx, uv, target, loss=_abi.LOSS_MSE, stream=None, **kw) -> torch.Tensor:
        """One full step; returns the batch loss as a device scalar."""
        a = self.args(uv, target, loss, **kw)
        self._workspace(ctx, a)
        out = torch.empty(1, dtype=torch.float32, device=self.device)
        s = c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        check(ctx.lib.nbtc_train_step(ctx.handle, byref(a), _p(out), s))
        self.step_count += 1
        return out

    def forward(self, ctx, uv, stream=None, **kw) -> torch.Tensor:
        a = self.args(uv, **kw)
        y = torch.empty((int(uv.shape[0]), self.dims[-1]), dtype=torch.float32, device=self.device)
        s = c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        check(ctx.lib.nbtc_forward_continuous(ctx.handle, byref(a), _p(y), s))
        return y

    def backward(self, ctx, uv, dy, stream=None, **kw):
        """Gradients of sum(dy * y) into grad_w / grad_b / latent_grads."""
        a = self.args(uv, **kw)
        self._workspace(ctx, a)
        s = c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        check(ctx.lib.nbtc_backward_continuous(ctx.handle, byref(a), _p(dy), s))


def _stride_ok(t):
    try:
        texel_stride(t)
        return True
    except ValueError:
        return False


class NbtcDecodeFn(torch.autograd.Function):
    """y = f(uv; latents, W, b): differentiable decode of continuous latents.
    Forward and backward are the library's kernels (activations recomputed in
    the backward, not stored)."""

    @staticmethod
    def forward(fctx, ctx, model, uv, lat0, lat1, lat2, lat3, weights, biases):
        lats = [l if _stride_ok(l) else l.contiguous() for l in (lat0, lat1, lat2, lat3)]
        w, b = weights.contiguous(), biases.contiguous()
        fctx.saved = (ctx, model, uv, lats, w, b)
        return model.forward(ctx, uv, latents=lats, weights=w, biases=b)

    @staticmethod
    def backward(fctx, dy):
        ctx, model, uv, lats, w, b = fctx.saved
        model.backward(ctx, uv, dy.contiguous().float(), latents=lats, weights=w, biases=b)
        grads = model.grads_for(texel_stride(lats[0]))
        return (None, None, None, *[g.clone(memory_format=torch.contiguous_format) if l.shape[2] == 3 else
                                    torch.nn.functional.pad(g, (0, l.shape[2] - 3)) for g, l in zip(grads, lats)],
                model.grad_w.clone(), model.grad_b.clone())


class QatModel(ContinuousModel):
    """Quantisation-aware BC1 latents (Sec. 3.2, Eqs. 1-3) + MLP [12, 64, 64, C]:
    per level raw endpoints e0, e1 [h/4, w/4, 3] and blend factors alpha [h, w]
    with their gradients and Adam moments.  The decoded textures (and their
    gradients) live in the base class's latent buffers, rewritten every step."""

    def __init__(self, e0, e1, alpha, shifts, weights, biases, device="cuda", latent_stride=4):
        dev = torch.device(device)
        f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        decoded = [np.zeros((a.shape[0], a.shape[1], 3), np.float32) for a in alpha]
        super().__init__(decoded, shifts, weights, biases, device, latent_stride)
        self.e0, self.e1, self.alpha = [f32(a) for a in e0], [f32(a) for a in e1], [f32(a) for a in alpha]
        z = torch.zeros_like
        self.g_e0, self.g_e1, self.g_alpha = [z(a) for a in self.e0], [z(a) for a in self.e1], [z(a) for a in self.alpha]
        self.m_e0, self.v_e0 = [z(a) for a in self.e0], [z(a) for a in self.e0]
        self.m_e1, self.v_e1 = [z(a) for a in self.e1], [z(a) for a in self.e1]
        self.m_alpha, self.v_alpha = [z(a) for a in self.alpha], [z(a) for a in self.alpha]

    def level(self, k) -> _abi.QatLevel:
        q = _abi.QatLevel()
        q.height, q.width = int(self.alpha[k].shape[0]), int(self.alpha[k].shape[1])
        for name in ("e0", "e1", "alpha", "g_e0", "g_e1", "g_alpha", "m_e0", "v_e0", "m_e1", "v_e1", "m_alpha",
                     "v_alpha"):
            setattr(q, name, getattr(self, name)[k].data_ptr())
        return q

    def decode_level(self, ctx, k, stream=None) -> torch.Tensor:
        """Decoded texture [h, w, 3] of level k from the current raw parameters."""
        q = self.level(k)
        out = torch.empty((q.height, q.width, 3), dtype=torch.float32, device=self.device)
        s = c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        check(ctx.lib.nbtc_qat_decode(ctx.handle, byref(q), _p(out), s))
        return out

    def encode_level(self, ctx, k, stream=None) -> torch.Tensor:
        """BC1 blocks (int64 view of the uint64 words) of level k."""
        q = self.level(k)
        out = torch.empty((q.height // 4) * (q.width // 4), dtype=torch.int64, device=self.device)
        s = c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        check(ctx.lib.nbtc_qat_encode(ctx.handle, byref(q), _p(out), s))
        return out

    def train_step(self, ctx, uv, target, loss=_abi.LOSS_MSE, stream=None, **kw) -> torch.Tensor:
        """One QAT step (decode, forward, loss, backward, straight-through
        backward, Adam on MLP and raw parameters); returns the batch loss."""
        a = self.args(uv, target, loss, **kw)
        self._workspace(ctx, a)
        levels = (_abi.QatLevel * 4)(*[self.level(k) for k in range(4)])
        out = torch.empty(1, dtype=torch.float32, device=self.device)
        s = c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        check(ctx.lib.nbtc_train_step_qat(ctx.handle, byref(a), levels, _p(out), s))
        self.step_count += 1
        return out
