"""Checkpoint files round-trip the whole training state exactly (host only):
continuous and QAT models, both latent texel strides, moments and step."""
import numpy as np
import pytest
import torch

import synth
from paper_2506_06040_gb300 import checkpoint
from paper_2506_06040_gb300.train import ContinuousModel, QatModel


def _fill(model, seed):
    g = torch.Generator().manual_seed(seed)
    for name, t in checkpoint._arrays(model).items():
        t.copy_(torch.randn(t.shape, generator=g))
    model.step_count = 17


def _same(a, b):
    xa, xb = checkpoint._arrays(a), checkpoint._arrays(b)
    assert xa.keys() == xb.keys()
    for n in xa:
        assert torch.equal(xa[n].contiguous(), xb[n].contiguous()), n
    assert a.step_count == b.step_count and a.shifts == b.shifts and a.dims == b.dims


@pytest.mark.parametrize("stride", [3, 4])
def test_continuous_round_trip(tmp_path, stride):
    rng = synth.Rng(5, 1)
    sides = [32, 16, 8, 4]
    lat = [rng.normal(s * s * 3, 0.1).reshape(s, s, 3).astype(np.float32) for s in sides]
    mlp = synth.he_mlp(synth.Rng(5, 2), [12, 64, 64, 9])
    m = ContinuousModel(lat, synth.SHIFTS, mlp.weights, mlp.biases, device="cpu", latent_stride=stride)
    _fill(m, 1)
    p = str(tmp_path / "c.ckpt")
    checkpoint.save(m, p)
    _same(m, checkpoint.load(p, device="cpu"))


def test_qat_round_trip(tmp_path):
    rng = synth.Rng(6, 1)
    sides = [16, 8, 8, 4]
    e0 = [rng.normal(s * s // 16 * 3, 1.0).reshape(s // 4, s // 4, 3) for s in sides]
    e1 = [rng.normal(s * s // 16 * 3, 1.0).reshape(s // 4, s // 4, 3) for s in sides]
    al = [rng.normal(s * s, 1.0).reshape(s, s) for s in sides]
    mlp = synth.he_mlp(synth.Rng(6, 2), [12, 64, 64, 5])
    m = QatModel(e0, e1, al, synth.SHIFTS, mlp.weights, mlp.biases, device="cpu")
    _fill(m, 2)
    p = str(tmp_path / "q.ckpt")
    checkpoint.save(m, p)
    r = checkpoint.load(p, device="cpu")
    assert isinstance(r, QatModel)
    _same(m, r)


def test_rejects_other_files(tmp_path):
    p = tmp_path / "x.bin"
    p.write_bytes(b"not a checkpoint")
    with pytest.raises(ValueError):
        checkpoint.load(str(p), device="cpu")
