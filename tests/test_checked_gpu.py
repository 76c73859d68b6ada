"""The bounds-checked build of the library (libnbtc_checked.so, NBTC_CHECKED):
on valid inputs it reports nothing and gives the oracle's results; with a
test-only offset added to every gather index it records NBTC_ERR_BOUNDS once
(each out-of-range index is replaced by a valid one before any access, so
nothing leaves its array) and the context then works again.  Runs the 256^2
decode, a decode from 4x4-block latents, an FP16 tensor-core decode, a training
step and a small frame."""
import numpy as np
import pytest
import torch

import oracle
import synth
import tc_parity as tp
from gpu_util import max_abs, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    require_gpu()
    import paper_2506_06040_gb300 as nb
    return nb


@pytest.fixture(scope="module")
def cctx(nb):
    c = nb.Context(0, checked=True)
    yield c
    c.close()


def _grid_x(material, gw, gh):
    idx = np.arange(gw * gh)
    return oracle.decode.features_at(material, oracle.sample.grid_coord(idx % gw, gw).astype(np.float64),
                                     oracle.sample.grid_coord(idx // gw, gh).astype(np.float64))


def test_checked_decodes_match_the_oracle(nb, cctx):
    from paper_2506_06040_gb300 import _abi
    wl = synth.decode_workload(0)
    mat = nb.Material.from_synth(wl.material)
    y = nb.decode(cctx, mat, grid=(256, 256))
    assert cctx.status() == _abi.OK
    assert max_abs(y.cpu().numpy(), oracle.decode.decode_grid(wl.material, 256, 256)) <= 1e-5
    # latents of 4 x 4 blocks (16 x 16 texels) on every level, 64 x 64 output, clamp and wrap
    for address in ("clamp", "wrap"):
        small = synth.small_decode_workload(64, [12, 64, 64, 9], seed=501, address=address,
                                            level_sides=[16, 16, 16, 16])
        m = nb.Material.from_synth(small.material)
        y = nb.decode(cctx, m, grid=(64, 64))
        assert cctx.status() == _abi.OK
        assert max_abs(y.cpu().numpy(), oracle.decode.decode_grid(small.material, 64, 64)) <= 1e-5
        packed = nb.pack_mlp(cctx, m, nb.FP16)
        y16 = nb.decode(cctx, m, nb.FP16, packed, grid=(128, 64))
        assert cctx.status() == _abi.OK
        tp.check_interval(y16.float().cpu().numpy(), small.material, _grid_x(small.material, 128, 64), "fp16")


def test_checked_planted_indices_report_bounds_and_recover(nb, cctx):
    from paper_2506_06040_gb300 import _abi
    wl = synth.decode_workload(0)
    mat = nb.Material.from_synth(wl.material)
    cctx.set_check_plant(1 << 24)
    try:
        y = nb.decode(cctx, mat, grid=(256, 256))
        assert cctx.status() == _abi.ERR_BOUNDS
        assert cctx.status() == _abi.OK      # reported once, then cleared
        assert torch.isfinite(y).all()       # the replaced indices read valid blocks
        packed = nb.pack_mlp(cctx, mat, nb.FP16)
        nb.decode(cctx, mat, nb.FP16, packed, grid=(256, 64))
        assert cctx.status() == _abi.ERR_BOUNDS
    finally:
        cctx.set_check_plant(0)
    y = nb.decode(cctx, mat, grid=(256, 256))
    assert cctx.status() == _abi.OK
    assert max_abs(y.cpu().numpy(), oracle.decode.decode_grid(wl.material, 256, 256)) <= 1e-5


def test_checked_training_step(nb, cctx):
    """One reduced training step through the checked build: no report, and the
    loss and MLP gradients of the default build; planted tap indices report."""
    from paper_2506_06040_gb300 import _abi
    from paper_2506_06040_gb300.train import ContinuousModel
    wl = synth.train_workload(full=False)
    uv = torch.from_numpy(wl.uv(0)).cuda()
    tgt = torch.from_numpy(wl.target).cuda()
    ref_ctx = nb.Context(0)
    ref = ContinuousModel.from_synth(wl)
    chk = ContinuousModel.from_synth(wl)
    l_ref = ref.train_step(ref_ctx, uv, tgt)
    l_chk = chk.train_step(cctx, uv, tgt)
    assert cctx.status() == _abi.OK
    ref_ctx.sync()
    assert abs(l_chk.item() - l_ref.item()) <= 1e-6 * abs(l_ref.item())
    assert (chk.grad_w - ref.grad_w).abs().max().item() <= 1e-6 * ref.grad_w.abs().max().item()
    cctx.set_check_plant(1 << 24)
    try:
        chk.train_step(cctx, uv, tgt)
        assert cctx.status() == _abi.ERR_BOUNDS
    finally:
        cctx.set_check_plant(0)
    ref_ctx.close()


def test_checked_frame(nb, cctx):
    """A small frame (classification, binning, trilinear decode) through the
    checked build: no report, every pixel inside its admissible interval."""
    from paper_2506_06040_gb300 import _abi
    bw = synth.batch_workload(num_materials=4, frame_w=256, frame_h=128, smin=256, smax=512, seed=81)
    mats = [nb.Material.from_synth(m) for m in bw.materials]
    out = torch.empty((bw.frame_h, bw.frame_w, 9), dtype=torch.float16, device="cuda")
    fr = {"mat_id": torch.from_numpy(bw.mat_id.astype(np.int32)).cuda(),
          "uv": torch.from_numpy(np.ascontiguousarray(bw.uv)).cuda(),
          "lod": torch.from_numpy(np.ascontiguousarray(bw.lod)).cuda(), "out": out}
    plan = nb.Batch(cctx, mats, None, fr, autotune=False)
    plan.render()
    assert cctx.status() == _abi.OK
    got = out.view(-1, 9).float().cpu().numpy()
    ids = bw.mat_id.reshape(-1)
    uv, lod = bw.uv.reshape(-1, 2), bw.lod.reshape(-1)
    for m in np.unique(ids[ids >= 0]):
        sel = ids == m
        x = oracle.frame.pixel_features_direct(bw.materials[m], uv[sel], lod[sel])
        tp.check_interval(got[sel], bw.materials[m], x, "fp16", sigma_x=2.0 ** -21)
    plan.close()


def test_default_build_has_no_plant(nb):
    from paper_2506_06040_gb300 import _abi
    c = nb.Context(0)
    with pytest.raises(nb.NbtcError) as e:
        c.set_check_plant(1)
    assert e.value.code == _abi.ERR_UNSUPPORTED
    c.close()
