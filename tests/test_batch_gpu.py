"""GPU parity of the batched multi-material decode and the frame pipeline
(Sec. 4, Algorithm 1) against the oracle: every material's FP16 full decode,
every frame pixel's decode, the tile classification counts."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import require_gpu
import tc_parity as tp

pytestmark = pytest.mark.gpu
NAN16 = 0x7E00
# FP32 error of the kernels' features (standard deviation of the interval's
# error model): trilinear features blend two bilinear samples; anisotropic ones
# average up to 16 trilinear probes
SIGMA_TRILINEAR = 2.0 ** -21
SIGMA_ANISO = 2.0 ** -20


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


def _grid_check(mat, S, got, idx):
    uv = np.stack([oracle.sample.grid_coord(idx % S, S), oracle.sample.grid_coord(idx // S, S)], -1).astype(np.float64)
    lod = np.full(len(idx), -64.0)   # mip 0 of every level
    tp.check_interval(got, mat, oracle.frame.pixel_features_direct(mat, uv, lod), "fp16", what="material grid")


def _frame_tensors(bw, nout=9):
    h, w = bw.frame_h, bw.frame_w
    out = torch.full((h, w, nout), 0, dtype=torch.int16, device="cuda")
    out.fill_(NAN16)
    return {"mat_id": torch.from_numpy(bw.mat_id.astype(np.int32)).cuda(),
            "uv": torch.from_numpy(np.ascontiguousarray(bw.uv)).cuda(),
            "lod": torch.from_numpy(np.ascontiguousarray(bw.lod)).cuda(),
            "out": out.view(torch.float16)}


def _frame_check(bw, out, pixels):
    got = out.view(-1, 9)[torch.from_numpy(pixels).cuda()].float().cpu().numpy().astype(np.float64)
    ids = bw.mat_id.reshape(-1)[pixels]
    uv = bw.uv.reshape(-1, 2)[pixels]
    lod = bw.lod.reshape(-1)[pixels]
    for m in np.unique(ids[ids >= 0]):
        sel = ids == m
        mat = bw.materials[m]
        x = oracle.frame.pixel_features_direct(mat, uv[sel], lod[sel])
        tp.check_interval(got[sel], mat, x, "fp16", sigma_x=SIGMA_TRILINEAR, what=f"frame material {m}")
    raw = out.view(torch.int16).view(-1, 9)[torch.from_numpy(pixels).cuda()].cpu().numpy()
    assert np.all(raw[ids < 0] == NAN16)  # pixels without a material are left untouched


def _make(nb, ctx, bw, frame=True, autotune=True):
    mats = [nb.Material.from_synth(m) for m in bw.materials]
    outs = [(torch.empty((S * S, 9), dtype=torch.float16, device="cuda"), S, S) for S in bw.sizes]
    fr = _frame_tensors(bw) if frame else None
    plan = nb.Batch(ctx, mats, outs, fr, autotune=autotune)
    return plan, mats, outs, fr


def test_small_batch_decode_and_frame(nb, ctx):
    bw = synth.batch_workload(num_materials=8, frame_w=512, frame_h=256, smin=256, smax=1024, seed=2024)
    bw.mat_id[np.random.default_rng(1).random(bw.mat_id.shape) < 0.03] = -1   # pixels without material
    plan, mats, outs, fr = _make(nb, ctx, bw)
    plan.decode()
    plan.render()
    ctx.sync()
    rng = np.random.default_rng(3)
    for m, (S, mat) in enumerate(zip(bw.sizes, bw.materials)):
        idx = np.concatenate([rng.integers(0, S * S, 1500), np.arange(S)])
        got = outs[m][0][torch.from_numpy(idx).cuda()].float().cpu().numpy().astype(np.float64)
        _grid_check(mat, S, got, idx)
    _frame_check(bw, fr["out"], np.arange(bw.frame_w * bw.frame_h))
    # classification counts (Algorithm 1 pass A/B) for the tile shape the plan picked
    info = plan.info()
    kind, _ = oracle.frame.classify(bw.mat_id, info["tile_w"], info["tile_h"])
    counts, _ = oracle.frame.mixed_counts(bw.mat_id, kind, info["tile_w"], info["tile_h"], len(bw.materials))
    assert info["frame_uniform_tiles"] == int(np.sum(kind == oracle.frame.UNIFORM))
    assert info["frame_mixed_tiles"] == int(np.sum(kind == oracle.frame.MIXED))
    assert info["frame_packed_tiles"] == int(np.sum((counts + 127) // 128))
    # graph replay gives the same frame
    first = fr["out"].clone()
    plan.render()
    ctx.sync()
    assert torch.equal(first.view(torch.int16), fr["out"].view(torch.int16))
    plan.close()


@pytest.mark.parametrize("shape", [(16, 8), (128, 1)])
def test_frame_without_autotune_all_pixels(nb, ctx, shape):
    bw = synth.batch_workload(num_materials=5, frame_w=256, frame_h=128, smin=256, smax=512, seed=77)
    mats = [nb.Material.from_synth(m) for m in bw.materials]
    fr = _frame_tensors(bw)
    plan = nb.Batch(ctx, mats, None, fr, autotune=False)
    plan.render()
    ctx.sync()
    _frame_check(bw, fr["out"], np.arange(bw.frame_w * bw.frame_h))
    plan.close()


@pytest.mark.parametrize("max_aniso", [16, 4])
def test_frame_anisotropic_filter_all_pixels(nb, ctx, max_aniso):
    """The frame with the anisotropic latent filter (footprints stretched 1x..16x
    down the frame along per-material directions): every pixel against the
    oracle's filter + FP16 emulator."""
    bw = synth.batch_workload(num_materials=5, frame_w=256, frame_h=128, smin=256, smax=512, seed=78)
    mats = [nb.Material.from_synth(m) for m in bw.materials]
    fr = _frame_tensors(bw)
    fr["lod"] = torch.from_numpy(np.ascontiguousarray(bw.lod_bias)).cuda()
    fr["duv"] = torch.from_numpy(np.ascontiguousarray(bw.duv)).cuda()
    fr["max_aniso"] = max_aniso
    plan = nb.Batch(ctx, mats, None, fr, autotune=False)
    plan.render()
    ctx.sync()
    got = fr["out"].view(-1, 9).float().cpu().numpy().astype(np.float64)
    ids = bw.mat_id.reshape(-1)
    uv, duv, bias = bw.uv.reshape(-1, 2), bw.duv.reshape(-1, 4), bw.lod_bias.reshape(-1)
    n, _, _ = oracle.frame.aniso_count(duv, max_aniso)
    assert n.max() == max_aniso and n.min() <= 2
    for m in np.unique(ids[ids >= 0]):
        sel = ids == m
        mat = bw.materials[m]
        mips = [oracle.frame.level_mips_rgb(lv) for lv in mat.levels]
        x = oracle.frame.aniso_features(mat, mips, uv[sel], duv[sel], bias[sel], max_aniso)
        tp.check_interval(got[sel], mat, x, "fp16", sigma_x=SIGMA_ANISO, what=f"aniso frame material {m}")
    plan.close()


def test_frame_lighting_pass(nb, ctx):
    """The fused lighting pass against the oracle's shading of the same FP16
    G-buffer values the kernel produced.  FP32 vs FP64: the GGX term is the only
    ill-conditioned one (near a sharp highlight a relative change e in n.h
    changes D by about cond * e, cond = 4 (n.h)^2 (1 - a^2) / d), so the bound
    is (256 + 16 cond) FP32 ulps of the pixel's largest channel."""
    bw = synth.batch_workload(num_materials=4, frame_w=256, frame_h=128, smin=256, smax=512, seed=79)
    bw.mat_id[np.random.default_rng(2).random(bw.mat_id.shape) < 0.02] = -1
    mats = [nb.Material.from_synth(m) for m in bw.materials]
    fr = _frame_tensors(bw)
    shaded = torch.full((bw.frame_h, bw.frame_w, 4), float("nan"), dtype=torch.float32, device="cuda")
    light = {"light_dir": (0.3, -0.5, 0.8), "light_rgb": (3.0, 2.5, 2.0), "view_dir": (0.1, 0.2, 1.0),
             "sky": (0.5, 0.6, 0.9), "ground": (0.2, 0.15, 0.1)}
    fr["shaded"], fr["light"] = shaded, light
    plan = nb.Batch(ctx, mats, None, fr, autotune=False)
    plan.render()
    ctx.sync()
    ids = bw.mat_id.reshape(-1)
    y = fr["out"].view(-1, 9).float().cpu().numpy().astype(np.float64)[ids >= 0]
    got = shaded.view(-1, 4).cpu().numpy().astype(np.float64)
    assert np.all(np.isnan(got[ids < 0]))           # pixels without a material are left untouched
    got = got[ids >= 0]
    ref = oracle.shade.shade(y, light["light_dir"], light["light_rgb"], light["view_dir"], light["sky"], light["ground"])
    albedo, n, rough, metal, ao = oracle.shade.surface(y)
    l = np.array(light["light_dir"]) / np.linalg.norm(light["light_dir"])
    v = np.array(light["view_dir"]) / np.linalg.norm(light["view_dir"])
    h = (l + v) / np.linalg.norm(l + v)
    a2 = rough ** 4
    x = np.maximum(n @ h, 0.0)
    dd = x * x * (a2 - 1.0) + 1.0
    cond = 4.0 * x * x * (1.0 - a2) / dd
    bound = (256.0 + 16.0 * cond) * 2.0 ** -24 * np.abs(ref).max(axis=1) + 1e-6
    err = np.abs(got[:, :3] - ref).max(axis=1)
    assert np.all(err <= bound), float((err / bound).max())
    assert np.all(got[:, 3] == 1.0)
    assert np.isfinite(got).all()
    plan.close()


def test_full_size_batch(nb, ctx):
    """64 materials of 256^2..4096^2 and a 3840x2160 frame, as the benchmark runs
    them: sampled texels of every material and 20,000 frame pixels."""
    bw = synth.batch_workload()
    plan, mats, outs, fr = _make(nb, ctx, bw)
    plan.decode()
    plan.render()
    ctx.sync()
    rng = np.random.default_rng(4)
    for m, (S, mat) in enumerate(zip(bw.sizes, bw.materials)):
        idx = rng.integers(0, S * S, 300)
        got = outs[m][0][torch.from_numpy(idx).cuda()].float().cpu().numpy().astype(np.float64)
        _grid_check(mat, S, got, idx)
    _frame_check(bw, fr["out"], rng.integers(0, bw.frame_w * bw.frame_h, 20000))
    info = plan.info()
    assert info["decode_tiles"] == sum(S * S // 128 for S in bw.sizes)
    plan.close()


def test_full_size_anisotropic_and_lit_frames(nb, ctx):
    """The benchmark's 3840x2160 frame with the anisotropic latent filter (cap 16)
    and, separately, with the fused lighting pass: 6,000 sampled pixels each
    against the oracle (the lit frame's shading from its own FP16 G-buffer)."""
    bw = synth.batch_workload()
    mats = [nb.Material.from_synth(m) for m in bw.materials]
    rng = np.random.default_rng(8)
    pix = rng.integers(0, bw.frame_w * bw.frame_h, 6000)
    ids = bw.mat_id.reshape(-1)[pix]
    # anisotropic
    fa = _frame_tensors(bw)
    fa["lod"] = torch.from_numpy(np.ascontiguousarray(bw.lod_bias)).cuda()
    fa["duv"] = torch.from_numpy(np.ascontiguousarray(bw.duv)).cuda()
    fa["max_aniso"] = 16
    plan = nb.Batch(ctx, mats, None, fa, autotune=False)
    plan.render()
    ctx.sync()
    got = fa["out"].view(-1, 9)[torch.from_numpy(pix).cuda()].float().cpu().numpy().astype(np.float64)
    uv, duv, bias = bw.uv.reshape(-1, 2)[pix], bw.duv.reshape(-1, 4)[pix], bw.lod_bias.reshape(-1)[pix]
    for m in np.unique(ids[ids >= 0]):
        sel = ids == m
        mat = bw.materials[m]
        mips = [oracle.frame.level_mips_rgb(lv) for lv in mat.levels]
        x = oracle.frame.aniso_features(mat, mips, uv[sel], duv[sel], bias[sel], 16)
        tp.check_interval(got[sel], mat, x, "fp16", sigma_x=SIGMA_ANISO, what=f"aniso frame material {m}")
    plan.close()
    del fa
    # lit
    fl = _frame_tensors(bw)
    shaded = torch.empty((bw.frame_h, bw.frame_w, 4), dtype=torch.float32, device="cuda")
    light = {"light_dir": (0.3, 0.4, 1.0), "light_rgb": (3.0, 3.0, 3.0), "view_dir": (0.0, 0.0, 1.0),
             "sky": (0.6, 0.7, 0.9), "ground": (0.15, 0.12, 0.1)}
    fl["shaded"], fl["light"] = shaded, light
    plan = nb.Batch(ctx, mats, None, fl, autotune=False)
    plan.render()
    ctx.sync()
    keep = ids >= 0
    y = fl["out"].view(-1, 9)[torch.from_numpy(pix[keep]).cuda()].float().cpu().numpy().astype(np.float64)
    lit = shaded.view(-1, 4)[torch.from_numpy(pix[keep]).cuda()].cpu().numpy().astype(np.float64)
    ref = oracle.shade.shade(y, light["light_dir"], light["light_rgb"], light["view_dir"], light["sky"], light["ground"])
    _, n, rough, _, _ = oracle.shade.surface(y)
    l = np.array(light["light_dir"]) / np.linalg.norm(light["light_dir"])
    h = (l + np.array([0.0, 0.0, 1.0])) / np.linalg.norm(l + np.array([0.0, 0.0, 1.0]))
    a2 = rough ** 4
    x = np.maximum(n @ h, 0.0)
    cond = 4.0 * x * x * (1.0 - a2) / (x * x * (a2 - 1.0) + 1.0)
    bound = (256.0 + 16.0 * cond) * 2.0 ** -24 * np.abs(ref).max(axis=1) + 1e-6
    assert np.all(np.abs(lit[:, :3] - ref).max(axis=1) <= bound)
    plan.close()


def test_plan_refuses_host_buffers(nb, ctx):
    """Material outputs are written with bulk copies and frame buffers are read
    and written by the kernels: host buffers are refused when the plan is made."""
    from paper_2506_06040_gb300 import _abi
    mats = [nb.Material.from_synth(synth.small_decode_workload(256, [12, 64, 64, 9], seed=70).material)]
    with pytest.raises(nb.NbtcError) as e:
        nb.Batch(ctx, mats, [(torch.empty((256 * 256, 9), dtype=torch.float16).pin_memory(), 256, 256)],
                 autotune=False)
    assert e.value.code == _abi.ERR_INVALID_ARG
    h, w = 16, 128
    fr = {"mat_id": torch.zeros((h, w), dtype=torch.int32), "uv": torch.zeros((h, w, 2), device="cuda"),
          "lod": torch.zeros((h, w), device="cuda"), "out": torch.empty((h, w, 9), dtype=torch.float16, device="cuda")}
    with pytest.raises(nb.NbtcError) as e:
        nb.Batch(ctx, mats, None, fr, autotune=False)
    assert e.value.code == _abi.ERR_INVALID_ARG
    ctx.sync()
