"""GPU parity of the split-operand tensor-core forms (every weight and
activation as hi + lo of FP16 or E4M3, three products per layer, FP32
accumulation, FP16 output) against the oracle's emulator -- every output inside
its admissible interval -- and their max abs error against the FP64 oracle per
output channel: at most 2e-3 (FP16 split) and 2e-2 (FP8 split) on the 4096^2
12-64-64-64-9 decode."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
import tc_parity as tp
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

BOUND = {"fp16s": 2e-3, "fp8s": 2e-2}


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


def _code(nb, form):
    return {"fp16": nb.FP16, "fp16s": nb.FP16_SPLIT, "fp8": nb.FP8_E4M3, "fp8s": nb.FP8_E4M3_SPLIT}[form]


def _prepare(nb, ctx, wl, form, calib):
    """Packed MLP of `form` (FP8 forms: calibrated on the calib grid, scales
    checked against the oracle's) and the oracle's scales."""
    mat = nb.Material.from_synth(wl.material)
    if form.startswith("fp8"):
        absmax = nb.fp8_calibrate(ctx, mat, calib[0], calib[1], 16)
        packed = nb.pack_mlp(ctx, mat, _code(nb, form), act_absmax=absmax)
        ctx.sync()
        scales = oracle.decode.fp8_calibration(wl.material, calib[0], calib[1], 16)
        sa_gpu = [float(oracle.quant.pow2_ceil(a / 448.0)) for a in absmax.cpu().numpy().astype(np.float64)]
        assert sa_gpu == scales[1]
        return mat, packed, scales
    return mat, nb.pack_mlp(ctx, mat, _code(nb, form)), None


def _grid_x(material, gw, gh):
    idx = np.arange(gw * gh)
    return oracle.decode.features_at(material, oracle.sample.grid_coord(idx % gw, gw).astype(np.float64),
                                     oracle.sample.grid_coord(idx // gw, gh).astype(np.float64))


@pytest.mark.parametrize("form", ["fp16s", "fp8s"])
@pytest.mark.parametrize("dims", [[12, 64, 9], [12, 64, 64, 9], [12, 64, 64, 64, 9], [12, 32, 32, 9]])
def test_split_grid_every_texel(nb, ctx, form, dims):
    wl = synth.small_decode_workload(512, dims, seed=400 + len(dims) + dims[1])
    mat, packed, scales = _prepare(nb, ctx, wl, form, (512, 96))
    y = nb.decode(ctx, mat, _code(nb, form), packed, grid=(512, 96))
    ctx.sync()
    got = y.float().cpu().numpy()
    st = tp.check_interval(got, wl.material, _grid_x(wl.material, 512, 96), form, scales)
    print(form, dims, st)


@pytest.mark.parametrize("form", ["fp16s", "fp8s"])
@pytest.mark.parametrize("gw,gh", [(200, 72), (130, 3), (7, 5), (128, 1), (65536, 1), (1, 4096), (1024, 300)])
def test_split_ragged_and_extreme(nb, ctx, form, gw, gh):
    """Grids that are not tile multiples, narrower than a tile, a single row of
    65,536 texels, a single column, and a grid spanning many strips."""
    wl = synth.small_decode_workload(256, [12, 64, 64, 64, 9], seed=410)
    mat, packed, scales = _prepare(nb, ctx, wl, form, (256, 256))
    y = nb.decode(ctx, mat, _code(nb, form), packed, grid=(gw, gh))
    ctx.sync()
    tp.check_interval(y.float().cpu().numpy(), wl.material, _grid_x(wl.material, gw, gh), form, scales)


@pytest.mark.parametrize("form", ["fp16s", "fp8s"])
@pytest.mark.parametrize("address", ["clamp", "wrap"])
def test_split_uv_list(nb, ctx, form, address):
    wl = synth.small_decode_workload(256, [12, 64, 64, 9], seed=420, address=address)
    mat, packed, scales = _prepare(nb, ctx, wl, form, (256, 256))
    uv = synth.random_uv(421, 9000 + 77, lo=-0.25, hi=1.25)
    y = nb.decode(ctx, mat, _code(nb, form), packed, uv=torch.from_numpy(uv).cuda())
    ctx.sync()
    x = oracle.decode.features_at(wl.material, uv[:, 0].astype(np.float64), uv[:, 1].astype(np.float64))
    tp.check_interval(y.float().cpu().numpy(), wl.material, x, form, scales)


def test_split_empty_decode(nb, ctx):
    wl = synth.small_decode_workload(256, [12, 64, 64, 9], seed=430)
    mat, packed, _ = _prepare(nb, ctx, wl, "fp16s", None)
    for code in (nb.FP16_SPLIT, nb.FP8_E4M3_SPLIT):
        if code == nb.FP8_E4M3_SPLIT:
            _, packed, _ = _prepare(nb, ctx, wl, "fp8s", (256, 256))
        y = nb.decode(ctx, mat, code, packed, uv=torch.empty((0, 2), dtype=torch.float32, device="cuda"))
        ctx.sync()
        assert y.shape == (0, 9)


@pytest.mark.parametrize("form", ["fp16", "fp16s", "fp32tc", "fp8", "fp8s"])
def test_tmem_and_shared_memory_operands_agree(nb, ctx, form):
    """The tensor-core forms keep their MMA A operands in tensor memory
    (default) or in shared memory (NBTC_TC_TMEM_A=0): the same products in the
    same order, so bit-identical outputs -- on a ragged grid (1024 x 200 plus a
    partial last tile) and a uv list."""
    dims = [12, 64, 64, 9] if form == "fp32tc" else [12, 64, 64, 64, 9]
    wl = synth.small_decode_workload(1024, dims, seed=440)
    code = {"fp16": nb.FP16, "fp16s": nb.FP16_SPLIT, "fp32tc": nb.FP32_TC, "fp8": nb.FP8_E4M3,
            "fp8s": nb.FP8_E4M3_SPLIT}[form]
    os.environ["NBTC_TC_TMEM_A"] = "0"
    try:
        c2 = nb.Context(0)
    finally:
        del os.environ["NBTC_TC_TMEM_A"]
    mat = nb.Material.from_synth(wl.material)
    uv = torch.from_numpy(synth.Rng(441, 1).uniform(2 * 30011, -0.25, 1.25).reshape(-1, 2).astype(np.float32)).cuda()
    for c in (ctx, c2):
        c.sync()
    outs = []
    absmax = nb.fp8_calibrate(ctx, mat, 1024, 200, 16) if form.startswith("fp8") else None
    for c in (ctx, c2):
        packed = nb.pack_mlp(c, mat, code, act_absmax=absmax)
        outs.append((nb.decode(c, mat, code, packed, grid=(1024, 200)), nb.decode(c, mat, code, packed, uv=uv)))
        c.sync()
    iv = torch.int32 if form == "fp32tc" else torch.int16
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a.view(iv), b.view(iv))
    c2.close()


def test_fp16_split_full_size_every_texel_and_error_bound(nb, ctx):
    """The 4096^2 12-64-64-64-9 decode in the benchmark's launch configuration:
    every one of the 16.8M texels inside its admissible interval, and the max abs
    error against the FP64 oracle at most 2e-3 in every channel."""
    wl = synth.decode_workload(2)
    mat, packed, _ = _prepare(nb, ctx, wl, "fp16s", None)
    y = nb.decode(ctx, mat, nb.FP16_SPLIT, packed, grid=(4096, 4096))
    ctx.sync()
    got = y.view(4096, 4096, 9).cpu().numpy()
    _full_size_check("fp16s", got, None)


def test_fp8_split_full_size_error_bound(nb, ctx):
    """The 4096^2 FP8 split decode: 512 rows spread over the texture (every
    texel of them, 2.1M) inside their admissible intervals, max abs error against
    FP64 at most 2e-2 in every channel."""
    wl = synth.decode_workload(2)
    mat, packed, scales = _prepare(nb, ctx, wl, "fp8s", (4096, 4096))
    y = nb.decode(ctx, mat, nb.FP8_E4M3_SPLIT, packed, grid=(4096, 4096))
    ctx.sync()
    got = y.view(4096, 4096, 9).cpu().numpy()
    _full_size_check("fp8s", got, scales, rows_every=8)


def _full_size_check(form, got, scales, rows_every=1):
    band = 32
    tasks = [(2, form, scales, r, n, got[r:r + n].reshape(-1, 9))
             for r, n in tp.bands(4096, band) if (r // band) % rows_every == 0]
    with tp.pool() as p:
        res = p.map(tp.band_form, tasks)
    kern = np.max([r[1] for r in res], axis=0)
    emu = np.max([r[2] for r in res], axis=0)
    equal = np.mean([r[0]["equal"] for r in res])
    single = np.mean([r[0]["single"] for r in res])
    print(f"{form} 4096^2 ({len(tasks) * band} rows): kernel == emulator on {equal:.5f} of outputs, "
          f"single admissible value on {single:.5f}")
    print(f"{form} per-channel max abs error vs FP64, kernel:  ", np.round(kern, 6).tolist())
    print(f"{form} per-channel max abs error vs FP64, emulator:", np.round(emu, 6).tolist())
    assert np.all(kern <= BOUND[form]), kern
