"""GPU parity of the BC1 decode (bit-exact) and the FP32 fused decode
(max abs error 1e-5 against the FP64 oracle), through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import max_abs, require_gpu

pytestmark = pytest.mark.gpu
TOL_FP32 = 1e-5


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


@pytest.mark.parametrize("k", [0, 1])
def test_bc1_every_texel_every_level(nb, ctx, k):
    wl = synth.decode_workload(k)
    mat = nb.Material.from_synth(wl.material)
    for i, lv in enumerate(wl.material.levels):
        got = nb.bc1_decode_level(ctx, mat, i).cpu().numpy()
        want = oracle.bc1.decode_level(lv.blocks[0], lv.width, lv.height)
        assert np.array_equal(got, want), f"level {i}"
    ctx.sync()


def test_bc1_mips_and_golden_blocks(nb, ctx):
    bw = synth.batch_workload(num_materials=1, frame_w=32, frame_h=16, smin=512, smax=512)
    m = bw.materials[0]
    mat = nb.Material.from_synth(m)
    for i, lv in enumerate(m.levels):
        w = lv.width
        for mip in range(lv.num_mips):
            got = nb.bc1_decode_level(ctx, mat, i, mip).cpu().numpy()
            want = oracle.bc1.decode_level(lv.blocks[mip], w, w)
            assert np.array_equal(got, want), (i, mip)
            w = max(4, w // 2)


def test_decode_config0_full(nb, ctx):
    wl = synth.decode_workload(0)
    mat = nb.Material.from_synth(wl.material)
    y = nb.decode(ctx, mat, grid=(256, 256))
    ctx.sync()
    ref = oracle.decode.decode_grid(wl.material, 256, 256)
    assert max_abs(y.cpu().numpy(), ref) <= TOL_FP32


@pytest.mark.parametrize("gw,gh", [(200, 136), (333, 3), (1, 1), (4, 1), (129, 65)])
def test_decode_ragged_grids(nb, ctx, gw, gh):
    wl = synth.decode_workload(0)
    mat = nb.Material.from_synth(wl.material)
    y = nb.decode(ctx, mat, grid=(gw, gh))
    ctx.sync()
    ref = oracle.decode.decode_grid(wl.material, gw, gh)
    assert max_abs(y.cpu().numpy(), ref) <= TOL_FP32


@pytest.mark.parametrize("gw,gh", [(200, 136), (333, 3), (1, 1), (768, 5), (4096, 2), (1280, 9), (65536, 1), (1, 4096)])
def test_decode_ragged_grids_wide(nb, ctx, gw, gh):
    """The wide kernel (hidden width 64, two hidden layers): grids whose width is
    not a multiple of its 256-texel tiles (per-texel features, ragged last tile),
    widths that are (row-footprint features), and grids with fewer tiles than
    thread groups."""
    wl = synth.small_decode_workload(1024, [12, 64, 64, 9], seed=31)
    mat = nb.Material.from_synth(wl.material)
    y = nb.decode(ctx, mat, grid=(gw, gh))
    ctx.sync()
    ref = oracle.decode.decode_grid(wl.material, gw, gh)
    assert max_abs(y.cpu().numpy(), ref) <= TOL_FP32


def test_wide_kernel_group_counts_agree(nb):
    """One 512-thread group per CTA (NBTC_FP32_GROUPS=1) and two 256-thread groups
    compute every texel with the same arithmetic: bit-identical outputs."""
    import os
    wl = synth.small_decode_workload(1024, [12, 64, 64, 9], seed=32)
    outs = []
    for groups in ("1", "2"):
        old = os.environ.get("NBTC_FP32_GROUPS")
        os.environ["NBTC_FP32_GROUPS"] = groups
        try:
            c = nb.Context(0)
        finally:
            if old is None:
                del os.environ["NBTC_FP32_GROUPS"]
            else:
                os.environ["NBTC_FP32_GROUPS"] = old
        mat = nb.Material.from_synth(wl.material)
        outs.append([nb.decode(c, mat, grid=g).cpu() for g in ((1024, 256), (1000, 37))])
        outs[-1].append(nb.decode(c, mat, uv=torch.from_numpy(synth.random_uv(5, 3001)).cuda()).cpu())
        c.sync()
        c.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("address", ["clamp", "wrap"])
def test_decode_uv_list(nb, ctx, address):
    wl = synth.small_decode_workload(128, [12, 64, 64, 9], seed=77, address=address)
    mat = nb.Material.from_synth(wl.material)
    uv = synth.random_uv(78, 20001, lo=-0.5, hi=1.5)
    y = nb.decode(ctx, mat, uv=torch.from_numpy(uv).cuda())
    ctx.sync()
    ref = oracle.decode.decode_uv(wl.material, uv)
    assert max_abs(y.cpu().numpy(), ref) <= TOL_FP32


@pytest.mark.parametrize("dims,layout", [([12, 16, 9], "B"), ([12, 32, 9], "B"), ([12, 64, 9], "B"),
                                         ([12, 32, 32, 9], "B"), ([12, 64, 64, 64, 9], "B"), ([12, 16, 16, 9], "A"),
                                         ([12, 32, 32, 32, 9], "A"), ([12, 16, 16, 16, 9], "B")])
def test_decode_mlp_shapes(nb, ctx, dims, layout):
    """Hidden widths 16 / 32 / 64 with 1-3 hidden layers on both latent layouts
    (variant B: 1/4, 1/8, 1/16, 1/32 of the output side; variant A: 1/4, 1/4,
    1/8, 1/8) -- the tiled kernel's instantiations."""
    lv = None if layout == "B" else [64, 64, 32, 32]
    wl = synth.small_decode_workload(256, dims, seed=90 + len(dims) + dims[1], level_sides=lv)
    mat = nb.Material.from_synth(wl.material)
    y = nb.decode(ctx, mat, grid=(256, 96))
    ctx.sync()
    ref = oracle.decode.decode_grid(wl.material, 256, 96)
    assert max_abs(y.cpu().numpy(), ref) <= TOL_FP32


def test_decode_config1_full_size_every_texel(nb, ctx):
    """The 4096^2 decode in the launch configuration the benchmark times: every one
    of its 16.8M texels x 9 channels within 1e-5 of the FP64 oracle (the oracle
    runs on row bands in one spawned worker per host core)."""
    import tc_parity as tp
    wl = synth.decode_workload(1)
    mat = nb.Material.from_synth(wl.material)
    y = nb.decode(ctx, mat, grid=(4096, 4096))
    ctx.sync()
    got = y.view(4096, 4096, 9).cpu().numpy()
    with tp.pool() as p:
        err = np.max(p.map(tp.band_fp32, [(1, r, n, got[r:r + n].reshape(-1, 9)) for r, n in tp.bands(4096, 64)]),
                     axis=0)
    print("FP32 4096^2 per-channel max abs error vs FP64 (every texel):", np.round(err, 8).tolist())
    assert np.all(err <= TOL_FP32), err


def test_zero_and_one_texel(nb, ctx):
    wl = synth.decode_workload(0)
    mat = nb.Material.from_synth(wl.material)
    empty = torch.empty((0, 2), dtype=torch.float32, device="cuda")
    y = nb.decode(ctx, mat, uv=empty)
    assert y.shape == (0, 9)
    uv = np.array([[0.3, 0.7]], dtype=np.float32)
    y = nb.decode(ctx, mat, uv=torch.from_numpy(uv).cuda())
    ctx.sync()
    assert max_abs(y.cpu().numpy(), oracle.decode.decode_uv(wl.material, uv)) <= TOL_FP32


def test_nan_weights_propagate(nb, ctx):
    wl = synth.decode_workload(0)
    wl.material.mlp.weights[2] = wl.material.mlp.weights[2].copy()
    wl.material.mlp.weights[2][3, 5] = np.nan
    mat = nb.Material.from_synth(wl.material)
    y = nb.decode(ctx, mat, grid=(64, 64))
    ctx.sync()
    assert torch.isnan(y[:, 3]).any() and torch.isfinite(y[:, 0]).all()


def test_invalid_arguments(nb, ctx):
    from paper_2506_06040_gb300 import _abi
    wl = synth.decode_workload(0)
    mat = nb.Material.from_synth(wl.material)
    with pytest.raises(nb.NbtcError) as e:
        nb.decode(ctx, mat, grid=(64, 64), out=torch.empty((100, 9), device="cuda")[1:])  # misaligned
    assert e.value.code == _abi.ERR_INVALID_ARG
    # pointer kinds: pageable host memory is refused before any launch; pinned
    # host uv is read over the host link; the packed image must be device memory
    uv = synth.random_uv(3, 1000)
    with pytest.raises(nb.NbtcError) as e:
        nb.decode(ctx, mat, uv=torch.from_numpy(uv))
    assert e.value.code == _abi.ERR_INVALID_ARG
    want = nb.decode(ctx, mat, uv=torch.from_numpy(uv).cuda())
    got = nb.decode(ctx, mat, uv=torch.from_numpy(uv).pin_memory())
    ctx.sync()
    assert torch.equal(got, want)
    wl64 = synth.small_decode_workload(256, [12, 64, 64, 9], seed=12)
    mat64 = nb.Material.from_synth(wl64.material)
    packed = nb.pack_mlp(ctx, mat64, nb.FP16)
    with pytest.raises(nb.NbtcError) as e:
        nb.decode(ctx, mat64, nb.FP16, packed.cpu(), grid=(256, 16))
    assert e.value.code == _abi.ERR_INVALID_ARG
    mat.level_meta[0] = (66, 64, 1, 0.0)  # not a multiple of 4
    with pytest.raises(nb.NbtcError) as e:
        nb.decode(ctx, mat, grid=(8, 8))
    assert e.value.code == _abi.ERR_INVALID_ARG
    ctx.sync()


@pytest.mark.parametrize("dims", [[12, 64, 64, 9], [12, 32, 9], [12, 64, 64, 64, 9]])
def test_row_bands_equal_the_whole_grid(nb, ctx, dims):
    """nbtc_decode_rows: any band of rows is bit-identical to those rows of the
    whole-grid decode (FP32 and, for width 64, FP16); FP32 decodes straight into
    pinned host memory and the FP16 banded host stream reassemble the texture."""
    from paper_2506_06040_gb300 import _abi
    wl = synth.small_decode_workload(1024, dims, seed=150 + len(dims))
    mat = nb.Material.from_synth(wl.material)
    gw, gh = 1024, 600
    full = nb.decode(ctx, mat, grid=(gw, gh))
    for r0, nr in ((0, 1), (7, 100), (100, 137), (599, 1), (512, 88)):
        band = nb.decode(ctx, mat, grid=(gw, gh), rows=(r0, nr))
        assert torch.equal(band, full[r0 * gw:(r0 + nr) * gw])
    # FP32 straight into pinned host memory: the whole grid, and a band of rows
    host = torch.full((gw * gh, 9), float("nan"), dtype=torch.float32).pin_memory()
    nb.decode_to_host(ctx, mat, host, (gw, gh))
    ctx.sync()
    assert torch.equal(host, full.cpu())
    host.fill_(float("nan"))
    nb.decode(ctx, mat, grid=(gw, gh), rows=(100, 137), out=host[100 * gw:237 * gw])
    ctx.sync()
    assert torch.equal(host[100 * gw:237 * gw], full[100 * gw:237 * gw].cpu())
    assert torch.isnan(host[:100 * gw]).all() and torch.isnan(host[237 * gw:]).all()
    if dims[1] == 64:
        packed = nb.pack_mlp(ctx, mat, nb.FP16)
        f16 = nb.decode(ctx, mat, nb.FP16, packed, grid=(gw, gh))
        for r0, nr in ((3, 50), (300, 300)):
            band = nb.decode(ctx, mat, nb.FP16, packed, grid=(gw, gh), rows=(r0, nr))
            assert torch.equal(band.view(torch.int16), f16[r0 * gw:(r0 + nr) * gw].view(torch.int16))
        # FP16 to the host: row bands on the device, each copied out while the next decodes
        h16 = torch.empty((gw * gh, 9), dtype=torch.float16).pin_memory()
        cs = torch.cuda.Stream()
        nb.decode_to_host(ctx, mat, h16, (gw, gh), nb.FP16, packed, bands=7, copy_stream=cs)
        cs.synchronize()
        assert torch.equal(h16.view(torch.int16), f16.cpu().view(torch.int16))
        # the tensor-core kernels do not write host memory
        with pytest.raises(nb.NbtcError) as e:
            nb.decode(ctx, mat, nb.FP16, packed, grid=(gw, gh), out=h16)
        assert e.value.code == _abi.ERR_UNSUPPORTED
    # pageable host memory is refused before any launch
    with pytest.raises(nb.NbtcError) as e:
        nb.decode(ctx, mat, grid=(gw, gh), out=torch.empty((gw * gh, 9), dtype=torch.float32))
    assert e.value.code == _abi.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        nb.decode_to_host(ctx, mat, torch.empty((gw * gh, 9), dtype=torch.float32), (gw, gh))
    ctx.sync()
    with pytest.raises(nb.NbtcError):
        nb.decode(ctx, mat, grid=(gw, gh), rows=(590, 20))
