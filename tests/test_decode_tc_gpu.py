"""GPU parity of the tensor-core forms (tcgen05, FP16 / FP8 E4M3 operands, FP32
accumulation, FP16 output) against the oracle's quantisation emulator, and
their error against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _grid_uv(idx, gw, gh):
    """Texel-centre uv of grid indices, FP32 as the decode forms them."""
    return (oracle.sample.grid_coord(idx % gw, gw).astype(np.float64),
            oracle.sample.grid_coord(idx // gw, gh).astype(np.float64))


def ulp16(x):
    """Spacing of binary16 numbers at |x| (2^-24 below the normal range)."""
    ax = np.maximum(np.abs(np.asarray(x, dtype=np.float64)), 2.0 ** -14)
    return np.ldexp(1.0, np.floor(np.log2(ax)).astype(np.int64) - 10)


# Kernel vs emulator.  The two differ only where an FP32 intermediate of the kernel
# (tensor-core accumulation, bias add, FP32 features) lands on the other side of a
# rounding boundary of a hidden activation than the exact value does: that
# activation then differs by one unit of the narrow format.  To first order such
# flips move output c by at most  u * sum_l |W_L| ... |W_(l+1)| |h_l|,  bounded by
#   u * NHID * absnet(x),   absnet = the network run on |W|, |b|, |x|,
# with u = 2^-10 (FP16 unit) or 2^-3 (E4M3 unit).  The output rounding adds its own
# few FP16 ulps.  Statistically almost every output must still match to an ulp.
TOL_ULPS_FP16 = 4
FRAC_1ULP_FP16 = 0.99


def absnet(material, x):
    h = np.abs(np.asarray(x, dtype=np.float64))
    for w, b in zip(material.mlp.weights, material.mlp.biases):
        h = h @ np.abs(w.astype(np.float64)).T + np.abs(b.astype(np.float64))
    return h


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


def _fp16_case(nb, ctx, wl, grid=None, uv=None):
    mat = nb.Material.from_synth(wl.material)
    packed = nb.pack_mlp(ctx, mat, nb.FP16)
    if uv is not None:
        y = nb.decode(ctx, mat, nb.FP16, packed, uv=torch.from_numpy(uv).cuda())
    else:
        y = nb.decode(ctx, mat, nb.FP16, packed, grid=grid)
    ctx.sync()
    return y.float().cpu().numpy().astype(np.float64)


def _check(got, emu, material, x, unit, frac_1ulp):
    err = np.abs(got - emu)
    assert np.all(np.isfinite(got))
    nhid = len(material.mlp.weights) - 1
    bound = TOL_ULPS_FP16 * ulp16(emu) + unit * nhid * absnet(material, x)
    assert np.all(err <= bound), float((err / bound).max())
    frac = float(np.mean(err <= ulp16(emu) + 2.0 ** -24))
    assert frac >= frac_1ulp, frac
    return float(err.max()), frac


def _check_fp16(got, emu, material, x):
    return _check(got, emu, material, x, 2.0 ** -10, FRAC_1ULP_FP16)


def _grid_x(material, gw, gh, idx=None):
    if idx is None:
        idx = np.arange(gw * gh)
    return oracle.decode.features_at(material, oracle.sample.grid_coord(idx % gw, gw).astype(np.float64),
                                     oracle.sample.grid_coord(idx // gw, gh).astype(np.float64))


@pytest.mark.parametrize("dims", [[12, 64, 9], [12, 64, 64, 9], [12, 64, 64, 64, 9]])
def test_fp16_grid_footprint(nb, ctx, dims):
    wl = synth.small_decode_workload(512, dims, seed=300 + len(dims))
    got = _fp16_case(nb, ctx, wl, grid=(512, 96))
    emu = oracle.decode.decode_grid(wl.material, 512, 96, precision="fp16")
    _check_fp16(got, emu, wl.material, _grid_x(wl.material, 512, 96))


@pytest.mark.parametrize("gw,gh,levels", [(1024, 768, None), (384, 1024, [384, 192, 96, 48])])
def test_fp16_grid_long_strips(nb, ctx, gw, gh, levels):
    """Every texel of grids whose per-warpgroup tile ranges run many rows down a
    column strip and cross strip boundaries: the feature stage's column cache
    (blocks decoded again only when a level's vertical tap pair changes, next
    row's blocks prefetched) against the emulator everywhere.  The second grid's
    levels (1, 1/2, 1/4, 1/8 of its width) need 248 latent columns per 128-texel
    tile, more than one per thread.  Both keep the texel coordinates exact in
    FP32 along x (dyadic level/output ratios); off-dyadic grids differ from the
    FP64 emulator by FP32 coordinate rounding, which flips FP16 roundings of
    features more often than the 1-ulp criterion assumes."""
    wl = synth.small_decode_workload(1024, [12, 64, 64, 64, 9], seed=330 + gh, level_sides=levels)
    got = _fp16_case(nb, ctx, wl, grid=(gw, gh))
    emu = oracle.decode.decode_grid(wl.material, gw, gh, precision="fp16")
    _check_fp16(got, emu, wl.material, _grid_x(wl.material, gw, gh))


@pytest.mark.parametrize("gw,gh", [(200, 72), (130, 3), (7, 5), (128, 1), (256, 2), (65536, 1), (1, 4096)])
def test_fp16_ragged(nb, ctx, gw, gh):
    wl = synth.small_decode_workload(256, [12, 64, 64, 9], seed=310)
    got = _fp16_case(nb, ctx, wl, grid=(gw, gh))
    emu = oracle.decode.decode_grid(wl.material, gw, gh, precision="fp16")
    _check_fp16(got, emu, wl.material, _grid_x(wl.material, gw, gh))


@pytest.mark.parametrize("address", ["clamp", "wrap"])
def test_fp16_uv_list(nb, ctx, address):
    wl = synth.small_decode_workload(256, [12, 64, 64, 64, 9], seed=320, address=address)
    uv = synth.random_uv(321, 5000 * 2 + 77, lo=-0.25, hi=1.25)
    got = _fp16_case(nb, ctx, wl, uv=uv)
    emu = oracle.decode.decode_uv(wl.material, uv, precision="fp16")
    x = oracle.decode.features_at(wl.material, uv[:, 0].astype(np.float64), uv[:, 1].astype(np.float64))
    _check_fp16(got, emu, wl.material, x)


def test_fp16_full_size_sampled_and_error_budget(nb, ctx):
    """The 4096^2, 12-64-64-64-9 FP16 decode in the benchmark's launch configuration:
    65,536 random texels and the border rows against the emulator; per-channel max abs
    error against the FP64 oracle reported and bounded."""
    wl = synth.decode_workload(2)
    mat = nb.Material.from_synth(wl.material)
    packed = nb.pack_mlp(ctx, mat, nb.FP16)
    y = nb.decode(ctx, mat, nb.FP16, packed, grid=(4096, 4096))
    ctx.sync()
    rng = np.random.default_rng(6)
    idx = np.concatenate([rng.integers(0, 4096 * 4096, 65536), np.arange(4096), 4096 * 4095 + np.arange(4096)])
    got = y[torch.from_numpy(idx).cuda()].float().cpu().numpy().astype(np.float64)
    tex = [oracle.decode.level_rgb(lv) for lv in wl.material.levels]
    emu = oracle.decode.decode_grid(wl.material, 4096, 4096, idx, precision="fp16", tex=tex)
    x = oracle.decode.features_at(wl.material, *_grid_uv(idx, 4096, 4096), tex)
    e_emu, frac = _check_fp16(got, emu, wl.material, x)
    ref = oracle.decode.decode_grid(wl.material, 4096, 4096, idx, tex=tex)
    per_channel = np.abs(got - ref).max(axis=0)
    emu_channel = np.abs(emu - ref).max(axis=0)
    print(f"FP16 kernel vs emulator: max {e_emu:.3g}, {frac:.5f} within 1 ulp")
    print("FP16 per-channel max abs error vs FP64, kernel:  ", np.round(per_channel, 6).tolist())
    print("FP16 per-channel max abs error vs FP64, emulator:", np.round(emu_channel, 6).tolist())
    # The FP16 operands themselves cost ~3.3e-3 on this He-initialised network (the
    # emulator's floor, above the 2e-3 target); the kernel must add nothing beyond it.
    assert np.all(per_channel <= emu_channel + 2.0 ** -11)
    assert torch.isfinite(y).all()


def _fp8_setup(nb, ctx, wl, gw, gh):
    mat = nb.Material.from_synth(wl.material)
    absmax = nb.fp8_calibrate(ctx, mat, gw, gh, 16)
    packed = nb.pack_mlp(ctx, mat, nb.FP8_E4M3, act_absmax=absmax)
    ctx.sync()
    sw, sa = oracle.decode.fp8_calibration(wl.material, gw, gh, 16)
    sa_gpu = [float(oracle.quant.pow2_ceil(a / 448.0)) for a in absmax.cpu().numpy().astype(np.float64)]
    assert sa_gpu == sa, (sa_gpu, sa)
    return mat, packed, (sw, sa)


@pytest.mark.parametrize("dims,layout", [([12, 16, 9], "B"), ([12, 32, 9], "A"), ([12, 32, 32, 9], "B"),
                                         ([12, 16, 9], "A"), ([12, 64, 9], "A")])
def test_fp16_hidden_width_sweep(nb, ctx, dims, layout):
    """Table 1's one-hidden-layer MLPs of width D = 16 / 32 / 64 (zero-padded to
    the 64-wide image) on the paper's latent layouts: variant B (1/4, 1/8, 1/16,
    1/32 of the output side) and variant A (1/4, 1/4, 1/8, 1/8)."""
    side = 512
    lv = [side // 4, side // 8, side // 16, side // 32] if layout == "B" else [side // 4, side // 4, side // 8, side // 8]
    wl = synth.small_decode_workload(side, dims, seed=340 + dims[1] + len(dims), level_sides=lv)
    got = _fp16_case(nb, ctx, wl, grid=(side, 96))
    emu = oracle.decode.decode_grid(wl.material, side, 96, precision="fp16")
    _check_fp16(got, emu, wl.material, _grid_x(wl.material, side, 96))


@pytest.mark.parametrize("dims", [[12, 64, 9], [12, 64, 64, 64, 9], [12, 32, 9]])
def test_fp8_grid(nb, ctx, dims):
    wl = synth.small_decode_workload(512, dims, seed=330 + len(dims))
    mat, packed, scales = _fp8_setup(nb, ctx, wl, 512, 128)
    y = nb.decode(ctx, mat, nb.FP8_E4M3, packed, grid=(512, 128))
    ctx.sync()
    got = y.float().cpu().numpy().astype(np.float64)
    emu = oracle.decode.decode_grid(wl.material, 512, 128, precision="fp8", fp8=scales)
    e, frac = _check(got, emu, wl.material, _grid_x(wl.material, 512, 128), 2.0 ** -3, 0.99)
    ref = oracle.decode.decode_grid(wl.material, 512, 128)
    print(f"FP8 {dims}: kernel vs emulator max {e:.3g} ({frac:.5f} within 1 ulp16); "
          f"per-channel max abs vs FP64 kernel {np.round(np.abs(got - ref).max(0), 4).tolist()} "
          f"emulator {np.round(np.abs(emu - ref).max(0), 4).tolist()}")


def test_fp8_full_size_sampled(nb, ctx):
    """The 4096^2, 12-64-64-64-9 FP8 decode as the benchmark runs it: 65,536
    random texels and the border rows against the FP8 emulator."""
    wl = synth.decode_workload(2)
    mat, packed, scales = _fp8_setup(nb, ctx, wl, 4096, 4096)
    y = nb.decode(ctx, mat, nb.FP8_E4M3, packed, grid=(4096, 4096))
    ctx.sync()
    rng = np.random.default_rng(9)
    idx = np.concatenate([rng.integers(0, 4096 * 4096, 65536), np.arange(4096), 4096 * 4095 + np.arange(4096)])
    got = y[torch.from_numpy(idx).cuda()].float().cpu().numpy().astype(np.float64)
    tex = [oracle.decode.level_rgb(lv) for lv in wl.material.levels]
    emu = oracle.decode.decode_grid(wl.material, 4096, 4096, idx, precision="fp8", fp8=scales, tex=tex)
    x = oracle.decode.features_at(wl.material, *_grid_uv(idx, 4096, 4096), tex)
    _check(got, emu, wl.material, x, 2.0 ** -3, 0.99)


def test_fp8_calibration_matches_oracle(nb, ctx):
    wl = synth.decode_workload(2)
    _fp8_setup(nb, ctx, wl, 4096, 4096)


def test_packed_sizes(nb, ctx):
    from paper_2506_06040_gb300 import api
    wl = synth.decode_workload(2)
    mat = nb.Material.from_synth(wl.material)
    assert api.packed_mlp_bytes(mat, nb.FP16) % 16 == 0
    assert api.packed_mlp_bytes(mat, nb.FP8_E4M3) < api.packed_mlp_bytes(mat, nb.FP16)
    # hidden width 32 packs zero-padded into the same 64-wide image
    wl0 = synth.decode_workload(0)
    m32 = nb.Material.from_synth(synth.small_decode_workload(256, [12, 32, 32, 9], seed=5).material)
    assert api.packed_mlp_bytes(m32, nb.FP16) == api.packed_mlp_bytes(
        nb.Material.from_synth(synth.small_decode_workload(256, [12, 64, 64, 9], seed=5).material), nb.FP16)
    assert api.packed_mlp_bytes(nb.Material.from_synth(wl0.material), nb.FP16) > 0
    # other widths have no tensor-core kernel
    with pytest.raises(nb.NbtcError):
        api.packed_mlp_bytes(nb.Material.from_synth(synth.small_decode_workload(256, [12, 48, 9], seed=5).material),
                             nb.FP16)


@pytest.mark.parametrize("batched", [False, True])
def test_forced_timeout_reports_status_and_context_recovers(nb, ctx, batched):
    """Every bounded wait of the decode loop gives up at once (test budget -1):
    the launch completes, records NBTC_ERR_TIMEOUT in the context's status word
    and the next sync reports it (once); with the budget restored the same
    context decodes correctly again.  Single-material launches read the budget
    per call; a batch plan bakes it into its graph when it is created."""
    from paper_2506_06040_gb300 import _abi
    if batched:
        mats = [nb.Material.from_synth(synth.small_decode_workload(256, [12, 64, 64, 9], seed=45 + i).material)
                for i in range(3)]
        outs = [(torch.empty((256 * 256, 9), dtype=torch.float16, device="cuda"), 256, 256) for _ in mats]
        make = lambda: nb.Batch(ctx, mats, outs, autotune=False)
        result = lambda: torch.cat([o[0] for o in outs])
    else:
        wl = synth.small_decode_workload(512, [12, 64, 64, 64, 9], seed=44)
        mat = nb.Material.from_synth(wl.material)
        packed = nb.pack_mlp(ctx, mat, nb.FP16)
        out = torch.empty((512 * 64, 9), dtype=torch.float16, device="cuda")

        class _Single:
            def decode(self):
                nb.decode(ctx, mat, nb.FP16, packed, grid=(512, 64), out=out)
        make = _Single
        result = lambda: out
    make().decode()
    ctx.sync()
    ref = result().clone()
    ctx.set_wait_budget(-1)
    try:
        make().decode()
        assert ctx.status() == _abi.ERR_TIMEOUT
        assert ctx.status() == _abi.OK   # reported once, then cleared
    finally:
        ctx.set_wait_budget(0)
    result().zero_()
    make().decode()
    ctx.sync()
    assert torch.equal(result().view(torch.int16), ref.view(torch.int16))
