"""GPU parity of the FP32-accurate tensor-core form (NBTC_FP32_TC: the split
FP16 operands of NBTC_FP16_SPLIT, FP32 accumulation in TMEM, the accumulator
written as FP32): held to the FP32 form's bound, max abs error <= 1e-5 against
the FP64 oracle, on every texel -- including all 16.8M texels of the 4096^2
decodes of both networks."""
import numpy as np
import pytest
import torch

import oracle
import synth
import tc_parity as tp
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


def _decode(nb, ctx, wl, grid=None, uv=None):
    mat = nb.Material.from_synth(wl.material)
    packed = nb.pack_mlp(ctx, mat, nb.FP32_TC)
    if uv is not None:
        y = nb.decode(ctx, mat, nb.FP32_TC, packed, uv=torch.from_numpy(uv).cuda())
    else:
        y = nb.decode(ctx, mat, nb.FP32_TC, packed, grid=grid)
    ctx.sync()
    assert y.dtype == torch.float32
    return y.cpu().numpy()


@pytest.mark.parametrize("dims", [[12, 64, 9], [12, 64, 64, 9], [12, 64, 64, 64, 9], [12, 32, 32, 9], [12, 16, 9]])
def test_fp32tc_grid_every_texel(nb, ctx, dims):
    wl = synth.small_decode_workload(512, dims, seed=600 + len(dims) + dims[1])
    got = _decode(nb, ctx, wl, grid=(512, 96))
    assert max_abs(got, oracle.decode.decode_grid(wl.material, 512, 96)) <= TOL_FP32


@pytest.mark.parametrize("gw,gh", [(200, 72), (130, 3), (7, 5), (128, 1), (65536, 1), (1, 4096), (1024, 300)])
def test_fp32tc_ragged_and_extreme(nb, ctx, gw, gh):
    wl = synth.small_decode_workload(256, [12, 64, 64, 9], seed=610)
    got = _decode(nb, ctx, wl, grid=(gw, gh))
    assert max_abs(got, oracle.decode.decode_grid(wl.material, gw, gh)) <= TOL_FP32


@pytest.mark.parametrize("address", ["clamp", "wrap"])
def test_fp32tc_uv_list(nb, ctx, address):
    wl = synth.small_decode_workload(256, [12, 64, 64, 64, 9], seed=620, address=address)
    uv = synth.random_uv(621, 9000 + 77, lo=-0.25, hi=1.25)
    got = _decode(nb, ctx, wl, uv=uv)
    assert max_abs(got, oracle.decode.decode_uv(wl.material, uv)) <= TOL_FP32


def test_fp32tc_refuses_host_output(nb, ctx):
    from paper_2506_06040_gb300 import _abi
    wl = synth.small_decode_workload(256, [12, 64, 64, 9], seed=630)
    mat = nb.Material.from_synth(wl.material)
    packed = nb.pack_mlp(ctx, mat, nb.FP32_TC)
    host = torch.empty((256 * 16, 9), dtype=torch.float32).pin_memory()
    with pytest.raises(nb.NbtcError) as e:
        nb.decode(ctx, mat, nb.FP32_TC, packed, grid=(256, 16), out=host)
    assert e.value.code == _abi.ERR_UNSUPPORTED
    ctx.sync()


@pytest.mark.parametrize("k", [1, 2])
def test_fp32tc_full_size_every_texel(nb, ctx, k):
    """The 4096^2 decodes of 12-64-64-9 (the FP32 headline workload) and
    12-64-64-64-9: every texel x 9 channels within 1e-5 of the FP64 oracle."""
    wl = synth.decode_workload(k)
    mat = nb.Material.from_synth(wl.material)
    packed = nb.pack_mlp(ctx, mat, nb.FP32_TC)
    y = nb.decode(ctx, mat, nb.FP32_TC, packed, grid=(4096, 4096))
    ctx.sync()
    got = y.view(4096, 4096, 9).cpu().numpy()
    with tp.pool() as p:
        err = np.max(p.map(tp.band_fp32, [(k, r, n, got[r:r + n].reshape(-1, 9)) for r, n in tp.bands(4096, 64)]),
                     axis=0)
    print(f"FP32-TC 4096^2 workload {k} per-channel max abs error vs FP64 (every texel):", np.round(err, 8).tolist())
    assert np.all(err <= TOL_FP32), err
