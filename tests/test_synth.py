"""The seeded generators are deterministic and produce the workloads' shapes."""
import numpy as np

import synth


def test_rng_deterministic_and_streams_independent():
    a = synth.Rng(42, 1).u64(10)
    b = synth.Rng(42, 1).u64(10)
    c = synth.Rng(42, 2).u64(10)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    r = synth.Rng(42, 1)
    r.u64(4)
    assert np.array_equal(r.u64(6), a[4:])


def test_uniform_and_normal_moments():
    r = synth.Rng(1, 3)
    u = r.uniform(200000)
    assert 0 <= u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.005
    z = synth.Rng(1, 4).normal(200000, 2.0)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 2.0) < 0.02


def test_decode_workload_shapes():
    w = synth.decode_workload(0)
    assert [lv.width for lv in w.material.levels] == [64, 32, 16, 8]
    assert [lv.shift for lv in w.material.levels] == [0.0, 0.5, 0.0, 0.5]
    assert w.material.mlp.dims == [12, 32, 32, 9]
    for lv in w.material.levels:
        assert synth.has_both_modes(lv.blocks[0])
    w2 = synth.decode_workload(2)
    assert w2.material.mlp.dims == [12, 64, 64, 64, 9]
    assert [lv.width for lv in w2.material.levels] == [1024, 512, 256, 128]


def test_batch_workload_small():
    bw = synth.batch_workload(num_materials=5, frame_w=128, frame_h=64)
    assert all(256 <= s <= 4096 and s % 128 == 0 for s in bw.sizes)
    assert bw.mat_id.min() >= 0 and bw.mat_id.max() < 5
    assert bw.uv.shape == (64, 128, 2) and bw.lod_bias.shape == (64, 128)
    lv = bw.materials[0].levels[3]
    assert lv.num_mips == synth.full_mips(lv.width)
