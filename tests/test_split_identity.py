"""The tensor-core kernels split a ReLU'd FP32 activation v into FP16 hi + lo
without forming relu(v) in FP32: hi = RN16(relu v) (the converting ReLU),
r = RN16(v - hi) with v - hi formed exactly (a mixed-precision FMA), and
lo = max(r, -hi).  These tests check, on the host in IEEE arithmetic, that this
gives the definition's lo = RN16(relu(v) - hi) for every kind of input:
negative values (where r is negative and -hi is -0), values that round to
zero, FP16 subnormals, exact halfway cases and the FP16 range."""
import numpy as np


def _split_definition(v):
    hi = np.maximum(v, np.float32(0)).astype(np.float16)
    lo = (np.maximum(v, np.float32(0)) - hi.astype(np.float32)).astype(np.float16)
    return hi, lo


def _split_kernel(v):
    hi = np.maximum(v, np.float32(0)).astype(np.float16)             # cvt.rn.relu.f16x2.f32
    r = (v - hi.astype(np.float32)).astype(np.float16)               # fma(hi, -1, v), then cvt.rn.f16x2.f32
    lo = np.maximum(r, -hi)                                          # max.f16x2(r, -hi)
    return hi, lo


def _check(v):
    v = np.asarray(v, dtype=np.float32)
    h0, l0 = _split_definition(v)
    h1, l1 = _split_kernel(v)
    assert np.array_equal(h0.view(np.uint16), h1.view(np.uint16))
    # values equal; a zero lo may carry either sign
    assert np.array_equal(l0.astype(np.float32), l1.astype(np.float32))
    # the residual v - hi is exact in FP32 wherever v >= 0
    pos = v >= 0
    d = v[pos].astype(np.float64) - h0[pos].astype(np.float64)
    assert np.array_equal(d, (v[pos] - h0[pos].astype(np.float32)).astype(np.float64))


def test_random_activations():
    rng = np.random.default_rng(7)
    _check(rng.normal(0, 1, 1 << 20).astype(np.float32))
    _check((rng.normal(0, 1, 1 << 18) * 10.0 ** rng.uniform(-9, 4, 1 << 18)).astype(np.float32))


def test_edge_values():
    f16 = np.finfo(np.float16)
    tiny = float(np.float16(2.0 ** -24))  # smallest FP16 subnormal
    vals = [0.0, -0.0, 1.0, -1.0, tiny, tiny / 2, tiny * 0.75, -tiny, tiny * 1.5, 2.0 ** -14, 2.0 ** -15,
            float(f16.max), -float(f16.max), 1.0 + 2.0 ** -11, 1.0 + 2.0 ** -12, 1.0 + 3 * 2.0 ** -12,
            2048.0 + 1.0, 2048.0 + 0.5, -(2.0 ** -30), 2.0 ** -30]
    _check(vals)


def test_every_fp16_neighbourhood():
    """For every non-negative FP16 value h below the FP16 maximum: inputs at h,
    just above and below it, and at the midpoint to its upper neighbour (ties
    to even), and their negatives."""
    h = np.arange(0, 0x7BFF, dtype=np.uint16).view(np.float16).astype(np.float32)  # below the FP16 maximum
    nxt = np.nextafter(h.astype(np.float16), np.float16(np.inf)).astype(np.float32)
    mid = (h.astype(np.float64) + nxt.astype(np.float64)) / 2
    up = np.nextafter(h, np.float32(np.inf))
    down = np.nextafter(h, np.float32(-np.inf))
    _check(np.concatenate([h, up, down, mid.astype(np.float32), -h, -up]))
