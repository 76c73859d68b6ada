"""Pins of the QAT BC1 oracle (paper Sec. 3.2, Eqs. 1-3) against things it does
not compute itself: the nearest-level definition of quant evaluated in FP64 on
sigmoid values, closed-form special cases, finite differences of the
straight-through surrogate, and the BC1 decoder (pinned by its own golden
blocks) applied to the encoder's output."""
import numpy as np
import pytest

import oracle
from oracle import bc1, qat, train


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("bits", [2, 5, 6])
def test_level_is_nearest_level_of_sigmoid(bits):
    n = (1 << bits) - 1
    p = _rng(bits).normal(0, 3, 200000).astype(np.float32)
    s = 1.0 / (1.0 + np.exp(-p.astype(np.float64)))
    want = np.rint(s * n).astype(np.int64)
    got = qat.level(p, bits)
    # away from the decision midpoints the two must agree exactly
    far = np.abs(s * n - np.floor(s * n) - 0.5) > 1e-5
    assert far.mean() > 0.99
    assert np.array_equal(got[far], want[far])
    # near them they differ by at most one level
    assert np.all(np.abs(got - want) <= 1)
    assert got.min() >= 0 and got.max() <= n
    # monotone in p
    order = np.argsort(p, kind="stable")
    assert np.all(np.diff(got[order]) >= 0)


@pytest.mark.parametrize("bits", [2, 5, 6])
def test_level_of_exact_levels(bits):
    n = (1 << bits) - 1
    k = np.arange(1, n)
    p = np.log(k / (n - k))                       # sigmoid(p) = k / n exactly
    assert np.array_equal(qat.level(p, bits), k)
    assert qat.level(np.float32(-1e4), bits) == 0 and qat.level(np.float32(1e4), bits) == n
    assert np.allclose(qat.quant_value(p, bits), k / n, rtol=0, atol=0)


def test_decode_special_cases():
    r = _rng(1)
    e0, e1 = r.normal(0, 2, (2, 3, 3)), r.normal(0, 2, (2, 3, 3))
    E0 = qat.endpoint_values(e0)
    E1 = qat.endpoint_values(e1)
    big = np.full((8, 12), 50.0)
    # alpha -> -inf: a = 0, the texel is e0's colour; +inf: e1's
    assert np.allclose(qat.decode(e0, e1, -big), np.repeat(np.repeat(E0, 4, 0), 4, 1), atol=0)
    assert np.allclose(qat.decode(e0, e1, big), np.repeat(np.repeat(E1, 4, 0), 4, 1), atol=0)
    # sigmoid(alpha) = 1/3 exactly -> a = 1/3
    third = np.full((8, 12), np.log(0.5))
    want = np.repeat(np.repeat(2 / 3 * E0 + 1 / 3 * E1, 4, 0), 4, 1)
    assert np.allclose(qat.decode(e0, e1, third), want, rtol=0, atol=1e-15)
    # the endpoint levels are the [5, 6, 5] patterns
    assert set(np.unique(np.rint(E0[..., 0] * 31))) <= set(range(32))
    assert set(np.unique(np.rint(E0[..., 1] * 63))) <= set(range(64))


def test_backward_matches_finite_differences_of_the_straight_through_surrogate():
    """Straight-through: the quantised factors are held fixed and only the
    sigmoid of the differentiated parameter varies."""
    r = _rng(2)
    h, w = 8, 8
    e0, e1, alpha = r.normal(0, 1.5, (2, 2, 3)), r.normal(0, 1.5, (2, 2, 3)), r.normal(0, 1.5, (h, w))
    dT = r.normal(0, 1, (h, w, 3))
    g0, g1, ga = qat.backward(e0, e1, alpha, dT)
    E0 = np.repeat(np.repeat(qat.endpoint_values(e0), 4, 0), 4, 1)
    E1 = np.repeat(np.repeat(qat.endpoint_values(e1), 4, 0), 4, 1)
    a = qat.quant_value(alpha, 2)[..., None]
    sig = lambda x: 1.0 / (1.0 + np.exp(-x))
    eps = 1e-6
    for (y, x) in [(0, 0), (3, 5), (7, 7), (4, 1)]:
        def f(al):
            s = sig(al)
            return np.sum(dT[y, x] * ((1 - s) * E0[y, x] + s * E1[y, x]))
        fd = (f(alpha[y, x] + eps) - f(alpha[y, x] - eps)) / (2 * eps)
        assert abs(fd - ga[y, x]) < 1e-7 * max(1.0, abs(fd))
    for (by, bx, c) in [(0, 0, 0), (1, 1, 2), (0, 1, 1)]:
        sl = (slice(4 * by, 4 * by + 4), slice(4 * bx, 4 * bx + 4))

        def f0(v):
            return np.sum(dT[sl][..., c] * (1 - a[sl][..., 0]) * sig(v))

        def f1(v):
            return np.sum(dT[sl][..., c] * a[sl][..., 0] * sig(v))
        fd0 = (f0(e0[by, bx, c] + eps) - f0(e0[by, bx, c] - eps)) / (2 * eps)
        fd1 = (f1(e1[by, bx, c] + eps) - f1(e1[by, bx, c] - eps)) / (2 * eps)
        assert abs(fd0 - g0[by, bx, c]) < 1e-7 * max(1.0, abs(fd0))
        assert abs(fd1 - g1[by, bx, c]) < 1e-7 * max(1.0, abs(fd1))


def _expansion_error():
    """Largest |bit-replicated 8-bit endpoint - 255 k / n| over the 5- and 6-bit codes."""
    e = 0.0
    for bits in (5, 6):
        n = (1 << bits) - 1
        k = np.arange(n + 1)
        rep = (k << (8 - bits)) | (k >> (2 * bits - 8))
        e = max(e, float(np.max(np.abs(rep - 255.0 * k / n))))
    return e


def test_encode_decodes_to_the_qat_texture_within_bc1_rounding():
    r = _rng(3)
    h, w = 64, 48
    e0, e1, alpha = r.normal(0, 2, (h // 4, w // 4, 3)), r.normal(0, 2, (h // 4, w // 4, 3)), r.normal(0, 2, (h, w))
    blocks = qat.encode(e0, e1, alpha)
    rgb = bc1.decode_level(blocks, w, h).astype(np.float64)
    T = qat.decode(e0, e1, alpha) * 255.0
    # endpoints: bit replication vs k/n; thirds: integer rounding of (2a+b)/3 (at most 1/3)
    bound = _expansion_error() + 1.0 / 3.0 + 1e-9
    assert np.max(np.abs(rgb - T)) <= bound
    # every block is four-colour (c0 > c1) or has equal endpoints with all indices 0
    c0, c1, iw = bc1.split_block(blocks)
    assert np.all((c0 > c1) | ((c0 == c1) & (iw == 0)))
    assert np.any(c0 > c1)


def test_encode_ordering_rule_on_hand_built_blocks():
    """One block, endpoints chosen so that codes(e0) < codes(e1): the encoder
    swaps them and remaps every level q -> 3 - q; equal codes give index 0."""
    k = lambda v, n: np.log(v / (n - v))          # raw parameter with sigmoid = v / n
    lo = np.array([[[k(3, 31), k(10, 63), k(4, 31)]]])
    hi = np.array([[[k(20, 31), k(40, 63), k(25, 31)]]])
    q = np.array([0, 1, 2, 3] * 4).reshape(4, 4)
    alpha = np.where(q == 0, -20.0, np.where(q == 3, 20.0, np.where(q == 1, np.log(0.5), np.log(2.0))))
    b = qat.encode(lo, hi, alpha)
    c0, c1, iw = bc1.split_block(b)
    assert c0[0] == (20 << 11 | 40 << 5 | 25) and c1[0] == (3 << 11 | 10 << 5 | 4)
    # texel level q (a = q / 3 toward hi) must decode from (c0 = hi, c1 = lo) as weight on c0 = q / 3
    want_index = {0: 1, 1: 3, 2: 2, 3: 0}      # q -> palette index after the swap
    got = bc1.texel_index(iw[0], np.arange(16) % 4, np.arange(16) // 4)
    assert [int(g) for g in got] == [want_index[int(v)] for v in q.reshape(-1)]
    # not swapped: hi as e0
    b2 = qat.encode(hi, lo, alpha)
    c0b, c1b, iwb = bc1.split_block(b2)
    assert c0b[0] == c0[0] and c1b[0] == c1[0]
    got2 = bc1.texel_index(iwb[0], np.arange(16) % 4, np.arange(16) // 4)
    assert [int(g) for g in got2] == [{0: 0, 1: 2, 2: 3, 3: 1}[int(v)] for v in q.reshape(-1)]
    # equal endpoints: every index 0, the block decodes to the endpoint everywhere (no black)
    b3 = qat.encode(hi, hi, alpha)
    c0c, c1c, iwc = bc1.split_block(b3)
    assert c0c[0] == c1c[0] and iwc[0] == 0
    rgb = bc1.decode_level(b3, 4, 4)
    assert np.all(rgb == bc1.expand565(c0c[0]))


def test_train_step_composes_pinned_parts():
    """The QAT step's dL/dT is the continuous step's gradient at the decoded
    textures (pinned by finite differences in test_oracle_train), and its raw
    gradients are the pinned straight-through backward of that dL/dT."""
    r = _rng(4)
    sides = [16, 8, 8, 4]
    shifts = [0.0, 0.5, 0.0, 0.5]
    e0 = [r.normal(0, 1, (s // 4, s // 4, 3)) for s in sides]
    e1 = [r.normal(0, 1, (s // 4, s // 4, 3)) for s in sides]
    al = [r.normal(0, 1, (s, s)) for s in sides]
    W = [r.normal(0, 0.4, (64, 12)), r.normal(0, 0.2, (64, 64)), r.normal(0, 0.2, (9, 64))]
    B = [r.normal(0, 0.01, 64), r.normal(0, 0.01, 64), r.normal(0, 0.01, 9)]
    target = r.normal(0, 1, (32, 32, 9))
    uv = r.uniform(0, 1, (300, 2))
    st = qat.init_state(e0, e1, al, W, B)
    new = qat.train_step(st, shifts, target, uv)
    T = [qat.decode(a, b, c) for a, b, c in zip(e0, e1, al)]
    y, cache = train.forward(T, shifts, W, B, uv)
    loss, dy = train.loss_and_dy(y, train.target_sample(target, uv))
    dW, db, dT = train.backward(dy, cache, T, shifts, W)
    assert new["loss"] == loss
    for k in range(4):
        g = qat.backward(e0[k], e1[k], al[k], dT[k])
        assert np.array_equal(new["grad_e0"][k], g[0]) and np.array_equal(new["grad_alpha"][k], g[2])
    # lr = 0 leaves every parameter as it was
    same = qat.train_step(st, shifts, target, uv, lr_mlp=0.0, lr_latent=0.0)
    for k in range(4):
        assert np.array_equal(same["alpha"][k], al[k]) and np.array_equal(same["e1"][k], e1[k])
    assert oracle.qat is qat
