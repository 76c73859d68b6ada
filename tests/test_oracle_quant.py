"""Pins of the oracle's FP16 / FP8 E4M3 rounding and of the quantisation
emulator, against numpy float16 and torch float8_e4m3fn (library routines)."""
import numpy as np
import torch

from oracle import emulate, mlp, quant


def test_fp16_value_all_codes():
    bits = np.arange(1 << 16, dtype=np.uint16)
    lib = bits.view(np.float16).astype(np.float64)
    ours = quant.fp16_value(bits)
    same = (lib == ours) | (np.isnan(lib) & np.isnan(ours))
    assert same.all()


def test_round_fp16_against_numpy():
    rng = np.random.default_rng(9)
    # all finite fp16 values round to themselves
    vals = np.arange(1 << 16, dtype=np.uint16).view(np.float16).astype(np.float64)
    vals = vals[np.isfinite(vals)]
    np.testing.assert_array_equal(quant.round_fp16(vals), vals)
    # midpoints between neighbours (ties to even) and random values over all binades
    pos = np.sort(vals[vals >= 0])
    mids = (pos[:-1] + pos[1:]) / 2
    x = np.concatenate([mids, -mids, rng.normal(size=200000) * 10.0 ** rng.uniform(-9, 5, 200000),
                        [65519.0, 65520.0, 70000.0, -65520.0, 2.0 ** -25, 3 * 2.0 ** -26]])
    with np.errstate(over="ignore"):
        lib = x.astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(quant.round_fp16(x), lib)


def test_e4m3_value_all_codes():
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8)
    lib = codes.view(torch.float8_e4m3fn).to(torch.float64).numpy()
    ours = quant.e4m3_value(np.arange(256))
    same = (lib == ours) | (np.isnan(lib) & np.isnan(ours))
    assert same.all()


def test_round_e4m3_against_torch():
    rng = np.random.default_rng(10)
    vals = quant.e4m3_value(np.arange(256))
    vals = np.sort(vals[np.isfinite(vals) & (vals >= 0)])
    mids = (vals[:-1] + vals[1:]) / 2
    x = np.concatenate([vals, -vals, mids, -mids, rng.uniform(-460, 460, 100000),
                        rng.normal(size=100000) * 10.0 ** rng.uniform(-4, 2, 100000)])
    x = x[np.abs(x) < 464]  # torch turns the overflow range into NaN; satfinite is checked below
    lib = torch.tensor(x, dtype=torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(quant.round_e4m3_satfinite(x.astype(np.float32).astype(np.float64)), lib)
    np.testing.assert_array_equal(quant.round_e4m3_satfinite(np.array([464.0, 500.0, 1e9, -1e9])),
                                  [448.0, 448.0, 448.0, -448.0])


def test_pow2_ceil():
    np.testing.assert_array_equal(quant.pow2_ceil(np.array([1.0, 0.75, 3.0, 2.0 ** -20 * 1.1, 448.0])),
                                  [1.0, 1.0, 4.0, 2.0 ** -19, 512.0])


def _dyadic_mlp(rng, dims, step):
    ws = [np.round(rng.normal(size=(dims[i + 1], dims[i])) / step) * step for i in range(len(dims) - 1)]
    bs = [np.round(rng.normal(size=dims[i + 1]) / step) * step for i in range(len(dims) - 1)]
    return ws, bs


def test_fp16_emulator_exact_on_representable_operands():
    """Weights, inputs and every hidden activation exact in FP16 => emulator == FP64 oracle
    (then only the output rounding remains)."""
    rng = np.random.default_rng(11)
    dims = [12, 8, 8, 9]
    ws, bs = _dyadic_mlp(rng, dims, 0.25)
    x = np.round(rng.random((300, 12)) * 4) / 4
    want = mlp.forward(x, ws, bs)  # small dyadic numbers: hidden values stay exact in FP16
    np.testing.assert_array_equal(emulate.forward_fp16(x, ws, bs, round_output=False), want)
    np.testing.assert_array_equal(emulate.forward_fp16(x, ws, bs), quant.round_fp16(want))


def test_fp16_emulator_error_bound_and_rounding():
    rng = np.random.default_rng(12)
    dims = [12, 64, 64, 9]
    ws = [rng.normal(size=(dims[i + 1], dims[i])) * np.sqrt(2 / dims[i]) for i in range(3)]
    bs = [rng.normal(size=dims[i + 1]) * 0.01 for i in range(3)]
    x = rng.random((2000, 12))
    emu = emulate.forward_fp16(x, ws, bs)
    ref = mlp.forward(x, ws, bs)
    assert np.all(quant.round_fp16(emu) == emu)         # outputs are FP16 values
    err = np.abs(emu - ref).max()
    assert 1e-5 < err < 1e-2                            # rounding happened, and it is small
    # first-order bound: every operand carries <= 2^-11 relative error per rounding
    u = 2.0 ** -11
    a = np.abs(x)
    for l, (w, b) in enumerate(zip(ws, bs)):
        a = a @ np.abs(w).T + np.abs(b)
    assert np.all(np.abs(emu - ref) <= (2 * len(ws) + 2) * u * a + u * np.abs(ref) + 1e-12)


def test_fp8_emulator_exact_on_representable_operands():
    """Operands whose scaled values are E4M3 numbers (<= 4 significant bits, in range)
    => FP8 emulator == FP64 oracle before the output rounding."""
    rng = np.random.default_rng(13)
    x = rng.integers(0, 9, size=(200, 12)) / 8.0                 # i/8: 4-bit significands
    w1 = np.zeros((8, 12))
    for j in range(8):                                          # one +-2^k entry per row
        w1[j, rng.integers(0, 12)] = rng.choice([-2.0, -1.0, -0.5, 0.5, 1.0, 2.0])
    w2 = rng.integers(-4, 5, size=(9, 8)) / 4.0
    ws, bs = [w1, w2], [np.zeros(8), np.zeros(9)]
    acts = mlp.hidden_activations(x, ws, bs)
    sw, sa = emulate.fp8_scales(ws, acts)
    assert all(float(quant.pow2_ceil(s)) == s for s in sw + sa)
    for a, s in zip(acts, sa):
        np.testing.assert_array_equal(quant.round_e4m3_satfinite(a / s), a / s)
    emu = emulate.forward_fp8(x, ws, bs, sw, sa, round_output=False)
    np.testing.assert_array_equal(emu, mlp.forward(x, ws, bs))
    np.testing.assert_array_equal(emulate.forward_fp8(x, ws, bs, sw, sa), quant.round_fp16(emu))


def test_fp8_emulator_rounds_operands():
    rng = np.random.default_rng(14)
    dims = [12, 64, 64, 9]
    ws = [rng.normal(size=(dims[i + 1], dims[i])) * np.sqrt(2 / dims[i]) for i in range(3)]
    bs = [rng.normal(size=dims[i + 1]) * 0.01 for i in range(3)]
    x = rng.random((2000, 12))
    sw, sa = emulate.fp8_scales(ws, mlp.hidden_activations(x, ws, bs))
    emu = emulate.forward_fp8(x, ws, bs, sw, sa)
    ref = mlp.forward(x, ws, bs)
    err = np.abs(emu - ref)
    assert 1e-3 < err.max() < 0.5 and err.mean() < 0.05


def test_fp16_emulator_rounds_bias_as_operand():
    """The FP16 form's bias is an FP16 operand: 1 + 2^-12 rounds to 1."""
    ws = [np.zeros((2, 3)), np.zeros((1, 2))]
    bs = [np.array([0.5, 1.0 + 2.0 ** -12]), np.array([1.0 + 2.0 ** -12])]
    x = np.ones((1, 3))
    np.testing.assert_array_equal(emulate.forward_fp16(x, ws, bs, round_output=False), [[1.0]])
    np.testing.assert_array_equal(mlp.forward(x, ws, bs), [[1.0 + 2.0 ** -12]])
