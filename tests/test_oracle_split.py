"""Pins of the split-operand emulator (hi + lo operand pairs, three products
per layer) and of its admissible-output intervals, against numpy float16,
torch float8_e4m3fn (library routines), the FP64 MLP, explicit nested sums at
tiny widths and a plain FP32 simulation of a kernel."""
import numpy as np
import torch

from oracle import emulate, mlp, quant


def _net(rng, dims):
    ws = [rng.normal(size=(dims[i + 1], dims[i])) * np.sqrt(2 / dims[i]) for i in range(len(dims) - 1)]
    bs = [rng.normal(size=dims[i + 1]) * 0.01 for i in range(len(dims) - 1)]
    return ws, bs


def test_split_fp16_against_numpy_and_residual_bound():
    rng = np.random.default_rng(20)
    v = rng.normal(size=300000) * 10.0 ** rng.uniform(-6, 4, 300000)
    hi, lo = emulate.split_fp16(v)
    np.testing.assert_array_equal(hi, v.astype(np.float16).astype(np.float64))
    np.testing.assert_array_equal(lo, (v - hi).astype(np.float16).astype(np.float64))
    # hi + lo carries ~22 significant bits: |v - hi - lo| <= 2^-22 |v| + 2^-25
    assert np.all(np.abs(v - hi - lo) <= 2.0 ** -22 * np.abs(v) + 2.0 ** -25)
    # and a single rounding does not: the pair is ~1000x closer on average
    assert np.mean(np.abs(v - hi - lo)) < 2.0 ** -9 * np.mean(np.abs(v - hi))


def test_split_e4m3_against_torch():
    rng = np.random.default_rng(21)
    v = np.concatenate([rng.uniform(-448, 448, 100000), rng.normal(size=100000) * 10.0 ** rng.uniform(-3, 2, 100000)])
    hi, lo = emulate.split_e4m3(v)
    v16 = torch.from_numpy(v.astype(np.float16))   # numpy rounds FP64 -> FP16 once (torch may round twice)
    t_hi = v16.to(torch.float8_e4m3fn)
    t_res = (v16.to(torch.float64) - t_hi.to(torch.float64))
    # the residual of an E4M3 rounding of an FP16 value is itself an FP16 value
    assert torch.equal(t_res.to(torch.float16).to(torch.float64), t_res)
    t_lo = t_res.to(torch.float8_e4m3fn)
    np.testing.assert_array_equal(hi, t_hi.to(torch.float64).numpy())
    np.testing.assert_array_equal(lo, t_lo.to(torch.float64).numpy())
    # the pair holds ~8 significant bits: |v16 - hi - lo| <= 2^-8 |v16| + 2^-10
    v16 = v16.to(torch.float64).numpy()
    assert np.all(np.abs(v16 - hi - lo) <= 2.0 ** -8 * np.abs(v16) + 2.0 ** -10)


def test_fp16_split_brute_force_tiny():
    """Nested explicit sums of the three products at widths 3 -> 2 -> 2."""
    rng = np.random.default_rng(22)
    ws, bs = _net(rng, [3, 2, 2])
    x = rng.random((5, 3))
    got = emulate.forward_fp16_split(x, ws, bs, round_output=False)
    r16 = lambda t: float(quant.round_fp16(t))
    for t in range(5):
        h = [float(v) for v in x[t]]
        for l, (w, b) in enumerate(zip(ws, bs)):
            nxt = []
            for j in range(w.shape[0]):
                bh = r16(b[j]); bl = r16(b[j] - bh)
                acc = bh + bl
                for i in range(w.shape[1]):
                    ah = r16(h[i]); al = r16(h[i] - ah)
                    wh = r16(w[j, i]); wl = r16(w[j, i] - wh)
                    acc += ah * wh + al * wh + ah * wl
                nxt.append(max(acc, 0.0) if l == 0 else acc)
            h = nxt
        np.testing.assert_allclose(got[t], h, rtol=0, atol=1e-15)


def test_fp16_split_close_to_fp64_and_each_term_matters():
    """Before the output rounding the split form is within 1e-5 of the FP64 MLP on
    a He-initialised 12-64-64-64-9 network; dropping any of the three products
    (or a sign error in lo) leaves it ~1e-3 away."""
    rng = np.random.default_rng(23)
    ws, bs = _net(rng, [12, 64, 64, 64, 9])
    x = rng.random((4000, 12))
    ref = mlp.forward(x, ws, bs)
    got = emulate.forward_fp16_split(x, ws, bs, round_output=False)
    assert np.abs(got - ref).max() < 1e-5
    y = emulate.forward_fp16_split(x, ws, bs)
    assert np.all(quant.round_fp16(y) == y)
    # only the output rounding remains: within half an FP16 unit of |ref| (+ the 1e-5)
    assert np.all(np.abs(y - ref) <= 2.0 ** -11 * np.maximum(np.abs(ref), 2.0 ** -14) * 2 + 1e-5)

    def variant(drop):
        ah, al = emulate.split_fp16(x)
        for l, (w, b) in enumerate(zip(ws, bs)):
            wh, wl = emulate.split_fp16(w)
            bh, bl = emulate.split_fp16(b)
            terms = {"hh": ah @ wh.T, "lh": al @ wh.T, "hl": ah @ wl.T}
            z = sum(t for k, t in terms.items() if k != drop) + bh + bl
            if drop == "sign":
                z = ah @ wh.T - al @ wh.T + ah @ wl.T + bh + bl
            if l < len(ws) - 1:
                ah, al = emulate.split_fp16(np.maximum(z, 0.0))
        return z
    for drop in ("hh", "lh", "hl", "sign"):
        assert np.abs(variant(drop) - ref).max() > 3e-4, drop


def test_fp8_split_brute_force_tiny_and_bound():
    rng = np.random.default_rng(24)
    ws, bs = _net(rng, [3, 2, 2])
    x = rng.random((5, 3))
    sw, sa = emulate.fp8_scales(ws, mlp.hidden_activations(x, ws, bs))
    got = emulate.forward_fp8_split(x, ws, bs, sw, sa, round_output=False)
    e4 = lambda t: float(quant.round_e4m3_satfinite(t))
    r16 = lambda t: float(quant.round_fp16(t))
    for t in range(5):
        h = [float(v) for v in x[t]]
        for l, (w, b) in enumerate(zip(ws, bs)):
            nxt = []
            for j in range(w.shape[0]):
                acc = 0.0
                for i in range(w.shape[1]):
                    q16 = r16(h[i] / sa[l]); qh = e4(q16); ql = e4(q16 - qh)
                    w16 = r16(w[j, i] / sw[l]); wh = e4(w16); wl = e4(w16 - wh)
                    acc += qh * wh + ql * wh + qh * wl
                z = acc * sw[l] * sa[l] + b[j]
                nxt.append(max(z, 0.0) if l == 0 else z)
            h = nxt
        np.testing.assert_allclose(got[t], h, rtol=0, atol=1e-15)
    # on the 12-64-64-64-9 network the split E4M3 form stays within 2e-2 of FP64
    # (the single-rounding E4M3 form does not)
    ws, bs = _net(rng, [12, 64, 64, 64, 9])
    x = rng.random((4000, 12))
    sw, sa = emulate.fp8_scales(ws, mlp.hidden_activations(x, ws, bs))
    ref = mlp.forward(x, ws, bs)
    assert np.abs(emulate.forward_fp8_split(x, ws, bs, sw, sa) - ref).max() < 2e-2
    assert np.abs(emulate.forward_fp8(x, ws, bs, sw, sa) - ref).max() > 5e-2


def _fp32_kernel(form, x, ws, bs, scales, drop_lo_a=False, seed=1):
    """A plain FP32 simulation of a kernel of `form`: features perturbed at the
    FP32 level, every product sum and epilogue in float32 (numpy's order)."""
    rng = np.random.default_rng(seed)
    f32 = lambda t: np.asarray(t, dtype=np.float32)
    n = len(ws)
    sw, sa = scales if form.startswith("fp8") else ([1.0] * n, [1.0] * (n + 1))
    v = (x * (1 + rng.uniform(-2.0 ** -23, 2.0 ** -23, x.shape))).astype(np.float32).astype(np.float64) / sa[0]
    for l, (w, b) in enumerate(zip(ws, bs)):
        ah, al = emulate._parts(form, f32(v).astype(np.float64))
        if drop_lo_a:
            al = 0.0 * al
        wh, wl = emulate._parts(form, np.asarray(w, np.float64) / sw[l])
        acc = f32(ah) @ f32(wh).T + f32(al) @ f32(wh).T + f32(ah) @ f32(wl).T
        if form.startswith("fp8"):
            z = f32(acc * np.float32(sw[l] * sa[l]) + f32(b))
        else:
            bh, bl = emulate._parts(form, np.asarray(b, np.float64))
            z = f32(acc + f32(bh) + f32(bl))
        z = z.astype(np.float64)
        if l < n - 1:
            v = np.maximum(z, 0.0) / sa[l + 1]
    return quant.round_fp16(z)


def test_output_interval_holds_an_fp32_kernel_and_rejects_a_broken_one():
    rng = np.random.default_rng(25)
    ws, bs = _net(rng, [12, 64, 64, 64, 9])
    x = rng.random((3000, 12))
    scales = emulate.fp8_scales(ws, mlp.hidden_activations(x, ws, bs))
    for form in emulate.FORMS:
        sc = scales if form.startswith("fp8") else None
        y, lo, hi = emulate.output_interval(form, x, ws, bs, sc)
        ref_emu = {"fp16": lambda: emulate.forward_fp16(x, ws, bs),
                   "fp16s": lambda: emulate.forward_fp16_split(x, ws, bs),
                   "fp8": lambda: emulate.forward_fp8(x, ws, bs, *scales),
                   "fp8s": lambda: emulate.forward_fp8_split(x, ws, bs, *scales)}[form]()
        np.testing.assert_array_equal(y, ref_emu)
        assert np.all((lo <= y) & (y <= hi))
        for seed in (1, 2):
            k = _fp32_kernel(form, x, ws, bs, sc, seed=seed)
            assert np.all((lo <= k) & (k <= hi)), form
        if form in ("fp16s", "fp8s"):
            bad = _fp32_kernel(form, x, ws, bs, sc, drop_lo_a=True)
            assert np.mean((bad < lo) | (bad > hi)) > 0.05, form


def test_output_interval_fp16_split_is_tight():
    """Split FP16: no hidden rounding decision moves an output, so each output's
    admissible interval is its emulated value or that and one FP16 neighbour (an
    output rounding tie) -- for outputs whose FP16 unit exceeds the FP32 noise of
    the sums (|y| >= 1/4 here; smaller outputs get a few of their finer units)."""
    rng = np.random.default_rng(26)
    ws, bs = _net(rng, [12, 64, 64, 64, 9])
    x = rng.random((3000, 12))
    y, lo, hi = emulate.output_interval("fp16s", x, ws, bs)
    big = np.abs(y) >= 0.25
    ulp = np.ldexp(1.0, np.floor(np.log2(np.abs(y[big]))).astype(np.int64) - 10)
    assert np.all((hi[big] - lo[big]) <= 2 * ulp)
    assert np.all(hi - lo <= 2.0 ** -9)
    assert np.mean(lo == hi) > 0.8
