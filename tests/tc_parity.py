"""Parity checks of the precision forms against the oracle's emulator, shared by
the GPU tests (the oracle side only; no method arithmetic here).

check_interval: every kernel output must lie in the interval of FP16 values the
emulator admits for it (oracle.emulate.output_interval): the emulated value
itself wherever no rounding decision of the network is within FP32 noise of a
boundary, else the values the doubtful decisions can reach.

Full-size checks run the oracle on row bands of the 4096^2 workloads in a pool of
spawned worker processes (one per host core): each worker regenerates the seeded
workload, decodes the BC1 levels once and checks the bands it is given."""
import os
import multiprocessing as mp

import numpy as np

import oracle
import synth

FORM_NAMES = ("fp16", "fp16s", "fp8", "fp8s")
# FP32 error of the kernels' features (standard deviation of the error model):
# single-level bilinear blends in FP32 on FP32 texture coordinates
SIGMA_GRID = 2.0 ** -22


def ulp16(x):
    """Spacing of binary16 numbers at |x| (2^-24 below the normal range)."""
    ax = np.maximum(np.abs(np.asarray(x, dtype=np.float64)), 2.0 ** -14)
    return np.ldexp(1.0, np.floor(np.log2(ax)).astype(np.int64) - 10)


def check_interval(got, material, x, form, scales=None, sigma_x=SIGMA_GRID, what=""):
    """Asserts every output lies in its admissible interval; returns statistics."""
    got = np.asarray(got, dtype=np.float64)
    assert np.all(np.isfinite(got)), what
    y, lo, hi = oracle.decode.mlp_interval(material, x, form, scales, sigma_x=sigma_x)
    bad = (got < lo) | (got > hi)
    if bad.any():
        t, c = np.argwhere(bad)[0]
        raise AssertionError(f"{what} {form}: {int(bad.sum())} of {bad.size} outputs outside their admissible "
                             f"interval; first texel {t} channel {c}: got {got[t, c]!r}, emulator {y[t, c]!r}, "
                             f"interval [{lo[t, c]!r}, {hi[t, c]!r}]")
    return {"n": int(got.size), "equal": float(np.mean(got == y)), "single": float(np.mean(lo == hi)),
            "max_dev": float(np.abs(got - y).max()),
            "max_width_ulps": float(np.max((hi - lo) / ulp16(y)))}


# ------------------------------------------------------------------ full-size bands

_CACHE = {}


def _workload(k):
    if k not in _CACHE:
        wl = synth.decode_workload(k)
        tex = [oracle.decode.level_rgb(lv) for lv in wl.material.levels]
        _CACHE.clear()
        _CACHE[k] = (wl, tex)
    return _CACHE[k]


def _band_x(k, row0, rows):
    wl, tex = _workload(k)
    idx = np.arange(row0 * wl.out_w, (row0 + rows) * wl.out_w)
    u = oracle.sample.grid_coord(idx % wl.out_w, wl.out_w).astype(np.float64)
    v = oracle.sample.grid_coord(idx // wl.out_w, wl.out_h).astype(np.float64)
    return wl, oracle.decode.features_at(wl.material, u, v, tex)


def band_fp32(args):
    """FP32 form: per-channel max |kernel - FP64 oracle| of rows [row0, row0 + rows)."""
    k, row0, rows, got = args
    wl, x = _band_x(k, row0, rows)
    ref = oracle.mlp.forward(x, wl.material.mlp.weights, wl.material.mlp.biases)
    return np.abs(got.astype(np.float64) - ref).max(axis=0)


def band_form(args):
    """Precision form: interval statistics and per-channel max |kernel - FP64| and
    |emulator - FP64| of rows [row0, row0 + rows)."""
    k, form, scales, row0, rows, got = args
    wl, x = _band_x(k, row0, rows)
    got = got.astype(np.float64)
    st = check_interval(got, wl.material, x, form, scales, what=f"rows {row0}..{row0 + rows}")
    ref = oracle.mlp.forward(x, wl.material.mlp.weights, wl.material.mlp.biases)
    emu = oracle.decode.run_mlp(wl.material, x, form, scales)
    return st, np.abs(got - ref).max(axis=0), np.abs(emu - ref).max(axis=0)


def pool():
    """Spawned workers, one per host core, single-threaded BLAS each."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 4)
    return mp.get_context("spawn").Pool(n)


def bands(height, rows):
    return [(r, min(rows, height - r)) for r in range(0, height, rows)]
