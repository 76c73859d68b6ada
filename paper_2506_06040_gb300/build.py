"""Builds the in-tree CUDA library `libnbtc.so` for sm_103a with nvcc, and its
checked twin `libnbtc_checked.so` (the same sources compiled with NBTC_CHECKED:
every gather index of the kernels is tested against its array's extent, and an
index outside it records NBTC_ERR_BOUNDS in the status word instead of being
used).

Each `csrc/*.cu` compiles to an object under `_build/` (and `_build/checked/`)
in one parallel pass (rebuilt when it or any header is newer), then nvcc links
each set into its shared library next to this file, with the CUDA runtime
linked statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnbtc.so")
LIB_CHECKED = os.path.join(HERE, "libnbtc_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", SRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest_header() -> float:
    hs = glob.glob(os.path.join(SRC, "*.cuh")) + glob.glob(os.path.join(SRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(verbose: bool = False, extra_flags=None, checked: bool = True) -> str:
    """Builds libnbtc.so (and, with checked=True, libnbtc_checked.so); returns
    the path of libnbtc.so."""
    nvcc = _nvcc()
    srcs = sorted(glob.glob(os.path.join(SRC, "*.cu")))
    hdr_t = _newest_header()
    variants = [(OUT_DIR, LIB, [])] + ([(os.path.join(OUT_DIR, "checked"), LIB_CHECKED, ["-DNBTC_CHECKED"])]
                                       if checked else [])
    for d, _, _ in variants:
        os.makedirs(d, exist_ok=True)

    def compile_one(job) -> str:
        src, out_dir, defs = job
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_t) and not extra_flags:
            return obj
        cmd = [nvcc, *ARCH, *FLAGS, *defs, *list(extra_flags or []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    jobs = [(src, d, defs) for d, _, defs in variants for src in srcs]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, jobs))
    for i, (_, lib, _) in enumerate(variants):
        mine = objs[i * len(srcs):(i + 1) * len(srcs)]
        if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in mine):
            cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", lib, *mine, "-cudart", "static"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
