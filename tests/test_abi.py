"""The C-ABI library builds, loads and exports every entry point include/nbtc.h
declares; ctypes struct layouts match the C compiler's; host-only argument
checks answer without a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nbtc.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:nbtc_status|const char\*|void)\s+(nbtc_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_06040_gb300 import _abi
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2506_06040_gb300 import _abi
    assert sorted(_abi.PROTOTYPES) == _declared()


def test_struct_layouts_match_c():
    from paper_2506_06040_gb300 import _abi
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "nbtc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(nbtc_level), offsetof(nbtc_level, width), offsetof(nbtc_level, shift),
         sizeof(nbtc_latents), offsetof(nbtc_latents, levels));
  printf("%zu %zu %zu\n", sizeof(nbtc_mlp), offsetof(nbtc_mlp, weights), offsetof(nbtc_mlp, biases));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(nbtc_train_args), offsetof(nbtc_train_args, mlp),
         offsetof(nbtc_train_args, target_w), offsetof(nbtc_train_args, batch), offsetof(nbtc_train_args, loss),
         offsetof(nbtc_train_args, workspace), offsetof(nbtc_train_args, workspace_bytes));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    got = [int(x) for x in out]
    want = [ctypes.sizeof(_abi.Level), _abi.Level.width.offset, _abi.Level.shift.offset,
            ctypes.sizeof(_abi.Latents), _abi.Latents.levels.offset,
            ctypes.sizeof(_abi.Mlp), _abi.Mlp.weights.offset, _abi.Mlp.biases.offset,
            ctypes.sizeof(_abi.TrainArgs), _abi.TrainArgs.mlp.offset, _abi.TrainArgs.target_w.offset,
            _abi.TrainArgs.batch.offset, _abi.TrainArgs.loss.offset, _abi.TrainArgs.workspace.offset,
            _abi.TrainArgs.workspace_bytes.offset]
    assert got == want


def test_host_only_checks(lib):
    from paper_2506_06040_gb300 import _abi
    for code in range(6):
        assert lib.nbtc_status_string(code)
    assert lib.nbtc_destroy(None) == _abi.OK
    assert lib.nbtc_create(0, None) == _abi.ERR_INVALID_ARG
    n = ctypes.c_size_t(7)
    assert lib.nbtc_packed_mlp_bytes(None, 0, ctypes.byref(n)) == _abi.ERR_INVALID_ARG
    m = _abi.Mlp()
    m.num_layers = 3
    for i, d in enumerate([12, 64, 64, 9]):
        m.dims[i] = d
    assert lib.nbtc_packed_mlp_bytes(ctypes.byref(m), 0, ctypes.byref(n)) == _abi.ERR_INVALID_ARG  # NULL weights
    m.weights, m.biases = 16, 16
    assert lib.nbtc_packed_mlp_bytes(ctypes.byref(m), _abi.FP32, ctypes.byref(n)) == _abi.OK and n.value == 0
    m.num_layers = 7
    assert lib.nbtc_packed_mlp_bytes(ctypes.byref(m), _abi.FP32, ctypes.byref(n)) == _abi.ERR_INVALID_ARG
    assert b"num_layers" in lib.nbtc_last_error()
    assert lib.nbtc_set_wait_budget(None, 5) == _abi.ERR_INVALID_ARG


def test_product_path_fails_loudly_without_library(monkeypatch):
    from paper_2506_06040_gb300 import _abi
    monkeypatch.setattr(_abi, "LIB_PATH", "/nonexistent/libnbtc.so")
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _abi.load()
