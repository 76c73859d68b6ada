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
    """Every ctypes struct of the binding has the C compiler's size and every
    field the C compiler's offset; the precision codes match the header's."""
    from paper_2506_06040_gb300 import _abi
    pairs = [("nbtc_level", _abi.Level), ("nbtc_latents", _abi.Latents), ("nbtc_mlp", _abi.Mlp),
             ("nbtc_train_args", _abi.TrainArgs), ("nbtc_batch_material", _abi.BatchMaterial),
             ("nbtc_frame", _abi.Frame), ("nbtc_batch_info", _abi.BatchInfo)]
    lines, want = [], []
    for cname, val in [("NBTC_FP32", _abi.FP32), ("NBTC_FP16", _abi.FP16), ("NBTC_FP8_E4M3", _abi.FP8_E4M3),
                       ("NBTC_FP16_SPLIT", _abi.FP16_SPLIT), ("NBTC_FP8_E4M3_SPLIT", _abi.FP8_E4M3_SPLIT),
                       ("NBTC_FP32_TC", _abi.FP32_TC)]:
        lines.append(f'  printf("%d\\n", (int){cname});')
        want.append(val)
    for cname, cls in pairs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
            want.append(getattr(cls, f).offset)
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"nbtc.h\"\nint main(void) {\n" + "\n".join(lines) + \
        "\n  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).decode().split()]
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
    sizes = {}
    for prec in (_abi.FP16, _abi.FP8_E4M3, _abi.FP16_SPLIT, _abi.FP8_E4M3_SPLIT, _abi.FP32_TC):
        assert lib.nbtc_packed_mlp_bytes(ctypes.byref(m), prec, ctypes.byref(n)) == _abi.OK
        sizes[prec] = n.value
        assert n.value % 16 == 0
    # the split forms store hi and lo of every weight tile
    assert sizes[_abi.FP16_SPLIT] > sizes[_abi.FP16] > sizes[_abi.FP8_E4M3]
    assert sizes[_abi.FP8_E4M3_SPLIT] > sizes[_abi.FP8_E4M3]
    assert sizes[_abi.FP32_TC] == sizes[_abi.FP16_SPLIT]   # the same operands, FP32 output
    assert lib.nbtc_packed_mlp_bytes(ctypes.byref(m), 6, ctypes.byref(n)) == _abi.ERR_INVALID_ARG
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
