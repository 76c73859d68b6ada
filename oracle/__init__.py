"""CPU oracle for the neural block texture decode -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 (integer where the method is integer) restatement of what
the decode, training and batching paths compute, written from the paper
("Hardware Accelerated Neural Block Texture Compression with Cooperative
Vectors", arXiv 2506.06040) and the BC1 format definition it cites.  Each
function names the passage it follows.

Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline and
reference legs may import this package.  It shares no code with the CUDA
library (`paper_2506_06040_gb300`) and never imports it; the two meet only in
the seeded inputs of the `synth` module.

Pins: every function here is checked in `tests/test_oracle_*.py` against values
fixed by the format definition, closed forms, library routines (numpy float16,
torch float8_e4m3fn, scipy map_coordinates, torch float64 linear layers),
invariants and finite differences.  No function is "parity unpinned".
"""
from . import bc1, sample, mlp, quant, emulate, train, frame, decode, qat, shade  # noqa: F401
