"""The invariant-divisor division the tensor-core decode uses to map tile
numbers to (column block, row) -- Granlund and Montgomery's multiply-and-shift
with N = 31 -- against exact integer division, host-compiled with g++: every
divisor up to 2^16 and powers of two, near-powers and random divisors up to
2^31 - 1, each on the dividends where an error would first show (multiples of
d and their neighbours, the top of the range) plus random ones."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cstdio>
#include <cstdint>
#include <random>
#include "fastdiv.h"
using namespace nbtc;
static int check(uint32_t d, std::mt19937_64& g) {
  const FastDiv f = make_fastdiv(d);
  if (f.m == 0 && d != 1) return 1;
  auto one = [&](uint32_t n) { return fastdiv(n, f) != n / d; };
  const uint32_t top = 0x7FFFFFFFu;
  for (uint32_t n : {0u, 1u, d - 1, d, d + 1, top, top - 1, top - d % 1000}) if (n <= top && one(n)) return 2;
  for (uint64_t q = top / d; q + 3 > top / d && q > 0 && q * d <= top; --q) {  // last multiples
    const uint32_t n = (uint32_t)(q * d);
    if (one(n) || (n > 0 && one(n - 1)) || (n < top && one(n + 1))) return 3;
  }
  for (int i = 0; i < 200; ++i) { const uint32_t n = (uint32_t)(g() & top); if (one(n)) return 4; }
  return 0;
}
int main() {
  std::mt19937_64 g(12345);
  for (uint32_t d = 1; d <= 65536; ++d) if (int e = check(d, g)) { printf("FAIL d=%u code=%d\n", d, e); return 1; }
  for (int l = 16; l < 31; ++l) for (int64_t dd : {-1, 0, 1}) {
    const uint32_t d = (uint32_t)((int64_t(1) << l) + dd);
    if (int e = check(d, g)) { printf("FAIL d=%u code=%d\n", d, e); return 1; }
  }
  for (int i = 0; i < 20000; ++i) {
    const uint32_t d = 1 + (uint32_t)(g() % 0x7FFFFFFEu);
    if (int e = check(d, g)) { printf("FAIL d=%u code=%d\n", d, e); return 1; }
  }
  printf("OK\n");
  return 0;
}
'''


def test_fastdiv_matches_integer_division():
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.cpp")
        open(c, "w").write(SRC)
        exe = os.path.join(d, "t")
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-I",
                               os.path.join(ROOT, "paper_2506_06040_gb300", "csrc"), c, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300).stdout
    assert out.strip() == "OK", out
