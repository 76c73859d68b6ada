"""The grid texel-centre coordinate the decode kernels use -- (i + 1/2) / n as
RN(1/n) times the numerator plus Markstein's correction step -- against IEEE
FP32 division, host-compiled with g++ (same FMA semantics as the device's
fmaf): every index of every grid size up to 2^14, powers of two and their
neighbours up to 2^20 (where every index must come out exact for the powers),
and random sizes and indices up to 2^20."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cstdio>
#include <cstdint>
#include <random>
#include "gridcoord.h"
using namespace nbtc;
static volatile float sink;
static bool same(float a, float b) { return a == b; }
static int check(int n, int64_t i0, int64_t i1, int64_t step) {
  const GridCoord g = make_grid_coord(n);
  const float fn = (float)n;
  for (int64_t i = i0; i < i1; i += step) {
    const float a = (float)i + 0.5f;
    volatile float num = a, den = fn;
    const float want = num / den;  // IEEE FP32 division, correctly rounded
    const float got = grid_coord((float)i, g);
    if (!same(got, want)) { printf("FAIL n=%d i=%lld got=%a want=%a\n", n, (long long)i, got, want); return 1; }
    if ((n & (n - 1)) == 0 && (double)got * n != (double)i + 0.5) { printf("INEXACT n=%d i=%lld\n", n, (long long)i); return 1; }
  }
  return 0;
}
int main() {
  for (int n = 1; n <= 16384; ++n) if (check(n, 0, n, 1)) return 1;
  for (int l = 14; l <= 20; ++l)
    for (int d = -2; d <= 2; ++d) {
      const int n = (1 << l) + d;
      if (check(n, 0, n, 7) || check(n, n - 64, n, 1)) return 1;
    }
  std::mt19937_64 rng(2024);
  for (int t = 0; t < 4000; ++t) {
    const int n = 1 + (int)(rng() % (1u << 20));
    for (int k = 0; k < 250; ++k) { const int64_t i = (int64_t)(rng() % (uint64_t)n); if (check(n, i, i + 1, 1)) return 1; }
  }
  printf("OK\n");
  return 0;
}
'''


def test_grid_coord_is_correctly_rounded():
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.cpp"), os.path.join(d, "t")
        open(src, "w").write(SRC)
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                               "-I", os.path.join(ROOT, "paper_2506_06040_gb300", "csrc"), src, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout[-500:]
