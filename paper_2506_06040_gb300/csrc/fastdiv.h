// Division of a non-negative 31-bit integer by a run-time invariant divisor as
// one 32x32->64-bit multiply and a shift (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Theorem 4.2 with N = 31):
// for 1 <= d < 2^31, l = ceil(log2 d) and m = ceil(2^(31+l) / d) (< 2^32),
// floor(n / d) = floor(m n / 2^(31+l)) for every 0 <= n < 2^31.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define NBTC_HD __host__ __device__
#else
#define NBTC_HD
#endif

namespace nbtc {

struct FastDiv {
  uint32_t m;   // multiplier
  uint32_t sh;  // 31 + l
  uint32_t d;   // the divisor
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while (l < 31 && (1u << l) < d) ++l;
  const uint64_t p = (uint64_t)1 << (31 + l);
  FastDiv f;
  f.m = (uint32_t)((p + d - 1) / d);
  f.sh = 31 + l;
  f.d = d;
  return f;
}

// floor(n / f.d) for 0 <= n < 2^31
NBTC_HD inline uint32_t fastdiv(uint32_t n, const FastDiv& f) { return (uint32_t)(((uint64_t)n * f.m) >> f.sh); }

}  // namespace nbtc
