// Texel-centre coordinate (i + 1/2) / n of a grid index, correctly rounded to
// FP32, from a reciprocal fixed per grid: the correction step of Markstein
// ("Computation of elementary functions on the IBM RISC System/6000 processor",
// IBM J. Res. Dev. 34(1), 1990).  With r = RN(1/n) and a first quotient
// q = RN(a r) within an ulp of a / n, the remainder e = a - q n is exact as one
// FMA, and RN(q + e r) = RN(a / n).  Exact when n is a power of two; checked
// exhaustively against IEEE division on the host.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define NBTC_HD __host__ __device__
#else
#define NBTC_HD
#endif

namespace nbtc {

struct GridCoord {
  float n;  // grid size
  float r;  // RN(1 / n)
};

inline GridCoord make_grid_coord(int n) {
  GridCoord g;
  g.n = (float)n;
  g.r = 1.0f / (float)n;
  return g;
}

// i < 2^23, so i + 1/2 is exact.
NBTC_HD inline float grid_coord(float i, const GridCoord& g) {
  const float a = i + 0.5f;
#ifdef __CUDA_ARCH__
  const float q = __fmul_rn(a, g.r);
#else
  const float q = a * g.r;
#endif
  const float e = fmaf(-q, g.n, a);
  return fmaf(e, g.r, q);
}

}  // namespace nbtc
