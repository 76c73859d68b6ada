// Quantisation-aware BC1 latents (Sec. 3.2, Eqs. 1-3): decode of the raw
// parameters to the latent texture, the straight-through backward to the raw
// parameters, the encoder to BC1 blocks, and the QAT training step that wraps
// the continuous-latent step around them.
//
// Quantiser levels are decided without an exp: the level of raw parameter p
// on b bits is the number of thresholds logit((j + 1/2) / (2^b - 1)) (computed
// in double on the host, rounded to FP32) that p reaches, i.e. the nearest
// level of sigmoid(p).  The sigmoid itself only enters the gradients.
#include <cmath>

#include "host.h"

namespace nbtc {

namespace {

struct QatThresholds {
  float t2[3];    // alpha: 2 bits
  float t5[31];   // red / blue: 5 bits
  float t6[63];   // green: 6 bits
};

QatThresholds make_thresholds() {
  QatThresholds T;
  auto fill = [](float* t, int n) {
    for (int j = 0; j < n; ++j) {
      const double m = (j + 0.5) / n;
      t[j] = (float)std::log(m / (1.0 - m));
    }
  };
  fill(T.t2, 3);
  fill(T.t5, 31);
  fill(T.t6, 63);
  return T;
}

// Number of the (ascending) thresholds t[0 .. n-1] that p reaches (p >= t[j]),
// by binary search.
__device__ __forceinline__ int qlevel(float p, const float* t, int n) {
  int lo = 0, hi = n;  // answer in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (p >= t[mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ float sigm(float p) { return 1.0f / (1.0f + expf(-p)); }

struct QatLevelDev {
  int w, h;
  const float* e0;
  const float* e1;
  const float* alpha;
};

// Quantised endpoint colour (levels / (2^b - 1)) of raw endpoint e[0..2].
__device__ __forceinline__ float3 endpoint_value(const float* e, const QatThresholds& T) {
  return make_float3((float)qlevel(e[0], T.t5, 31) / 31.f, (float)qlevel(e[1], T.t6, 63) / 63.f,
                     (float)qlevel(e[2], T.t5, 31) / 31.f);
}

// Up to 4 levels per launch, level blockIdx.y: its raw parameters, its decoded
// texture (or dL/dT) and the straight-through gradients.
struct QatJobs {
  QatLevelDev L[4];
  float* tex[4];
  float* g_e0[4];
  float* g_e1[4];
  float* g_alpha[4];
};

// One thread per texel: T = (1 - a) E0 + a E1, written with ls floats per texel
// (3, or 4 with the padding channel set to 0).
__global__ void k_qat_decode(QatJobs J, QatThresholds T, int ls) {
  const QatLevelDev L = J.L[blockIdx.y];
  float* __restrict__ out = J.tex[blockIdx.y];
  const int64_t n = (int64_t)L.w * L.h;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / L.w), x = (int)(i - (int64_t)y * L.w);
    const int64_t b = (int64_t)(y >> 2) * (L.w >> 2) + (x >> 2);
    const float3 E0 = endpoint_value(L.e0 + 3 * b, T), E1 = endpoint_value(L.e1 + 3 * b, T);
    const float a = (float)qlevel(L.alpha[i], T.t2, 3) / 3.f;
    const float t0 = fmaf(a, E1.x - E0.x, E0.x), t1 = fmaf(a, E1.y - E0.y, E0.y), t2 = fmaf(a, E1.z - E0.z, E0.z);
    if (ls == 4) {
      reinterpret_cast<float4*>(out)[i] = make_float4(t0, t1, t2, 0.f);
    } else {
      out[3 * i + 0] = t0;
      out[3 * i + 1] = t1;
      out[3 * i + 2] = t2;
    }
  }
}

// One thread per block: straight-through gradients of its two endpoints and
// sixteen blend factors from dL/dT (ls floats per texel).
__global__ void k_qat_backward(QatJobs J, QatThresholds T, int ls) {
  const QatLevelDev L = J.L[blockIdx.y];
  const float* __restrict__ dT = J.tex[blockIdx.y];
  float* __restrict__ g_e0 = J.g_e0[blockIdx.y];
  float* __restrict__ g_e1 = J.g_e1[blockIdx.y];
  float* __restrict__ g_alpha = J.g_alpha[blockIdx.y];
  const int wb = L.w >> 2;
  const int64_t nb = (int64_t)wb * (L.h >> 2);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const int by = (int)(b / wb), bx = (int)(b - (int64_t)by * wb);
    const float3 E0 = endpoint_value(L.e0 + 3 * b, T), E1 = endpoint_value(L.e1 + 3 * b, T);
    float s0[3] = {0.f, 0.f, 0.f}, s1[3] = {0.f, 0.f, 0.f};
    for (int ty = 0; ty < 4; ++ty) {
      for (int tx = 0; tx < 4; ++tx) {
        const int64_t i = (int64_t)(4 * by + ty) * L.w + 4 * bx + tx;
        const float p = L.alpha[i];
        const float a = (float)qlevel(p, T.t2, 3) / 3.f;
        const float d0 = dT[ls * i], d1 = dT[ls * i + 1], d2 = dT[ls * i + 2];
        s0[0] = fmaf(d0, 1.f - a, s0[0]);
        s0[1] = fmaf(d1, 1.f - a, s0[1]);
        s0[2] = fmaf(d2, 1.f - a, s0[2]);
        s1[0] = fmaf(d0, a, s1[0]);
        s1[1] = fmaf(d1, a, s1[1]);
        s1[2] = fmaf(d2, a, s1[2]);
        const float sa = sigm(p);
        g_alpha[i] = (d0 * (E1.x - E0.x) + d1 * (E1.y - E0.y) + d2 * (E1.z - E0.z)) * (sa * (1.f - sa));
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float a0 = sigm(L.e0[3 * b + c]), a1 = sigm(L.e1[3 * b + c]);
      g_e0[3 * b + c] = s0[c] * (a0 * (1.f - a0));
      g_e1[3 * b + c] = s1[c] * (a1 * (1.f - a1));
    }
  }
}

__device__ __forceinline__ uint32_t code565(const float* e, const QatThresholds& T) {
  return ((uint32_t)qlevel(e[0], T.t5, 31) << 11) | ((uint32_t)qlevel(e[1], T.t6, 63) << 5) |
         (uint32_t)qlevel(e[2], T.t5, 31);
}

// One thread per block: four-colour BC1 block from the quantised parameters.
__global__ void k_qat_encode(QatLevelDev L, uint64_t* __restrict__ blocks, QatThresholds T) {
  const int wb = L.w >> 2;
  const int64_t nb = (int64_t)wb * (L.h >> 2);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const int by = (int)(b / wb), bx = (int)(b - (int64_t)by * wb);
    const uint32_t c0 = code565(L.e0 + 3 * b, T), c1 = code565(L.e1 + 3 * b, T);
    uint32_t word = 0;
    if (c0 != c1) {
      const bool swap = c0 < c1;
      for (int ty = 0; ty < 4; ++ty) {
        for (int tx = 0; tx < 4; ++tx) {
          int q = qlevel(L.alpha[(int64_t)(4 * by + ty) * L.w + 4 * bx + tx], T.t2, 3);
          if (swap) q = 3 - q;
          // level q (weight q / 3 on the second endpoint) -> palette index
          const uint32_t idx = q == 0 ? 0u : q == 1 ? 2u : q == 2 ? 3u : 1u;
          word |= idx << (2 * (4 * ty + tx));
        }
      }
    }
    const uint32_t first = c0 > c1 ? c0 : c1, second = c0 > c1 ? c1 : c0;
    blocks[b] = (uint64_t)first | ((uint64_t)second << 16) | ((uint64_t)word << 32);
  }
}

nbtc_status check_qat_level(const nbtc_qat_level* q, bool step) {
  if (!q) return fail(NBTC_ERR_INVALID_ARG, "QAT level NULL");
  if (q->width <= 0 || q->height <= 0 || q->width % 4 || q->height % 4 || q->width > (1 << 15) ||
      q->height > (1 << 15))
    return fail(NBTC_ERR_INVALID_ARG, "QAT level size must be positive multiples of 4 (<= 32768)");
  if (!q->e0 || !q->e1 || !q->alpha) return fail(NBTC_ERR_INVALID_ARG, "QAT parameters NULL");
  if (step && (!q->g_e0 || !q->g_e1 || !q->g_alpha || !q->m_e0 || !q->v_e0 || !q->m_e1 || !q->v_e1 ||
               !q->m_alpha || !q->v_alpha))
    return fail(NBTC_ERR_INVALID_ARG, "QAT gradients or moments NULL");
  // pointer kinds: device or pinned host memory
  const void* ptrs[12] = {q->e0, q->e1, q->alpha, q->g_e0, q->g_e1, q->g_alpha,
                          q->m_e0, q->v_e0, q->m_e1, q->v_e1, q->m_alpha, q->v_alpha};
  for (int i = 0; i < (step ? 12 : 3); ++i) {
    nbtc_status st = need_readable(ptrs[i], "a QAT parameter, gradient or moment array");
    if (st) return st;
  }
  return NBTC_OK;
}

QatLevelDev level_dev(const nbtc_qat_level* q) { return QatLevelDev{q->width, q->height, q->e0, q->e1, q->alpha}; }

int grid_for(nbtc_context* ctx, int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > (int64_t)ctx->sm_count * 16) g = (int64_t)ctx->sm_count * 16;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

nbtc_status qat_decode(nbtc_context* ctx, const nbtc_qat_level* q, float* out, cudaStream_t s) {
  nbtc_status st = check_qat_level(q, false);
  if (st) return st;
  if (!out) return fail(NBTC_ERR_INVALID_ARG, "out NULL");
  if ((st = need_readable(out, "out"))) return st;
  QatJobs J{};
  J.L[0] = level_dev(q);
  J.tex[0] = out;
  k_qat_decode<<<grid_for(ctx, (int64_t)q->width * q->height), 256, 0, s>>>(J, make_thresholds(), 3);
  return cuda_check(cudaGetLastError(), "launch k_qat_decode");
}

nbtc_status qat_encode(nbtc_context* ctx, const nbtc_qat_level* q, uint64_t* blocks, cudaStream_t s) {
  nbtc_status st = check_qat_level(q, false);
  if (st) return st;
  if (!blocks || !aligned(blocks, 8)) return fail(NBTC_ERR_INVALID_ARG, "blocks NULL or not 8-byte aligned");
  if ((st = need_readable(blocks, "blocks"))) return st;
  k_qat_encode<<<grid_for(ctx, (int64_t)(q->width / 4) * (q->height / 4)), 256, 0, s>>>(level_dev(q), blocks,
                                                                                      make_thresholds());
  return cuda_check(cudaGetLastError(), "launch k_qat_encode");
}

nbtc_status train_step_qat(nbtc_context* ctx, const nbtc_train_args* A, const nbtc_qat_level* levels, float* loss,
                           cudaStream_t s) {
  if (!A || !levels) return fail(NBTC_ERR_INVALID_ARG, "args or levels NULL");
  if (A->num_levels != 4) return fail(NBTC_ERR_UNSUPPORTED, "training takes 4 latent levels");
  nbtc_status st;
  const int ls = latent_stride(A);
  if (!ls) return fail(NBTC_ERR_INVALID_ARG, "latent_stride must be 3 or 4 (0 means 3)");
  for (int k = 0; k < 4; ++k) {
    if ((st = check_qat_level(&levels[k], true))) return st;
    if (ls == 4 && (!aligned(A->latents[k], 16) || !aligned(A->latent_grads[k], 16)))
      return fail(NBTC_ERR_INVALID_ARG, "latent_stride 4 wants 16-byte aligned latents and gradients");
    if (levels[k].width != A->widths[k] || levels[k].height != A->heights[k])
      return fail(NBTC_ERR_INVALID_ARG, "QAT level size differs from the decoded latent size");
    if (!A->latents[k] || !A->latent_grads[k]) return fail(NBTC_ERR_INVALID_ARG, "latent or gradient NULL");
  }
  // the four levels in one launch each: decode, straight-through backward, Adam
  const QatThresholds T = make_thresholds();
  QatJobs D{}, B{};
  AdamSegs S;
  S.count = 12;
  int64_t nt_max = 0, nb_max = 0;
  for (int k = 0; k < 4; ++k) {
    const nbtc_qat_level& q = levels[k];
    const int64_t nb = (int64_t)(q.width / 4) * (q.height / 4), nt = (int64_t)q.width * q.height;
    nt_max = nt > nt_max ? nt : nt_max;
    nb_max = nb > nb_max ? nb : nb_max;
    D.L[k] = B.L[k] = level_dev(&q);
    D.tex[k] = A->latents[k];
    B.tex[k] = A->latent_grads[k];
    B.g_e0[k] = q.g_e0;
    B.g_e1[k] = q.g_e1;
    B.g_alpha[k] = q.g_alpha;
    S.seg[3 * k + 0] = AdamSeg{q.e0, q.g_e0, q.m_e0, q.v_e0, 3 * nb};
    S.seg[3 * k + 1] = AdamSeg{q.e1, q.g_e1, q.m_e1, q.v_e1, 3 * nb};
    S.seg[3 * k + 2] = AdamSeg{q.alpha, q.g_alpha, q.m_alpha, q.v_alpha, nt};
  }
  k_qat_decode<<<dim3(grid_for(ctx, nt_max), 4), 256, 0, s>>>(D, T, ls);
  if ((st = cuda_check(cudaGetLastError(), "launch k_qat_decode"))) return st;
  if ((st = train_step_impl(ctx, A, loss, s, 3, nullptr, nullptr, A->workspace, A->workspace_bytes))) return st;
  k_qat_backward<<<dim3(grid_for(ctx, nb_max), 4), 256, 0, s>>>(B, T, ls);
  if ((st = cuda_check(cudaGetLastError(), "launch k_qat_backward"))) return st;
  return launch_adam(ctx, A, A->lr_latent, S, s);
}

}  // namespace nbtc
