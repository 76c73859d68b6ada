// C-ABI entry points: context, status, argument checks, dispatch.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "host.h"

namespace nbtc {

static thread_local std::string g_last_error;

nbtc_status fail(nbtc_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

nbtc_status cuda_check(cudaError_t err, const char* what) {
  if (err == cudaSuccess) return NBTC_OK;
  return fail(NBTC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
}

nbtc_status enter(nbtc_context* ctx) {
  if (!ctx) return fail(NBTC_ERR_INVALID_ARG, "context is NULL");
  return cuda_check(cudaSetDevice(ctx->device), "cudaSetDevice");
}

nbtc_status check_mlp(const nbtc_mlp* mlp) {
  if (!mlp) return fail(NBTC_ERR_INVALID_ARG, "mlp is NULL");
  if (mlp->num_layers < 2 || mlp->num_layers > NBTC_MAX_LAYERS)
    return fail(NBTC_ERR_INVALID_ARG, "mlp.num_layers must be 2..4");
  for (int l = 0; l <= mlp->num_layers; ++l)
    if (mlp->dims[l] <= 0 || mlp->dims[l] > 4096) return fail(NBTC_ERR_INVALID_ARG, "mlp.dims out of range");
  if (!mlp->weights || !mlp->biases) return fail(NBTC_ERR_INVALID_ARG, "mlp weights/biases NULL");
  if (!aligned(mlp->weights, 4) || !aligned(mlp->biases, 4))
    return fail(NBTC_ERR_INVALID_ARG, "mlp weights/biases not 4-byte aligned");
  return NBTC_OK;
}

PtrKind ptr_kind(const void* p) {
  cudaPointerAttributes pa;
  if (!p || cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    cudaGetLastError();
    return kPtrOther;
  }
  if (pa.type == cudaMemoryTypeManaged) return kPtrDevice;
  if (pa.type == cudaMemoryTypeDevice) {
    // device memory of another GPU is not this launch's to read
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess && pa.device == dev ? kPtrDevice : kPtrOther;
  }
  // pinned host memory that the kernels reach at its own address (the kernels
  // take the caller's pointer as is; a registration mapped elsewhere is refused)
  if (pa.type == cudaMemoryTypeHost && pa.devicePointer == p) return kPtrPinned;
  return kPtrOther;
}

nbtc_status need_readable(const void* p, const char* what) {
  if (ptr_kind(p) == kPtrOther)
    return fail(NBTC_ERR_INVALID_ARG, std::string(what) + " is neither device memory nor pinned host memory");
  return NBTC_OK;
}

nbtc_status need_device(const void* p, const char* what) {
  if (ptr_kind(p) != kPtrDevice) return fail(NBTC_ERR_INVALID_ARG, std::string(what) + " is not device memory");
  return NBTC_OK;
}

nbtc_status need_inputs(const nbtc_latents* lat, const nbtc_mlp* mlp) {
  nbtc_status st;
  if (lat)
    for (int k = 0; k < lat->num_levels && k < NBTC_MAX_LEVELS; ++k)
      if ((st = need_readable(lat->levels[k].blocks, "a level's blocks"))) return st;
  if (mlp) {
    if ((st = need_readable(mlp->weights, "mlp weights"))) return st;
    if ((st = need_readable(mlp->biases, "mlp biases"))) return st;
  }
  return NBTC_OK;
}

nbtc_status make_level_views(const nbtc_latents* lat, int mip, LevelView* views) {
  if (!lat) return fail(NBTC_ERR_INVALID_ARG, "latents is NULL");
  if (lat->num_levels < 1 || lat->num_levels > NBTC_MAX_LEVELS)
    return fail(NBTC_ERR_INVALID_ARG, "num_levels must be 1..8");
  if (lat->address != NBTC_CLAMP && lat->address != NBTC_WRAP)
    return fail(NBTC_ERR_INVALID_ARG, "address must be NBTC_CLAMP or NBTC_WRAP");
  for (int k = 0; k < lat->num_levels; ++k) {
    const nbtc_level& L = lat->levels[k];
    if (!L.blocks) return fail(NBTC_ERR_INVALID_ARG, "level blocks NULL");
    if (!aligned(L.blocks, 8)) return fail(NBTC_ERR_INVALID_ARG, "level blocks not 8-byte aligned");
    if (L.width < 4 || L.height < 4 || (L.width & 3) || (L.height & 3) || L.width > (1 << 16) ||
        L.height > (1 << 16))
      return fail(NBTC_ERR_INVALID_ARG, "level size must be a multiple of 4 in [4, 65536]");
    if (L.num_mips < 1 || L.num_mips > NBTC_MAX_MIPS)
      return fail(NBTC_ERR_INVALID_ARG, "num_mips must be 1..16");
    if (mip < 0 || mip >= L.num_mips) return fail(NBTC_ERR_INVALID_ARG, "mip out of range");
    {  // every mip must tile into whole 4x4 blocks: mip m is max(4, size >> m)
      int w = L.width, h = L.height;
      for (int m = 1; m < L.num_mips; ++m) {
        if ((w / 2 >= 4 && (w / 2) % 4) || (h / 2 >= 4 && (h / 2) % 4) || (w % 2 && w > 4) || (h % 2 && h > 4))
          return fail(NBTC_ERR_INVALID_ARG, "a mip is not a whole number of 4x4 blocks");
        w = w / 2 < 4 ? 4 : w / 2;
        h = h / 2 < 4 ? 4 : h / 2;
      }
    }
    if (!(L.shift > -64.f && L.shift < 64.f)) return fail(NBTC_ERR_INVALID_ARG, "shift out of range");
    size_t off = 0;
    int w = L.width, h = L.height;
    for (int m = 0; m < mip; ++m) {
      off += (size_t)(w / 4) * (h / 4);
      w = w / 2 < 4 ? 4 : w / 2;
      h = h / 2 < 4 ? 4 : h / 2;
    }
    views[k].blocks = L.blocks + off;
    views[k].w = w;
    views[k].h = h;
    views[k].wb = w / 4;
    views[k].shift = L.shift;
#ifdef NBTC_CHECKED
    views[k].status = nullptr;
    views[k].plant = 0;
#endif
  }
  return NBTC_OK;
}

void attach_checks(const nbtc_context* ctx, LevelView* views, int n) {
#ifdef NBTC_CHECKED
  for (int k = 0; k < n; ++k) {
    views[k].status = ctx->status_dev;
    views[k].plant = ctx->check_plant;
  }
#else
  (void)ctx;
  (void)views;
  (void)n;
#endif
}

}  // namespace nbtc

using namespace nbtc;

extern "C" {

nbtc_status nbtc_create(int device, nbtc_context** out) {
  if (!out) return fail(NBTC_ERR_INVALID_ARG, "ctx out-pointer is NULL");
  *out = nullptr;
  int count = 0;
  nbtc_status st = cuda_check(cudaGetDeviceCount(&count), "cudaGetDeviceCount");
  if (st) return st;
  if (device < 0 || device >= count) return fail(NBTC_ERR_INVALID_ARG, "no such device");
  cudaDeviceProp prop;
  if ((st = cuda_check(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties"))) return st;
  if (prop.major != 10 || prop.minor != 3)
    return fail(NBTC_ERR_UNSUPPORTED, "this library is built for sm_103a (compute capability 10.3)");
  if ((st = cuda_check(cudaSetDevice(device), "cudaSetDevice"))) return st;
  nbtc_context* ctx = new nbtc_context();
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  if (const char* e = getenv("NBTC_TC_GROUPS")) ctx->tc_groups = atoi(e) == 3 ? 3 : 4;
  if (const char* e = getenv("NBTC_TC_TMEM_A")) ctx->tc_tmem_a = atoi(e) == 0 ? 0 : 1;
  if (const char* e = getenv("NBTC_FP32_GROUPS")) ctx->fp32_groups = atoi(e) == 1 ? 1 : 2;
  if (const char* e = getenv("NBTC_TRAIN_SIMT")) ctx->train_tc = atoi(e) == 1 ? 0 : 1;
  if ((st = cuda_check(cudaMalloc(&ctx->status_dev, sizeof(int)), "cudaMalloc(status)"))) {
    delete ctx;
    return st;
  }
  if ((st = cuda_check(cudaMemset(ctx->status_dev, 0, sizeof(int)), "cudaMemset(status)"))) {
    cudaFree(ctx->status_dev);
    delete ctx;
    return st;
  }
  *out = ctx;
  return NBTC_OK;
}

nbtc_status nbtc_destroy(nbtc_context* ctx) {
  if (!ctx) return NBTC_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->status_dev);
  delete ctx;
  return NBTC_OK;
}

nbtc_status nbtc_status_sync(nbtc_context* ctx, void* stream) {
  nbtc_status st = enter(ctx);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize"))) return st;
  int code = 0;
  if ((st = cuda_check(cudaMemcpy(&code, ctx->status_dev, sizeof(int), cudaMemcpyDeviceToHost),
                       "read status")))
    return st;
  if (code) {
    cudaMemset(ctx->status_dev, 0, sizeof(int));
    return fail((nbtc_status)code, std::string("device reported: ") + nbtc_status_string((nbtc_status)code));
  }
  return NBTC_OK;
}

const char* nbtc_status_string(nbtc_status s) {
  switch (s) {
    case NBTC_OK: return "ok";
    case NBTC_ERR_INVALID_ARG: return "invalid argument";
    case NBTC_ERR_UNSUPPORTED: return "unsupported";
    case NBTC_ERR_CUDA: return "CUDA error";
    case NBTC_ERR_TIMEOUT: return "device wait timed out";
    case NBTC_ERR_BOUNDS: return "index out of bounds";
  }
  return "unknown status";
}

const char* nbtc_last_error(void) { return g_last_error.c_str(); }

nbtc_status nbtc_set_check_plant(nbtc_context* ctx, int32_t offset) {
  if (!ctx) return fail(NBTC_ERR_INVALID_ARG, "ctx is NULL");
#ifdef NBTC_CHECKED
  ctx->check_plant = offset;
  return NBTC_OK;
#else
  (void)offset;
  return fail(NBTC_ERR_UNSUPPORTED, "bounds checks exist only in the checked build (libnbtc_checked.so)");
#endif
}

nbtc_status nbtc_set_wait_budget(nbtc_context* ctx, int64_t spins) {
  if (!ctx) return fail(NBTC_ERR_INVALID_ARG, "context is NULL");
  if (spins < -1) return fail(NBTC_ERR_INVALID_ARG, "spins must be >= -1");
  ctx->wait_budget = spins;
  return NBTC_OK;
}

nbtc_status nbtc_bc1_decode_level(nbtc_context* ctx, const nbtc_level* level, int32_t mip,
                                  uint8_t* out_dev, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if (!level || !out_dev) return fail(NBTC_ERR_INVALID_ARG, "level or out is NULL");
  nbtc_latents lat;
  memset(&lat, 0, sizeof(lat));
  lat.num_levels = 1;
  lat.address = NBTC_CLAMP;
  lat.levels[0] = *level;
  LevelView v;
  if ((st = make_level_views(&lat, mip, &v))) return st;
  attach_checks(ctx, &v, 1);
  if ((st = need_inputs(&lat, nullptr)) || (st = need_readable(out_dev, "out"))) return st;
  return launch_bc1_decode(ctx, v, out_dev, (cudaStream_t)stream);
}

static nbtc_status make_decode_args(nbtc_context* ctx, const nbtc_latents* lat, const nbtc_mlp* mlp,
                                    const float* uv, int64_t n, int32_t grid_w, int32_t grid_h,
                                    void* out, DecodeArgs& a, bool need_out = true) {
  nbtc_status st;
  memset(&a, 0, sizeof(a));
  if ((st = check_mlp(mlp))) return st;
  if (!lat) return fail(NBTC_ERR_INVALID_ARG, "latents is NULL");
  if (lat->num_levels != 4) return fail(NBTC_ERR_UNSUPPORTED, "decode kernels take 4 latent levels");
  if (mlp->dims[0] != 3 * lat->num_levels)
    return fail(NBTC_ERR_INVALID_ARG, "mlp.dims[0] must be 3 * num_levels");
  if ((st = make_level_views(lat, 0, a.lv))) return st;
  attach_checks(ctx, a.lv, 4);
  if (n < 0) return fail(NBTC_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NBTC_OK;  // nothing to decode; no pointer is touched
  if ((st = need_inputs(lat, mlp))) return st;
  if (uv && (st = need_readable(uv, "uv"))) return st;
  if (!uv) {
    if (grid_w <= 0 || grid_h <= 0 || (int64_t)grid_w * grid_h != n)
      return fail(NBTC_ERR_INVALID_ARG, "grid mode needs n == grid_w * grid_h > 0");
    if (grid_w > (1 << 20) || grid_h > (1 << 20)) return fail(NBTC_ERR_INVALID_ARG, "grid too large");
  } else if (!aligned(uv, 8)) {
    return fail(NBTC_ERR_INVALID_ARG, "uv not 8-byte aligned");
  }
  if (need_out && !out) return fail(NBTC_ERR_INVALID_ARG, "out is NULL");
  if (out && !aligned(out, 16)) return fail(NBTC_ERR_INVALID_ARG, "out not 16-byte aligned");
  a.wrap = lat->address == NBTC_WRAP;
  a.uv = uv;
  a.n = n;
  a.grid_w = grid_w;
  a.grid_h = grid_h;
  a.cw = make_grid_coord(uv ? 1 : grid_w);
  a.ch = make_grid_coord(uv ? 1 : grid_h);
  a.out = out;
  a.status = ctx->status_dev;
  return NBTC_OK;
}

nbtc_status nbtc_fp8_calibrate(nbtc_context* ctx, const nbtc_latents* lat, const nbtc_mlp* mlp,
                               int32_t grid_w, int32_t grid_h, int32_t step, float* act_absmax_dev,
                               void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if (step < 1) return fail(NBTC_ERR_INVALID_ARG, "step must be >= 1");
  if (!act_absmax_dev) return fail(NBTC_ERR_INVALID_ARG, "act_absmax is NULL");
  if ((st = need_device(act_absmax_dev, "act_absmax"))) return st;
  DecodeArgs a;
  if ((st = make_decode_args(ctx, lat, mlp, nullptr, (int64_t)grid_w * grid_h, grid_w, grid_h, nullptr, a,
                             /*need_out=*/false)))
    return st;
  return launch_calibrate_fp32(ctx, a, mlp, step, act_absmax_dev, (cudaStream_t)stream);
}

// Where a decode may write: device (or managed) memory, or -- FP32 decodes,
// whose kernels store with plain global stores -- pinned host memory, which the
// kernel writes directly over the host link (its device address replaces out).
static nbtc_status resolve_out(int32_t precision, DecodeArgs& a) {
  cudaPointerAttributes pa;
  const cudaError_t e = cudaPointerGetAttributes(&pa, a.out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(NBTC_ERR_INVALID_ARG, "out is not a pointer CUDA knows");
  }
  if (pa.type == cudaMemoryTypeManaged) return NBTC_OK;
  if (pa.type == cudaMemoryTypeDevice) {
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && pa.device == dev) return NBTC_OK;
    return fail(NBTC_ERR_INVALID_ARG, "out is device memory of another GPU");
  }
  if (pa.type == cudaMemoryTypeHost && pa.devicePointer) {
    if (precision != NBTC_FP32)
      return fail(NBTC_ERR_UNSUPPORTED,
                  "pinned host output is for the FP32 SIMT decode; tensor-core forms decode into device memory");
    a.out = pa.devicePointer;
    if (!aligned(a.out, 16)) return fail(NBTC_ERR_INVALID_ARG, "out not 16-byte aligned");
    return NBTC_OK;
  }
  return fail(NBTC_ERR_INVALID_ARG, "out is neither device memory nor pinned host memory");
}

nbtc_status nbtc_decode(nbtc_context* ctx, const nbtc_latents* lat, const nbtc_mlp* mlp, int32_t precision,
                        const void* packed_dev, const float* uv_dev, int64_t n, int32_t grid_w,
                        int32_t grid_h, void* out_dev, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  DecodeArgs a;
  if ((st = make_decode_args(ctx, lat, mlp, uv_dev, n, grid_w, grid_h, out_dev, a))) return st;
  if (n == 0) return NBTC_OK;
  if ((st = resolve_out(precision, a))) return st;
  switch (precision) {
    case NBTC_FP32:
      return launch_decode_fp32(ctx, a, mlp, (cudaStream_t)stream);
    case NBTC_FP16:
    case NBTC_FP8_E4M3:
    case NBTC_FP16_SPLIT:
    case NBTC_FP8_E4M3_SPLIT:
    case NBTC_FP32_TC:
      if ((st = need_device(packed_dev, "packed MLP"))) return st;
      return launch_decode_tc(ctx, a, mlp, precision, packed_dev, (cudaStream_t)stream);
    default:
      return fail(NBTC_ERR_INVALID_ARG, "unknown precision");
  }
}

nbtc_status nbtc_decode_rows(nbtc_context* ctx, const nbtc_latents* lat, const nbtc_mlp* mlp, int32_t precision,
                             const void* packed_dev, int32_t grid_w, int32_t grid_h, int32_t row0, int32_t rows,
                             void* out_dev, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if (grid_h <= 0 || row0 < 0 || rows < 0 || row0 > grid_h || rows > grid_h - row0)
    return fail(NBTC_ERR_INVALID_ARG, "row range outside the grid");
  DecodeArgs a;
  if ((st = make_decode_args(ctx, lat, mlp, nullptr, (int64_t)grid_w * rows, grid_w, rows, out_dev, a))) return st;
  if (rows == 0) return NBTC_OK;
  if ((st = resolve_out(precision, a))) return st;
  a.row0 = row0;
  a.ch = make_grid_coord(grid_h);
  switch (precision) {
    case NBTC_FP32:
      return launch_decode_fp32(ctx, a, mlp, (cudaStream_t)stream);
    case NBTC_FP16:
    case NBTC_FP8_E4M3:
    case NBTC_FP16_SPLIT:
    case NBTC_FP8_E4M3_SPLIT:
    case NBTC_FP32_TC:
      if ((st = need_device(packed_dev, "packed MLP"))) return st;
      return launch_decode_tc(ctx, a, mlp, precision, packed_dev, (cudaStream_t)stream);
    default:
      return fail(NBTC_ERR_INVALID_ARG, "unknown precision");
  }
}

nbtc_status nbtc_packed_mlp_bytes(const nbtc_mlp* mlp, int32_t precision, size_t* bytes) {
  nbtc_status st = check_mlp(mlp);
  if (st) return st;
  if (!bytes) return fail(NBTC_ERR_INVALID_ARG, "bytes is NULL");
  if (precision == NBTC_FP32) {
    *bytes = 0;
    return NBTC_OK;
  }
  if (precision < NBTC_FP16 || precision > NBTC_FP32_TC) return fail(NBTC_ERR_INVALID_ARG, "unknown precision");
  return tc_packed_bytes(mlp, precision, bytes);
}

nbtc_status nbtc_pack_mlp(nbtc_context* ctx, const nbtc_mlp* mlp, int32_t precision,
                          const float* act_absmax_dev, void* packed_dev, size_t packed_bytes,
                          void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if ((st = check_mlp(mlp))) return st;
  if (precision < NBTC_FP16 || precision > NBTC_FP32_TC)
    return fail(NBTC_ERR_INVALID_ARG, "pack_mlp takes a tensor-core precision");
  // the packed image is later bulk-copied into shared memory: device memory only
  if ((st = need_inputs(nullptr, mlp)) || (st = need_device(packed_dev, "packed MLP"))) return st;
  if (act_absmax_dev && (st = need_readable(act_absmax_dev, "act_absmax"))) return st;
  return launch_pack_mlp(ctx, mlp, precision, act_absmax_dev, packed_dev, packed_bytes, (cudaStream_t)stream);
}

nbtc_status nbtc_train_workspace_bytes(nbtc_context* ctx, const nbtc_train_args* args, size_t* bytes) {
  if (!ctx || !args || !bytes) return fail(NBTC_ERR_INVALID_ARG, "NULL argument");
  *bytes = train_workspace(ctx, args);
  return NBTC_OK;
}

nbtc_status nbtc_train_step(nbtc_context* ctx, const nbtc_train_args* args, float* loss_dev, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if (!args) return fail(NBTC_ERR_INVALID_ARG, "args NULL");
  return train_step_impl(ctx, args, loss_dev, (cudaStream_t)stream, 2, nullptr, nullptr, args->workspace,
                         args->workspace_bytes);
}

nbtc_status nbtc_qat_decode(nbtc_context* ctx, const nbtc_qat_level* level, float* out, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  return qat_decode(ctx, level, out, (cudaStream_t)stream);
}

nbtc_status nbtc_qat_encode(nbtc_context* ctx, const nbtc_qat_level* level, uint64_t* blocks, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  return qat_encode(ctx, level, blocks, (cudaStream_t)stream);
}

nbtc_status nbtc_train_step_qat(nbtc_context* ctx, const nbtc_train_args* args, const nbtc_qat_level* levels,
                                float* loss_dev, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  return train_step_qat(ctx, args, levels, loss_dev, (cudaStream_t)stream);
}

nbtc_status nbtc_forward_continuous(nbtc_context* ctx, const nbtc_train_args* args, float* y_dev, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if (!args) return fail(NBTC_ERR_INVALID_ARG, "args NULL");
  return train_step_impl(ctx, args, nullptr, (cudaStream_t)stream, 0, nullptr, y_dev, nullptr, 0);
}

nbtc_status nbtc_backward_continuous(nbtc_context* ctx, const nbtc_train_args* args, const float* dy_dev,
                                     void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if (!args) return fail(NBTC_ERR_INVALID_ARG, "args NULL");
  return train_step_impl(ctx, args, nullptr, (cudaStream_t)stream, 1, dy_dev, nullptr, args->workspace,
                         args->workspace_bytes);
}

}  // extern "C"
