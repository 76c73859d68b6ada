// Host-side internals shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "common.cuh"

struct nbtc_context {
  int device = 0;
  int sm_count = 0;
  int* status_dev = nullptr;       // device status word (first recorded fault)
  long long wait_budget = 0;       // spins per bounded device wait (0 = default, -1 = give up at once)
  int tc_groups = 4;               // warpgroups per CTA of the tensor-core decode (3 or 4)
  int tc_tmem_a = 1;               // MMA A operands in TMEM (one slot per warpgroup; 0: shared memory)
  int fp32_groups = 2;             // independent thread groups per CTA of the FP32 wide decode (1 or 2)
  int check_plant = 0;             // checked build, tests only: offset added to gather indices
  int train_tc = 1;                // training steps with pre-gathered samples on tensor cores (0: SIMT)
};

#include <nvtx3/nvToolsExt.h>

namespace nbtc {

// Names a C-ABI call in profiler timelines: an NVTX range for the call's
// duration on the host (nothing happens unless a profiler is attached).
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
  CallRange(const CallRange&) = delete;
  CallRange& operator=(const CallRange&) = delete;
};
#define NBTC_RANGE() ::nbtc::CallRange nbtc_call_range_(__func__)


// Records `msg` as the calling thread's last error and returns `code`.
nbtc_status fail(nbtc_status code, const std::string& msg);
// Wraps a CUDA runtime result: NBTC_OK, or NBTC_ERR_CUDA with the CUDA message.
nbtc_status cuda_check(cudaError_t err, const char* what);

// Makes ctx->device current for the rest of the call.
nbtc_status enter(nbtc_context* ctx);

// Validates a latent pyramid for the decode kernels and fills the device
// views of mip `mip` of each level.
nbtc_status make_level_views(const nbtc_latents* lat, int mip, LevelView* views);

// Checked build: points the views' bounds checks at the context's status word
// (and its test-only index offset); no-op otherwise.
void attach_checks(const nbtc_context* ctx, LevelView* views, int n);

// Validates an MLP descriptor (shape and pointers).
nbtc_status check_mlp(const nbtc_mlp* mlp);

constexpr long long kDefaultWaitBudget = 1ll << 22;  // polls of up to 1 us: a few seconds

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Kernel launchers (one per translation unit).
nbtc_status launch_bc1_decode(nbtc_context* ctx, const LevelView& v, uint8_t* out, cudaStream_t s);
nbtc_status launch_decode_fp32(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp,
                               cudaStream_t s);
nbtc_status tc_packed_bytes(const nbtc_mlp* mlp, int precision, size_t* bytes);
nbtc_status launch_pack_mlp(nbtc_context* ctx, const nbtc_mlp* mlp, int precision, const float* act_absmax,
                            void* packed, size_t packed_bytes, cudaStream_t s);
nbtc_status launch_decode_tc(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp, int precision,
                             const void* packed, cudaStream_t s);
size_t train_workspace(nbtc_context* ctx, const nbtc_train_args* A);
// mode: 0 forward (y), 1 backward from dy, 2 full step (loss, grads, Adam), 3 full step
// without the latent Adam (latent gradients only)
nbtc_status train_step_impl(nbtc_context* ctx, const nbtc_train_args* A, float* loss, cudaStream_t s, int mode,
                            const float* dy, float* y, void* workspace, size_t workspace_bytes);
// QAT BC1 latents (qat.cu).
nbtc_status qat_decode(nbtc_context* ctx, const nbtc_qat_level* q, float* out, cudaStream_t s);
nbtc_status qat_encode(nbtc_context* ctx, const nbtc_qat_level* q, uint64_t* blocks, cudaStream_t s);
nbtc_status train_step_qat(nbtc_context* ctx, const nbtc_train_args* A, const nbtc_qat_level* levels, float* loss,
                           cudaStream_t s);
// Floats per latent texel of a training call (3 or 4), 0 when the stride is invalid.
int latent_stride(const nbtc_train_args* A);
// Pointer kinds the kernels can use: device (or managed) memory, or pinned host
// memory reached over the host link (plain loads and stores only, no bulk copies).
enum PtrKind { kPtrDevice, kPtrPinned, kPtrOther };
PtrKind ptr_kind(const void* p);
nbtc_status need_readable(const void* p, const char* what);  // device or pinned host
nbtc_status need_device(const void* p, const char* what);    // device (or managed) only
nbtc_status need_inputs(const nbtc_latents* lat, const nbtc_mlp* mlp);  // every level's blocks, weights, biases
// One Adam update (the step's betas, eps and step number; learning rate lr) of
// up to 12 parameter arrays of n[i] floats each, in one launch.
struct AdamSeg {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t n;
};
struct AdamSegs {
  AdamSeg seg[12];
  int count;  // <= 12
};
nbtc_status launch_adam(nbtc_context* ctx, const nbtc_train_args* A, float lr, const AdamSegs& S, cudaStream_t s);
nbtc_status launch_calibrate_fp32(nbtc_context* ctx, const DecodeArgs& a, const nbtc_mlp* mlp,
                                  int step, float* absmax, cudaStream_t s);

}  // namespace nbtc
