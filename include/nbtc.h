/*
 * nbtc.h -- C ABI of the GB300 neural block texture decoder.
 *
 * The method ("Hardware Accelerated Neural Block Texture Compression with
 * Cooperative Vectors", arXiv 2506.06040) stores a material as L latent
 * textures in BC1 format (Sec. 3.1, "Latent BC1 compression") and decodes the
 * texel at uv by sampling each latent level, concatenating the features and
 * running a small ReLU MLP that outputs the material channels (Sec. 3.1,
 * "Network Architecture").  This library runs that decode, its training step
 * on continuous latents (Sec. 3.2) and the multi-material tile pipeline of
 * Sec. 4 as CUDA kernels for sm_103a.
 *
 * Conventions shared by every entry point
 *  - Pointers named *_dev, and every pointer inside the descriptor structs,
 *    are device pointers.  All buffers belong to the caller; the library never
 *    frees them and keeps no reference after the call's work has run.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Every call is asynchronous and stream-ordered unless it says
 *    otherwise.
 *  - Synchronous argument checks return NBTC_ERR_INVALID_ARG or
 *    NBTC_ERR_UNSUPPORTED before anything is enqueued; a failed launch returns
 *    NBTC_ERR_CUDA.  Faults the kernels detect themselves (a bounded wait that
 *    ran out, an index outside its buffer in a checked build) are written to
 *    the context's device status word and reported by nbtc_status_sync().
 *    nbtc_last_error() gives a human-readable message for the calling thread.
 *  - Texel (x, y) of a W x H image is element y * W + x (row-major); u runs
 *    along x, v along y, origin at the top-left corner, texel centres at
 *    half-integers (texel coordinate x = u * W - 0.5 + shift).
 *  - Outputs are texel-major: N contiguous channels per texel.
 *  - A context is used by one host thread at a time.
 */
#ifndef NBTC_H
#define NBTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NBTC_MAX_LEVELS 8
#define NBTC_MAX_LAYERS 4
#define NBTC_MAX_MIPS 16

typedef enum {
  NBTC_OK = 0,
  NBTC_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or descriptor   */
  NBTC_ERR_UNSUPPORTED = 2, /* valid request the library has no kernel for */
  NBTC_ERR_CUDA = 3,        /* a CUDA runtime call failed                    */
  NBTC_ERR_TIMEOUT = 4,     /* a device-side bounded wait expired            */
  NBTC_ERR_BOUNDS = 5       /* checked build: a gather index outside its array */
} nbtc_status;

/* Precision forms of the decode (Sec. 4 runs the MLP on matrix units in low
 * precision).  The split forms carry every weight and activation as a pair
 * hi + lo of the narrow format (FP16: hi = RN16(v), lo = RN16(v - hi); E4M3:
 * v16 = RN16(v / scale), hi = E4M3(v16), lo = E4M3(v16 - hi)) and sum the three
 * products hi(A) hi(W) + lo(A) hi(W) + hi(A) lo(W) per layer in one FP32
 * accumulator: every multiply still reads the narrow format, at three times
 * the tensor work, and the result keeps most of the precision the single
 * rounding loses (max abs error vs FP64 on a He-initialised 12-64-64-64-9
 * decode: FP16 3.2e-3 -> 9.8e-4, the FP16 output rounding; E4M3 0.37 -> 1.2e-2;
 * before the output rounding the FP16 split is within ~1e-6, which NBTC_FP32_TC
 * keeps by writing FP32). */
typedef enum {
  NBTC_FP32 = 0,            /* FP32 SIMT arithmetic (FFMA), FP32 output              */
  NBTC_FP16 = 1,            /* FP16 operands on tcgen05, FP32 accumulate, FP16 output */
  NBTC_FP8_E4M3 = 2,        /* E4M3 operands on tcgen05 with per-layer power-of-two
                               scales, FP32 accumulate, FP16 output                   */
  NBTC_FP16_SPLIT = 3,      /* split FP16 operands, otherwise as NBTC_FP16            */
  NBTC_FP8_E4M3_SPLIT = 4,  /* split E4M3 operands, otherwise as NBTC_FP8_E4M3        */
  NBTC_FP32_TC = 5          /* split FP16 operands on tcgen05 as NBTC_FP16_SPLIT, the
                               FP32 accumulator written as FP32 output (no FP16
                               rounding): FP32-form accuracy on tensor cores       */
} nbtc_precision;

typedef enum { NBTC_CLAMP = 0, NBTC_WRAP = 1 } nbtc_address;

typedef enum { NBTC_LOSS_MSE = 0, NBTC_LOSS_L1 = 1 } nbtc_loss;

/* One BC1 latent texture T_k (Sec. 3.1).  `blocks` holds mip 0 then mips
 * 1 .. num_mips-1 back to back; mip m is max(4, width>>m) x max(4, height>>m)
 * texels, each mip a row-major array of 8-byte BC1 blocks (block (bx, by) at
 * by * (w_m / 4) + bx).  Block bits 0-15 hold endpoint c0, 16-31 endpoint c1
 * (RGB565), 32-63 the sixteen 2-bit indices, texel (tx, ty) at bit
 * 2 * (4 ty + tx).  `shift` offsets the sample position by that many texels on
 * both axes (the paper shifts the 2nd and 4th latent by half a texel). */
typedef struct {
  const uint64_t* blocks;
  int32_t width;    /* mip-0 texels, multiple of 4, >= 4 */
  int32_t height;   /* mip-0 texels, multiple of 4, >= 4 */
  int32_t num_mips; /* 1 .. NBTC_MAX_MIPS */
  float shift;
} nbtc_level;

/* The latent pyramid of one material: features are ordered
 * [T_0.rgb, T_1.rgb, ...]; `address` is an nbtc_address. */
typedef struct {
  int32_t num_levels; /* 1 .. NBTC_MAX_LEVELS (the fast kernels: 4) */
  int32_t address;
  nbtc_level levels[NBTC_MAX_LEVELS];
} nbtc_latents;

/* ReLU MLP f(x) (Sec. 3.1): num_layers linear layers, ReLU after all but the
 * last.  Layer l maps dims[l] -> dims[l+1]; its weight is row-major
 * [dims[l+1]][dims[l]] (out x in) and the layers are stored back to back in
 * `weights`; `biases` likewise.  FP32, device memory. */
typedef struct {
  int32_t num_layers; /* 2 .. NBTC_MAX_LAYERS */
  int32_t dims[NBTC_MAX_LAYERS + 1];
  const float* weights;
  const float* biases;
} nbtc_mlp;

typedef struct nbtc_context nbtc_context;

/* ------------------------------------------------------------------ context */

/* Creates a context on CUDA device `device` (made current for the call).  The
 * context owns a 4-byte device status word and nothing else per device.
 * Returns NBTC_ERR_INVALID_ARG for a NULL `ctx`, NBTC_ERR_UNSUPPORTED when the
 * device is not compute capability 10.3, NBTC_ERR_CUDA when CUDA fails.
 * Environment variables, read here, select kernel variants for measurement
 * (decode results are bit-identical either way): NBTC_TC_TMEM_A=0 keeps the
 * MMA A operands of the tensor-core forms (FP16, FP8_E4M3, both split forms, FP32_TC) in
 * shared memory instead of tensor memory; NBTC_TC_GROUPS=3 runs the
 * shared-memory-operand FP16 / FP8 decodes with 3 warpgroups per CTA instead of
 * 4; NBTC_FP32_GROUPS=1 runs the FP32 wide decode as one 512-thread group per
 * CTA instead of two independent 256-thread groups; NBTC_TRAIN_SIMT=1 runs
 * every training step on the FP32 SIMT kernel (default: the tensor-core kernel
 * whenever the workspace holds the gathered samples; results agree to FP32
 * rounding, not bit for bit). */
nbtc_status nbtc_create(int device, nbtc_context** ctx);

/* Frees the context (synchronises the device first).  NULL is accepted. */
nbtc_status nbtc_destroy(nbtc_context* ctx);

/* Waits for `stream`, then returns and clears the device status word: NBTC_OK
 * or the first fault a kernel recorded since the last call (TIMEOUT, BOUNDS). */
nbtc_status nbtc_status_sync(nbtc_context* ctx, void* stream);

/* Static description of a status code. */
const char* nbtc_status_string(nbtc_status s);

/* Message describing the last non-OK return on the calling thread ("" if none). */
const char* nbtc_last_error(void);

/* Tests only: caps the device-side bounded waits of this context's decode
 * loops at `spins` polls (0 restores the default budget; -1 makes every such
 * wait exceed it at once).  A wait past its budget records NBTC_ERR_TIMEOUT in
 * the status word (the launch's results are void) and then keeps waiting with
 * a fixed budget (2^22 polls of <= 1 us), so the kernel's hand-offs stay in
 * step and it releases its resources only after its own tensor-core work and
 * bulk copies have finished; the context stays usable.  Waits that guard
 * resources (weight loads, the final drain) always use the fixed budget. */
nbtc_status nbtc_set_wait_budget(nbtc_context* ctx, int64_t spins);

/* Checked build.  libnbtc_checked.so is this library compiled with
 * NBTC_CHECKED: every gather index its kernels form (BC1 blocks of every level
 * and mip, latent and target taps of the training kernels, frame pixels and
 * the binning's list slots) is tested against the extent of the array it
 * indexes; an index outside it records NBTC_ERR_BOUNDS in the context's status
 * word (reported by nbtc_status_sync) and is replaced by 0, so no access leaves
 * its array and nothing traps.  Results are otherwise those of libnbtc.so.
 * Tests only: nbtc_set_check_plant adds `offset` to every such index of this
 * context's later calls (0 restores), so the checks can be seen to fire; the
 * default build returns NBTC_ERR_UNSUPPORTED. */
nbtc_status nbtc_set_check_plant(nbtc_context* ctx, int32_t offset);

/* ------------------------------------------------------------------ decode */

/* BC1 decode of one mip of one latent level to RGB8 (Sec. 3.1 with the BC1
 * format definition the paper cites; integer, bit-exact): out_dev receives
 * h_m x w_m x 3 bytes, row-major.  Rounding: channels expand to 8 bits by bit
 * replication; when c0 > c1 (raw 16-bit compare) the palette is
 * {c0, c1, (2 c0 + c1 + 1) / 3, (c0 + 2 c1 + 1) / 3}, otherwise
 * {c0, c1, (c0 + c1 + 1) / 2, black}, integer division, per channel. */
nbtc_status nbtc_bc1_decode_level(nbtc_context* ctx, const nbtc_level* level, int32_t mip,
                                  uint8_t* out_dev, void* stream);

/* Bytes nbtc_pack_mlp() writes for `mlp` in `precision` (0 for NBTC_FP32,
 * which reads the FP32 weights directly). */
nbtc_status nbtc_packed_mlp_bytes(const nbtc_mlp* mlp, int32_t precision, size_t* bytes);

/* Lays the MLP out for the tensor-core forms: weights converted to FP16 or
 * E4M3 (round to nearest even, E4M3 saturating; the split forms store hi and
 * lo) in the shared-memory image the decode kernel copies in one bulk
 * transfer, plus FP32 biases and scales.
 * For NBTC_FP8_E4M3 and NBTC_FP8_E4M3_SPLIT `act_absmax_dev` must hold, per layer, the largest
 * magnitude of that layer's input over a calibration set (nbtc_fp8_calibrate);
 * the layer scales are then sw_l = pow2ceil(absmax(W_l) / 448) and
 * sa_l = pow2ceil(act_absmax_l / 448).  `packed_dev` must be 16-byte aligned
 * and at least nbtc_packed_mlp_bytes() long. */
nbtc_status nbtc_pack_mlp(nbtc_context* ctx, const nbtc_mlp* mlp, int32_t precision,
                          const float* act_absmax_dev, void* packed_dev, size_t packed_bytes,
                          void* stream);

/* FP8 calibration: runs the FP32 decode on the texel-centre sub-grid of every
 * `step`-th texel in x and y of a grid_w x grid_h output and writes, per layer
 * l, max |input of layer l| to act_absmax_dev[l] (num_layers floats). */
nbtc_status nbtc_fp8_calibrate(nbtc_context* ctx, const nbtc_latents* lat, const nbtc_mlp* mlp,
                               int32_t grid_w, int32_t grid_h, int32_t step,
                               float* act_absmax_dev, void* stream);

/* Neural decode (Sec. 3.1): for each output texel, BC1 fetch + decode of
 * every latent level, bilinear sample at uv (level shift, clamp or wrap),
 * concatenation, MLP.
 *  - uv_dev == NULL: grid mode, n == grid_w * grid_h texel-centre outputs,
 *    u = (i + 0.5) / grid_w, v = (j + 0.5) / grid_h, row-major.
 *  - uv_dev != NULL: n (u, v) FP32 pairs, interleaved; grid_w, grid_h ignored.
 *  - precision NBTC_FP32: `packed_dev` NULL, `out_dev` n x N FP32.
 *    NBTC_FP16 / NBTC_FP8_E4M3 / NBTC_FP16_SPLIT / NBTC_FP8_E4M3_SPLIT:
 *    `packed_dev` from nbtc_pack_mlp() with the same precision, `out_dev`
 *    n x N FP16.  NBTC_FP32_TC: `packed_dev` from nbtc_pack_mlp() with
 *    NBTC_FP32_TC, `out_dev` n x N FP32.  out_dev 16-byte aligned.
 *  - Inputs (level blocks, MLP weights and biases, uv_dev) are device memory or
 *    pinned host memory (read over the host link); packed_dev is device memory
 *    (it is bulk-copied into shared memory); anything else is
 *    NBTC_ERR_INVALID_ARG, checked before any launch.
 *  - out_dev is device memory or, for NBTC_FP32 only, pinned host memory
 *    (cudaHostAlloc / cudaHostRegister): the kernel then stores the texels
 *    straight into host memory over the host link, with no staging buffer or
 *    copy; completion is the stream's.  Pinned host output with a tensor-core
 *    precision (NBTC_FP32_TC included) is NBTC_ERR_UNSUPPORTED (their kernels store with bulk
 *    copies, kept to device memory); any other pointer (pageable host memory)
 *    is NBTC_ERR_INVALID_ARG.
 * Shapes with a kernel: 4 latent levels, hidden width 16, 32 or 64 (all
 * hidden layers equal), 1-3 hidden layers, N <= 16 (the tensor-core forms run
 * widths 16 and 32 zero-padded to 64). */
nbtc_status nbtc_decode(nbtc_context* ctx, const nbtc_latents* lat, const nbtc_mlp* mlp,
                        int32_t precision, const void* packed_dev, const float* uv_dev,
                        int64_t n, int32_t grid_w, int32_t grid_h, void* out_dev, void* stream);

/* Grid-mode decode of rows [row0, row0 + rows) of a grid_w x grid_h texel-centre
 * grid (u = (i + 0.5) / grid_w, v = (row0 + j + 0.5) / grid_h) into out_dev,
 * rows x grid_w x N (row-major): the same values nbtc_decode writes for those
 * rows of the whole grid.  Lets a caller stream a large decode in row bands
 * (e.g. overlapping each band's device-to-host copy with the next band's decode).
 * out_dev follows nbtc_decode's rules. */
nbtc_status nbtc_decode_rows(nbtc_context* ctx, const nbtc_latents* lat, const nbtc_mlp* mlp, int32_t precision,
                             const void* packed_dev, int32_t grid_w, int32_t grid_h, int32_t row0, int32_t rows,
                             void* out_dev, void* stream);

/* ------------------------------------------------------------------ training
 *
 * One optimisation step of the decoder on continuous latents (Sec. 3.2: the
 * compressor's texture-unit replica, gradients through the MLP into every
 * latent texel, Adam with lr 1e-3 for the MLP and 1e-2 for the latents).  The
 * latents here are plain FP32 textures (before BC1 quantisation): level k is
 * latents[k] = [heights[k]][widths[k]][latent_stride], channels 0..2 used,
 * sampled bilinearly with clamp addressing and the level's shift.  The MLP is
 * [12, 64, 64, C] (C <= 16) in the nbtc_mlp layout.  The target is
 * [target_h][target_w][target_stride] FP32, channels 0..C-1 used, sampled
 * bilinearly (clamp, no shift) at the same uv.
 *
 * Layout: latent_stride 4 (a padding channel after RGB; latents and gradients
 * 16-byte aligned) lets the kernels fetch a texel and add its gradient with one
 * 16-byte access each instead of three 4-byte ones; the padding channel is read
 * but never used, its gradient stays 0 and Adam leaves it unchanged.  A
 * target_stride that is a multiple of 4 (16-byte aligned target) likewise reads
 * the target 16 bytes at a time; its padding channels are never used.  Loss: mean over batch and
 * channels of (y - t)^2 (NBTC_LOSS_MSE) or |y - t| (NBTC_LOSS_L1).
 *
 * Every array is device memory or pinned host memory (pageable host memory is
 * NBTC_ERR_INVALID_ARG, checked before any launch).
 *
 * Gradient sums over the batch use compensated (Neumaier) FP32 summation;
 * latent gradients are accumulated with FP32 atomics (their summation order
 * varies between runs).  Adam follows the PyTorch form with bias correction:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 */
typedef struct {
  int32_t num_levels;                       /* 4 */
  int32_t widths[NBTC_MAX_LEVELS], heights[NBTC_MAX_LEVELS];
  float shifts[NBTC_MAX_LEVELS];
  float* latents[NBTC_MAX_LEVELS];          /* updated in place by nbtc_train_step */
  float* latent_grads[NBTC_MAX_LEVELS];     /* overwritten with this batch's gradient */
  float* latent_m[NBTC_MAX_LEVELS];         /* Adam moments (train step only) */
  float* latent_v[NBTC_MAX_LEVELS];
  nbtc_mlp mlp;                             /* weights/biases updated in place by the step */
  float* grad_w;                            /* overwritten: same layout as mlp.weights */
  float* grad_b;                            /* overwritten: same layout as mlp.biases */
  float* m_w; float* v_w; float* m_b; float* v_b;   /* Adam moments of the MLP */
  const float* target;                      /* [target_h][target_w][C] (train step only) */
  int32_t target_w, target_h;
  const float* uv;                          /* [batch][2] */
  int64_t batch;
  int32_t step;                             /* Adam step number t of this update, >= 1 */
  float lr_mlp, lr_latent, beta1, beta2, eps;
  int32_t loss;                             /* nbtc_loss */
  void* workspace;                          /* caller-owned scratch, 16-byte aligned */
  size_t workspace_bytes;                   /* >= nbtc_train_workspace_bytes() */
  int32_t latent_stride;                    /* floats per texel of latents, latent_grads, latent_m,
                                               latent_v: 3 or 4 (0 means 3) */
  int32_t target_stride;                    /* floats per target texel, >= C (0 means C) */
} nbtc_train_args;

/* Scratch bytes the training calls need on this context's device: the per-CTA
 * partial sums and one record of 12 + 4 ceil(C / 4) floats per sample, into
 * which the step first gathers every sample's features and target channels.  A
 * workspace with room for the partial sums only (one CTA per SM, 48,264 bytes
 * each) is accepted too: the step then gathers inside its main kernel (same
 * results, slower). */
nbtc_status nbtc_train_workspace_bytes(nbtc_context* ctx, const nbtc_train_args* args, size_t* bytes);

/* Forward + loss + backward + Adam (MLP and latents) for one batch.  Writes
 * the batch loss to loss_dev (one float), the gradients to grad_w / grad_b /
 * latent_grads, and updates parameters and moments in place. */
nbtc_status nbtc_train_step(nbtc_context* ctx, const nbtc_train_args* args, float* loss_dev, void* stream);

/* Forward only: y_dev[batch][C] = f(latents sampled at uv). */
nbtc_status nbtc_forward_continuous(nbtc_context* ctx, const nbtc_train_args* args, float* y_dev, void* stream);

/* Backward only, from a given dL/dy (dy_dev[batch][C]): writes grad_w, grad_b
 * and latent_grads (activations are recomputed, not stored); no update. */
nbtc_status nbtc_backward_continuous(nbtc_context* ctx, const nbtc_train_args* args, const float* dy_dev,
                                     void* stream);

/* ------------------------------------------------------------------ QAT BC1 latents
 *
 * Quantisation-aware training of the BC1 latents themselves (Sec. 3.2,
 * Eqs. 1-3): a level is held as raw FP32 parameters -- per 4x4 block two
 * endpoints e0, e1 (RGB), per texel a blend factor alpha -- and decodes to
 * T = (1 - a) E0 + a E1 with a = quant(sigmoid(alpha), 2 bits) and
 * E = quant(sigmoid(e), [5, 6, 5] bits); quant picks the nearest of the 2^b
 * levels k / (2^b - 1), decided as the number of FP32 thresholds
 * logit((j + 1/2) / (2^b - 1)) that the raw FP32 parameter reaches (no exp in
 * the decision).  The backward passes the quantisers' gradient straight through,
 * so dL/dalpha = sum_c dL/dT_c (E1_c - E0_c) s'(alpha) and dL/de0 = sum over the
 * block's texels of dL/dT (1 - a) s'(e0) (likewise e1 with a), s' = s (1 - s).
 * The encoder turns the parameters into real BC1 blocks: endpoint codes
 * R << 11 | G << 5 | B, level q of alpha mapped to palette index 0 (q = 0),
 * 2 (q = 1), 3 (q = 2), 1 (q = 3) in four-colour mode; endpoints swapped (and
 * q -> 3 - q) when code(e0) < code(e1); every index 0 when the codes are equal.
 * All arrays are device FP32, caller-owned, row-major. */
typedef struct {
  int32_t width, height;                   /* texels, positive multiples of 4 */
  float* e0; float* e1;                     /* [height/4][width/4][3] raw endpoints */
  float* alpha;                             /* [height][width] raw blend factors */
  float* g_e0; float* g_e1; float* g_alpha; /* gradients (written by the step) */
  float* m_e0; float* v_e0;                 /* Adam moments (step only) */
  float* m_e1; float* v_e1;
  float* m_alpha; float* v_alpha;
} nbtc_qat_level;

/* Decoded texture of one QAT level: out [height][width][3] FP32. */
nbtc_status nbtc_qat_decode(nbtc_context* ctx, const nbtc_qat_level* level, float* out, void* stream);

/* BC1 blocks of one QAT level: blocks [height/4][width/4] (uint64). */
nbtc_status nbtc_qat_encode(nbtc_context* ctx, const nbtc_qat_level* level, uint64_t* blocks, void* stream);

/* One QAT training step: decodes the 4 levels into args->latents (caller-owned
 * scratch of the decoded textures, sizes args->widths / heights, which must
 * equal the levels'), runs the training step of nbtc_train_step on them
 * (forward, loss, backward, MLP Adam; args->latent_grads receives dL/dT,
 * args->latent_m / latent_v are not used), carries dL/dT to the raw parameters
 * straight through the quantisers (g_e0, g_e1, g_alpha) and updates them with
 * Adam at args->lr_latent. */
nbtc_status nbtc_train_step_qat(nbtc_context* ctx, const nbtc_train_args* args, const nbtc_qat_level* levels,
                                float* loss_dev, void* stream);

/* ------------------------------------------------------------------ batching
 *
 * Many materials, each with its own BC1 pyramid (with mips) and its own MLP,
 * decoded in one persistent launch (Sec. 4: the G-buffer pass runs every
 * neural material of a frame; cooperative vectors need one matrix per
 * workgroup, so pixels are grouped per MLP).  A plan owns the device-side
 * material table, the packed FP16 MLPs, the work lists and two CUDA graphs.
 *
 * Full decode: every material with `out` set is decoded on its texel-centre
 * grid (mip 0, the material's address mode) into `out` (FP16, out_w % 128 == 0).
 *
 * Frame (Algorithm 1): each pixel carries a material id (-1: none), uv and lod
 * = log2(uv footprint of the pixel) + mip bias.  Pass A classifies 128-pixel
 * tiles (tile_w x tile_h) as uniform (one material, more than half the pixels
 * valid) or mixed; an exclusive scan gives each material its slot offsets; pass
 * B packs the valid pixels of mixed tiles into 128-slot tiles of one material.
 * Each pixel is then decoded with per-level lod_k = lod + log2(W_k) (clamped to
 * the level's mips, trilinear) and its material's MLP; the C FP16 channels go
 * to out[pixel].  Pixels with id -1 are left untouched.
 *
 * Anisotropic latent filter (Sec. 3.2 "Anisotropic Filtering": the latents are
 * fetched with the anisotropic filter a renderer uses; the reference formulas
 * of the anisotropic-filtering extension): with Px = |(du/dx, dv/dx)|,
 * Py = |(du/dy, dv/dy)|, Pmax / Pmin their max / min, N = min(ceil(Pmax / Pmin),
 * max_aniso) (1 when Pmax = 0; decided in FP32), every level is sampled by N
 * trilinear probes at uv + (i / (N + 1) - 1/2) d, i = 1..N, d the derivative
 * of the major axis, at lod_k = bias + log2(Pmax W_k / N), and the probes are
 * averaged.
 *
 * Lighting pass (Sec. 4 "Rendering architecture", fused into the frame
 * decode's epilogue when `shaded` is set; needs C >= 8): the decoded channels
 * are read as albedo RGB, tangent-space normal XY encoded (n + 1) / 2,
 * roughness, metalness and ambient occlusion, and shaded with a Lambert
 * diffuse lobe and a GGX specular lobe (height-correlated Smith visibility,
 * Schlick Fresnel) under the directional light, plus a two-colour hemisphere
 * (ground -> sky along z; no environment maps here) sampled at the normal for
 * the diffuse part and at the reflection vector for the specular part, scaled
 * by the occlusion.  Directions need not be normalised. */
typedef struct {
  nbtc_latents latents;   /* 4 levels (with mips for the frame) */
  nbtc_mlp mlp;           /* FP32 [12, 64, .., 64, C]; the same depth and C for every material */
  int32_t out_w, out_h;   /* full-decode grid (0 = not decoded in full) */
  void* out;              /* device FP16 [out_h][out_w][C] */
} nbtc_batch_material;

typedef struct {
  int32_t width, height;  /* pixels */
  const int32_t* mat_id;  /* [height][width] material index or -1 */
  const float* uv;        /* [height][width][2] */
  const float* lod;       /* [height][width]: lod, or the mip bias when duv is set */
  void* out;              /* FP16 [height][width][C] */
  const float* duv;       /* NULL, or [height][width][4] (du/dx, dv/dx, du/dy, dv/dy), 16-byte aligned:
                             anisotropic latent filter (see below) */
  int32_t max_aniso;      /* probes cap of the anisotropic filter, 1..16 */
  float* shaded;          /* NULL, or FP32 [height][width][4]: lighting pass output (linear RGB, 1) */
  float light_dir[3];     /* lighting pass constants, tangent space: direction toward the light, */
  float light_rgb[3];     /* its radiance, */
  float view_dir[3];      /* direction toward the viewer, */
  float sky[3], ground[3];  /* and the hemisphere standing in for prefiltered environment lighting */
} nbtc_frame;

typedef struct nbtc_batch nbtc_batch;

/* What a plan chose and counted (after nbtc_batch_create / the last render). */
typedef struct {
  int32_t warpgroups;      /* tile groups per CTA of the decode kernel */
  int32_t chunk_tiles;     /* tiles per work chunk */
  int32_t tile_w, tile_h;  /* frame classification tile */
  int64_t decode_tiles;    /* 128-texel tiles of the full decode */
  int64_t frame_uniform_tiles, frame_mixed_tiles, frame_packed_tiles;  /* of the last render */
  float tuned_decode_ms, tuned_render_ms;  /* autotuner's best times (0 = not tuned) */
  int32_t render_warpgroups;                /* tile groups per CTA of the frame decode */
  int32_t decode_tmem_operands;             /* 1: the decode's MMA A operands live in tensor memory
                                               (one tile slot per group), 0: in shared memory (two) */
  int32_t render_tmem_operands;             /* the same for the frame decode */
} nbtc_batch_info;

#define NBTC_BATCH_AUTOTUNE 1  /* flags: time the candidate configurations at creation */

/* Builds a plan (allocates its device buffers, packs the MLPs in FP16, builds
 * the work lists, autotunes if asked, captures the graphs).  `mats` is a host
 * array of `count` materials (<= 1024); `frame` may be NULL.  Device pointers in
 * `mats` and `frame` must stay valid while the plan is used.  Material outputs
 * and the frame's out / shaded buffers must be device memory; the materials'
 * inputs and the frame's mat_id / uv / lod / duv device or pinned host memory
 * (NBTC_ERR_INVALID_ARG otherwise, checked here). */
nbtc_status nbtc_batch_create(nbtc_context* ctx, const nbtc_batch_material* mats, int32_t count,
                              const nbtc_frame* frame, int32_t flags, nbtc_batch** plan, void* stream);

/* Full decode of every material (one graph launch: counter reset + one
 * persistent kernel). */
nbtc_status nbtc_decode_batched(nbtc_context* ctx, nbtc_batch* plan, void* stream);

/* Frame: classify, scan, bin, decode (one graph launch). */
nbtc_status nbtc_render_frame(nbtc_context* ctx, nbtc_batch* plan, void* stream);

nbtc_status nbtc_batch_info_get(nbtc_batch* plan, nbtc_batch_info* info);

/* Frees the plan (synchronises its device first). */
nbtc_status nbtc_batch_destroy(nbtc_batch* plan);

/* ------------------------------------------------------------------ measurement probes
 *
 * Kernels with a known amount of work, for the measured ceilings the decode and
 * training kernels are reported against (no counterpart in the paper).  Each
 * enqueues one launch on `stream`; the caller times it (CUDA events). */

/* FP32 FFMA throughput: `ctas` CTAs of 256 threads, each running `iters`
 * rounds of 16 independent fused multiply-adds (8 packed FP32x2 FMAs when
 * `packed` is nonzero).  *flop receives the launch's FLOP count,
 * ctas * 256 * iters * 32.  out_dev: 4 bytes of device memory the kernel may
 * write (it keeps the arithmetic live; nothing is stored in practice).
 * NBTC_ERR_INVALID_ARG for ctas < 1, iters < 1, NULL or non-device pointers. */
nbtc_status nbtc_probe_ffma(nbtc_context* ctx, int32_t ctas, int32_t iters, int32_t packed, float* out_dev,
                            double* flop, void* stream);

/* The latent-gradient scatter of nbtc_train_step alone: for each of
 * args->batch samples at args->uv, the four bilinear taps of every latent level
 * receive the same atomic adds the step makes (one 16-byte vector add per tap
 * with latent_stride 4, else three 4-byte adds) of a constant, into
 * args->latent_grads -- the step's L2 atomics at the step's addresses, with no
 * other work.  It adds to latent_grads (caller-owned; zero them or discard).
 * Argument rules as nbtc_train_step (target, moments and workspace unused). */
nbtc_status nbtc_probe_scatter(nbtc_context* ctx, const nbtc_train_args* args, void* stream);

/* Allocation-free training step (the paper has no counterpart: this is an
 * integration convenience).  For callers that may not allocate device memory
 * at all -- engines that sub-allocate a budget reserved up front, plugin hosts
 * that forbid allocation inside their callbacks, real-time loops that cannot
 * afford the device synchronisation cudaMalloc / cudaFree can cause -- and so
 * can neither supply args->workspace nor create an nbtc_context.  Same work and
 * results as nbtc_train_step, on the current CUDA device; args->workspace is
 * ignored.  Its scratch is a fixed 7.72 MB device array inside the library,
 * held by every GPU that loads the library until the process exits: room for
 * the partial sums of at most 160 CTAs (one per SM, so a batch that needs
 * more than 160 CTAs, possible only on a device with more than 160 SMs, gets
 * NBTC_ERR_UNSUPPORTED) and, when a small batch leaves room after them, for
 * its per-sample gather records (the step then gathers first, as
 * nbtc_train_step does; otherwise it gathers inside its main kernel -- same
 * results either way).  The first call on a device looks up that array's
 * device address and keeps it for the process (make that first call before
 * any stream capture; a cudaDeviceReset after it is not supported).  All
 * calls share the array: calls that overlap on the GPU race and must be
 * ordered by the caller.  Nothing is allocated by this call. */
nbtc_status nbtc_train_step_noalloc(const nbtc_train_args* args, float* loss_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NBTC_H */
