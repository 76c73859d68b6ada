// Batched multi-material decode and the frame pipeline of Sec. 4 /
// Algorithm 1, around the persistent tensor-core decode kernel.
//
// Plan: materials' FP16 MLPs packed once, a device table of per-material
// views (MatDev), a cost-sorted list of work chunks (runs of 128-texel tiles of
// one material) for the full decode, and the frame buffers.  The decode kernel
// takes chunks from an atomic counter, so materials of very different sizes
// share the SMs evenly; a CTA reloads an MLP only when its next chunk belongs
// to another material.
//
// Frame: pass A (k_frame_classify) marks each 128-pixel tile uniform or mixed
// and counts, per material, uniform tiles and valid pixels of mixed tiles
// (per-CTA shared-memory histograms, then one global atomic per material --
// the paper suggests shared-memory atomics for this, Sec. 6); k_frame_scan
// turns the counts into slot offsets (an exclusive prefix sum; Algorithm 1
// reads these offsets but does not say how they are made) and into the chunk
// list; pass B (k_frame_bin) appends uniform tiles to their material's list and
// packs mixed-tile pixels into their material's 128-slot tiles (warp-aggregated
// atomics: one atomic per material present in a warp).  Then the decode kernel
// runs over those chunks.  All four launches are captured in one CUDA graph.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "host.h"
#include "tc.cuh"

namespace nbtc {

constexpr int kMaxMaterials = 1024;
constexpr int kTileK = 128;  // pixels per classification tile

enum TileKind { kTileEmpty = 0, kTileUniform = 1, kTileMixed = 2 };

struct FrameDev {
  const int* mat_id;
  int w, h, tw, th, tiles_x, tiles;
  int nmat;
  int* tkind;
  int* tmat;
  int* ucount;   // uniform tiles per material
  int* pcount;   // valid pixels of mixed tiles per material
  int* ucur;
  int* pcur;
  int* uoff;     // first slot in ulist
  int* poff;     // first packed tile
  int* ulist;
  int* plist;
  WorkChunk* chunks;
  int* nchunks;
  int chunk_cap;
  int chunk_tiles;
  int* stats;    // [uniform tiles, mixed tiles, packed tiles]
  int64_t ulist_cap, plist_cap;  // slots of ulist and plist (bounds of the checked build)
  int* status;                   // context status word (checked build)
};

// Pixel j (0..127) of screen tile t.
__device__ __forceinline__ int tile_pixel(const FrameDev& F, int t, int j) {
  const int ty = t / F.tiles_x, tx = t - ty * F.tiles_x;
  const int r = j / F.tw;
  return (ty * F.th + r) * F.w + tx * F.tw + (j - r * F.tw);
}

// Pass A: one warp per tile, 4 pixels per lane.
__global__ void k_frame_classify(FrameDev F) {
  extern __shared__ int hist[];  // [nmat] mixed-tile pixel counts of this CTA
  for (int m = threadIdx.x; m < F.nmat; m += blockDim.x) hist[m] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (t < F.tiles) {
    int ids[4];
    int cnt = 0, mn = 0x7fffffff, mx = -1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ids[i] = __ldg(F.mat_id + tile_pixel(F, t, lane * 4 + i));
      if (ids[i] >= F.nmat) ids[i] = -1;  // out-of-range ids decode as "no material"
      if (ids[i] >= 0) {
        ++cnt;
        mn = min(mn, ids[i]);
        mx = max(mx, ids[i]);
      }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    const int kind = cnt == 0 ? kTileEmpty : (mn == mx && 2 * cnt > kTileK ? kTileUniform : kTileMixed);
    if (lane == 0) {
      F.tkind[t] = kind;
      F.tmat[t] = kind == kTileUniform ? mn : -1;
      if (kind == kTileUniform) atomicAdd(F.ucount + mn, 1);
      if (kind == kTileUniform) atomicAdd(F.stats + 0, 1);
      if (kind == kTileMixed) atomicAdd(F.stats + 1, 1);
    }
    if (kind == kTileMixed) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (ids[i] >= 0) atomicAdd_block(hist + ids[i], 1);
    }
  }
  __syncthreads();
  for (int m = threadIdx.x; m < F.nmat; m += blockDim.x)
    if (hist[m]) atomicAdd(F.pcount + m, hist[m]);
}

// Offsets (exclusive scans) and the chunk list: per material its uniform-tile
// chunks, then its packed-tile chunks.  One CTA.
__global__ void k_frame_scan(FrameDev F) {
  extern __shared__ int coff[];  // [nmat + 1] chunk offsets
  if (threadIdx.x == 0) {
    int su = 0, sp = 0, sc = 0;
    for (int m = 0; m < F.nmat; ++m) {
      const int U = F.ucount[m];
      const int P = (F.pcount[m] + kTileK - 1) / kTileK;
      F.uoff[m] = su;
      F.poff[m] = sp;
      coff[m] = sc;
      su += U;
      sp += P;
      sc += (U + F.chunk_tiles - 1) / F.chunk_tiles + (P + F.chunk_tiles - 1) / F.chunk_tiles;
    }
    coff[F.nmat] = sc;
    *F.nchunks = min(sc, F.chunk_cap);
    F.stats[2] = sp;
  }
  __syncthreads();
  for (int m = threadIdx.x; m < F.nmat; m += blockDim.x) {
    F.ucur[m] = 0;
    F.pcur[m] = 0;
    int c = coff[m];
    const int U = F.ucount[m], P = (F.pcount[m] + kTileK - 1) / kTileK;
    for (int i = 0; i < U; i += F.chunk_tiles, ++c)
      if (c < F.chunk_cap) F.chunks[c] = WorkChunk{m, kChunkUniform, (int64_t)F.uoff[m] + i, min(F.chunk_tiles, U - i), 0};
    for (int i = 0; i < P; i += F.chunk_tiles, ++c)
      if (c < F.chunk_cap) F.chunks[c] = WorkChunk{m, kChunkPacked, (int64_t)F.poff[m] + i, min(F.chunk_tiles, P - i), 0};
  }
}

// Pass B: uniform tiles -> their material's list; mixed-tile pixels -> packed
// slots of their material (one atomic per material present in the warp).
__global__ void k_frame_bin(FrameDev F) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (t >= F.tiles) return;
  const int kind = F.tkind[t];
  if (kind == kTileUniform) {
    if (lane == 0) {
      const int m = F.tmat[t];
      const int pos = atomicAdd(F.ucur + m, 1);
      int64_t slot = (int64_t)F.uoff[m] + pos;
      NBTC_CHECK_INDEX(slot, F.ulist_cap, F.status);
      F.ulist[slot] = t;
    }
    return;
  }
  if (kind != kTileMixed) return;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int px = tile_pixel(F, t, lane * 4 + i);
    int id = __ldg(F.mat_id + px);
    if (id >= F.nmat) id = -1;
    const unsigned peers = __match_any_sync(0xffffffffu, id);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (id >= 0 && lane == leader) base = atomicAdd(F.pcur + id, __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (id >= 0) {
      int64_t slot = (int64_t)F.poff[id] * kTileK + base + __popc(peers & lt);
      NBTC_CHECK_INDEX(slot, F.plist_cap, F.status);
      F.plist[slot] = px;
    }
  }
}

}  // namespace nbtc

using namespace nbtc;

struct nbtc_batch {
  int device = 0;
  int count = 0;
  int nhid = 0;
  int nout = 0;
  std::vector<nbtc_batch_material> host_mats;
  // device buffers
  MatDev* mats_dev = nullptr;
  unsigned char* packed_dev = nullptr;
  size_t packed_stride = 0;
  WorkChunk* dchunks = nullptr;
  int* dnchunks = nullptr;
  int* dcounter = nullptr;
  int64_t decode_tiles = 0;
  // frame
  bool has_frame = false;
  nbtc_frame frame{};
  FrameDev F{};
  int* frame_block = nullptr;  // all int frame buffers
  WorkChunk* fchunks = nullptr;
  int* fcounter = nullptr;
  size_t plist_ints = 0;
  // tuned configuration and graphs
  int W = 3, Wf = 3, chunk = 32, tw = 16, th = 8;  // W: decode warpgroups, Wf: render warpgroups
  int ta = 0, taf = 0;  // A operands in TMEM (4 warpgroups x 1 slot) for the decode / the frame
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g_decode = nullptr, g_render = nullptr;
  nbtc_batch_info info{};
};

namespace nbtc {

static nbtc_status upload(void* dst, const void* src, size_t n, cudaStream_t s) {
  return cuda_check(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s), "upload");
}

// Host-built chunk list of the full decode: largest materials first, each
// material's tiles in runs of `chunk` tiles (consecutive column-major tile
// numbers, i.e. neighbouring rows of one 128-texel column block).
static std::vector<WorkChunk> decode_chunks(const nbtc_batch* B, int chunk) {
  std::vector<int> order;
  for (int m = 0; m < B->count; ++m)
    if (B->host_mats[m].out) order.push_back(m);
  auto tiles = [&](int m) { return (int64_t)B->host_mats[m].out_w * B->host_mats[m].out_h / kTile; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tiles(a) > tiles(b); });
  std::vector<WorkChunk> v;
  for (int m : order)
    for (int64_t i = 0; i < tiles(m); i += chunk)
      v.push_back(WorkChunk{m, kChunkGrid, i, (int)std::min<int64_t>(chunk, tiles(m) - i), 0});
  return v;
}

static TcArgs base_args(nbtc_context* ctx, const nbtc_batch* B) {
  TcArgs p;
  memset(&p, 0, sizeof(p));
  p.d.status = ctx->status_dev;
  p.budget = ctx->wait_budget > 0 ? ctx->wait_budget : ctx->wait_budget < 0 ? 0 : kDefaultWaitBudget;
  p.mode = kModeBatch;
  p.mats = B->mats_dev;
  return p;
}

static nbtc_status enqueue_decode(nbtc_context* ctx, nbtc_batch* B, cudaStream_t s) {
  nbtc_status st = cuda_check(cudaMemsetAsync(B->dcounter, 0, sizeof(int), s), "reset chunk counter");
  if (st) return st;
  TcArgs p = base_args(ctx, B);
  p.chunks = B->dchunks;
  p.nchunks_dev = B->dnchunks;
  p.chunk_counter = B->dcounter;
  p.tmem_a = B->ta;
  return launch_tc_args(ctx, p, B->nhid, kF16, B->W, B->ta ? 1 : 2, ctx->sm_count, s);
}

// Lighting constants of a frame: unit directions and the half vector, in double
// before rounding to FP32.
static LightDev make_light(const nbtc_frame& f) {
  LightDev L;
  auto unit = [](const float* a, double* o) {
    const double n = std::sqrt((double)a[0] * a[0] + (double)a[1] * a[1] + (double)a[2] * a[2]);
    for (int i = 0; i < 3; ++i) o[i] = n > 0 ? a[i] / n : (i == 2 ? 1.0 : 0.0);
  };
  double l[3], v[3], h[3];
  unit(f.light_dir, l);
  unit(f.view_dir, v);
  const double hs[3] = {l[0] + v[0], l[1] + v[1], l[2] + v[2]};
  const double hn = std::sqrt(hs[0] * hs[0] + hs[1] * hs[1] + hs[2] * hs[2]);
  double ldoth = 0;
  for (int i = 0; i < 3; ++i) {
    h[i] = hn > 0 ? hs[i] / hn : (i == 2 ? 1.0 : 0.0);
    ldoth += l[i] * h[i];
  }
  for (int i = 0; i < 3; ++i) {
    L.l[i] = (float)l[i];
    L.v[i] = (float)v[i];
    L.h[i] = (float)h[i];
    L.rgb[i] = f.light_rgb[i];
    L.sky[i] = f.sky[i];
    L.ground[i] = f.ground[i];
  }
  L.ldoth = (float)(ldoth > 0 ? ldoth : 0);
  return L;
}

static nbtc_status enqueue_render(nbtc_context* ctx, nbtc_batch* B, cudaStream_t s) {
  FrameDev& F = B->F;
  nbtc_status st;
  const size_t zero_ints = (size_t)2 * F.nmat + 3;  // ucount, pcount, stats are contiguous
  if ((st = cuda_check(cudaMemsetAsync(F.ucount, 0, zero_ints * sizeof(int), s), "reset frame counts"))) return st;
  if ((st = cuda_check(cudaMemsetAsync(F.plist, 0xFF, B->plist_ints * sizeof(int), s), "reset packed slots")))
    return st;
  if ((st = cuda_check(cudaMemsetAsync(B->fcounter, 0, sizeof(int), s), "reset chunk counter"))) return st;
  const int blocks = (F.tiles + 7) / 8;
  k_frame_classify<<<blocks, 256, F.nmat * sizeof(int), s>>>(F);
  if ((st = cuda_check(cudaGetLastError(), "launch k_frame_classify"))) return st;
  k_frame_scan<<<1, 256, (F.nmat + 1) * sizeof(int), s>>>(F);
  if ((st = cuda_check(cudaGetLastError(), "launch k_frame_scan"))) return st;
  k_frame_bin<<<blocks, 256, 0, s>>>(F);
  if ((st = cuda_check(cudaGetLastError(), "launch k_frame_bin"))) return st;
  TcArgs p = base_args(ctx, B);
  p.chunks = B->fchunks;
  p.nchunks_dev = F.nchunks;
  p.chunk_counter = B->fcounter;
  p.ulist = F.ulist;
  p.plist = F.plist;
  p.fmat = B->frame.mat_id;
  p.fuv = B->frame.uv;
  p.flod = B->frame.lod;
  p.fduv = B->frame.duv;
  p.max_aniso = B->frame.duv ? B->frame.max_aniso : 1;
  p.fshade = B->frame.shaded;
  p.light = make_light(B->frame);
  p.fout = static_cast<uint16_t*>(B->frame.out);
  p.frame_w = F.w;
  p.frame_pixels = (int64_t)F.w * F.h;
  p.tile_w = F.tw;
  p.tile_h = F.th;
  p.tiles_x = F.tiles_x;
  p.tmem_a = B->taf;
  return launch_tc_args(ctx, p, B->nhid, kF16, B->Wf, B->taf ? 1 : 2, ctx->sm_count, s);
}

static nbtc_status set_tile_shape(nbtc_batch* B, int tw, int th) {
  FrameDev& F = B->F;
  if (F.w % tw || F.h % th) return fail(NBTC_ERR_UNSUPPORTED, "frame size not a multiple of the tile");
  F.tw = tw;
  F.th = th;
  F.tiles_x = F.w / tw;
  F.tiles = F.tiles_x * (F.h / th);
  B->tw = tw;
  B->th = th;
  return NBTC_OK;
}

static nbtc_status set_decode_chunk(nbtc_batch* B, int chunk, cudaStream_t s) {
  std::vector<WorkChunk> v = decode_chunks(B, chunk);
  const int n = (int)v.size();
  nbtc_status st;
  if (n && (st = upload(B->dchunks, v.data(), v.size() * sizeof(WorkChunk), s))) return st;
  if ((st = upload(B->dnchunks, &n, sizeof(int), s))) return st;
  B->chunk = chunk;
  return cuda_check(cudaStreamSynchronize(s), "chunk upload");
}

// Mean of `reps` timed runs after one warm-up run (CUDA events on `s`).
template <class F>
static float time_ms(F&& run, cudaStream_t s, int reps, nbtc_status& st) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  st = run();
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "tune warm-up");
  float ms = 0.f;
  if (!st) {
    cudaEventRecord(a, s);
    for (int i = 0; i < reps && !st; ++i) st = run();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

static nbtc_status capture(nbtc_context* ctx, nbtc_batch* B, bool render, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  // one uncaptured run first: kernel attributes are set outside the capture
  nbtc_status st = render ? enqueue_render(ctx, B, B->cap) : enqueue_decode(ctx, B, B->cap);
  if (!st) st = cuda_check(cudaStreamSynchronize(B->cap), "pre-capture run");
  if (st) return st;
  st = cuda_check(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (st) return st;
  nbtc_status run = render ? enqueue_render(ctx, B, B->cap) : enqueue_decode(ctx, B, B->cap);
  st = cuda_check(cudaStreamEndCapture(B->cap, &g), "end capture");
  if (run) {
    if (g) cudaGraphDestroy(g);
    return run;
  }
  if (st) return st;
  st = cuda_check(cudaGraphInstantiate(out, g, 0), "instantiate graph");
  cudaGraphDestroy(g);
  return st;
}

static void free_plan(nbtc_batch* B) {
  if (!B) return;
  cudaSetDevice(B->device);
  cudaDeviceSynchronize();
  if (B->g_decode) cudaGraphExecDestroy(B->g_decode);
  if (B->g_render) cudaGraphExecDestroy(B->g_render);
  if (B->cap) cudaStreamDestroy(B->cap);
  cudaFree(B->mats_dev);
  cudaFree(B->packed_dev);
  cudaFree(B->dchunks);
  cudaFree(B->dnchunks);
  cudaFree(B->dcounter);
  cudaFree(B->frame_block);
  cudaFree(B->fchunks);
  cudaFree(B->fcounter);
  delete B;
}

}  // namespace nbtc

extern "C" {

nbtc_status nbtc_batch_create(nbtc_context* ctx, const nbtc_batch_material* mats, int32_t count,
                              const nbtc_frame* frame, int32_t flags, nbtc_batch** plan, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if (!plan || !mats || count < 1 || count > kMaxMaterials)
    return fail(NBTC_ERR_INVALID_ARG, "plan/mats NULL or count outside 1..1024");
  *plan = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  // ---- validate
  int nhid = -1, nout = -1;
  for (int m = 0; m < count; ++m) {
    const nbtc_batch_material& M = mats[m];
    if ((st = check_mlp(&M.mlp))) return st;
    if (M.latents.num_levels != 4) return fail(NBTC_ERR_UNSUPPORTED, "batched materials take 4 latent levels");
    LevelView lv[NBTC_MAX_LEVELS];
    if ((st = make_level_views(&M.latents, 0, lv))) return st;
    if ((st = need_inputs(&M.latents, &M.mlp))) return st;
    size_t pb = 0;
    if ((st = tc_packed_bytes(&M.mlp, NBTC_FP16, &pb))) return st;
    const int h = M.mlp.num_layers - 1, c = M.mlp.dims[M.mlp.num_layers];
    if (nhid < 0) {
      nhid = h;
      nout = c;
    } else if (h != nhid || c != nout) {
      return fail(NBTC_ERR_UNSUPPORTED, "every material needs the same MLP depth and output channels");
    }
    if (M.out) {
      if (M.out_w <= 0 || M.out_h <= 0 || M.out_w % kTile) return fail(NBTC_ERR_INVALID_ARG, "out_w must be a positive multiple of 128");
      if ((int64_t)M.out_w * M.out_h / kTile >= (int64_t)1 << 31) return fail(NBTC_ERR_UNSUPPORTED, "material output too large");
      if (!aligned(M.out, 16)) return fail(NBTC_ERR_INVALID_ARG, "material out not 16-byte aligned");
      if ((st = need_device(M.out, "material out"))) return st;  // written with bulk copies
      for (int k = 0; k < 4; ++k)
        if (M.latents.levels[k].width > M.out_w) return fail(NBTC_ERR_UNSUPPORTED, "latent level wider than the output");
    }
  }
  if (frame) {
    if (frame->width <= 0 || frame->height <= 0 || !frame->mat_id || !frame->uv || !frame->lod || !frame->out)
      return fail(NBTC_ERR_INVALID_ARG, "frame buffers NULL or size <= 0");
    if (!aligned(frame->uv, 8)) return fail(NBTC_ERR_INVALID_ARG, "frame uv not 8-byte aligned");
    if (frame->duv && (!aligned(frame->duv, 16) || frame->max_aniso < 1 || frame->max_aniso > 16))
      return fail(NBTC_ERR_INVALID_ARG, "frame duv not 16-byte aligned or max_aniso outside 1..16");
    if (frame->shaded && !aligned(frame->shaded, 16))
      return fail(NBTC_ERR_INVALID_ARG, "frame shaded output not 16-byte aligned");
    if (frame->shaded && nout < 8) return fail(NBTC_ERR_UNSUPPORTED, "the lighting pass needs at least 8 channels");
    if ((st = need_readable(frame->mat_id, "frame mat_id")) || (st = need_readable(frame->uv, "frame uv")) ||
        (st = need_readable(frame->lod, "frame lod")) || (frame->duv && (st = need_readable(frame->duv, "frame duv"))) ||
        (st = need_device(frame->out, "frame out")) || (frame->shaded && (st = need_device(frame->shaded, "frame shaded"))))
      return st;
    if ((int64_t)frame->width * frame->height >= (int64_t)1 << 31) return fail(NBTC_ERR_UNSUPPORTED, "frame too large");
  }
  nbtc_batch* B = new nbtc_batch();
  B->device = ctx->device;
  B->count = count;
  B->nhid = nhid;
  B->nout = nout;
  B->host_mats.assign(mats, mats + count);
#define NBTC_TRY(x)     \
  do {                  \
    st = (x);           \
    if (st) {           \
      free_plan(B);     \
      return st;        \
    }                   \
  } while (0)
  NBTC_TRY(cuda_check(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking), "plan stream"));
  // ---- packed MLPs and the material table
  size_t pb = 0;
  tc_packed_bytes(&mats[0].mlp, NBTC_FP16, &pb);
  B->packed_stride = (pb + 255) & ~(size_t)255;
  NBTC_TRY(cuda_check(cudaMalloc(&B->packed_dev, B->packed_stride * count), "plan MLPs"));
  std::vector<MatDev> md(count);
  for (int m = 0; m < count; ++m) {
    const nbtc_batch_material& M = mats[m];
    NBTC_TRY(launch_pack_mlp(ctx, &M.mlp, NBTC_FP16, nullptr, B->packed_dev + B->packed_stride * m, pb, s));
    MatDev& d = md[m];
    memset(&d, 0, sizeof(d));
    make_level_views(&M.latents, 0, d.d.lv);
    attach_checks(ctx, d.d.lv, 4);
    d.d.wrap = M.latents.address == NBTC_WRAP;
    d.d.grid_w = M.out ? M.out_w : 0;
    d.d.grid_h = M.out ? M.out_h : 0;
    d.d.n = M.out ? (int64_t)M.out_w * M.out_h : 0;
    d.d.cw = make_grid_coord(M.out ? M.out_w : 1);
    d.d.ch = make_grid_coord(M.out ? M.out_h : 1);
    d.d.out = M.out;
    d.d.status = ctx->status_dev;
    d.packed = B->packed_dev + B->packed_stride * m;
    d.nout = nout;
    d.hdiv = make_fastdiv(M.out ? (uint32_t)M.out_h : 1u);
    d.tiles = d.d.n / kTile;
    B->decode_tiles += d.tiles;
    for (int k = 0; k < 4; ++k) {
      const nbtc_level& Lv = M.latents.levels[k];
      d.mips[k] = Lv.num_mips;
      d.log2w[k] = (float)std::log2((double)Lv.width);
      int w = Lv.width, h = Lv.height, off = 0;
      for (int mm = 0; mm < NBTC_MAX_MIPS; ++mm) {
        d.mip_off[k][mm] = off;
        off += (w / 4) * (h / 4);
        w = std::max(4, w / 2);
        h = std::max(4, h / 2);
      }
    }
  }
  NBTC_TRY(cuda_check(cudaMalloc(&B->mats_dev, sizeof(MatDev) * count), "plan table"));
  NBTC_TRY(upload(B->mats_dev, md.data(), sizeof(MatDev) * count, s));
  // ---- full-decode work list (largest chunk count over the candidate chunk sizes)
  const size_t max_chunks = decode_chunks(B, 8).size() + 1;
  NBTC_TRY(cuda_check(cudaMalloc(&B->dchunks, sizeof(WorkChunk) * max_chunks), "decode chunks"));
  NBTC_TRY(cuda_check(cudaMalloc(&B->dnchunks, sizeof(int)), "decode chunk count"));
  NBTC_TRY(cuda_check(cudaMalloc(&B->dcounter, sizeof(int)), "decode counter"));
  NBTC_TRY(set_decode_chunk(B, 32, s));
  // ---- frame buffers
  if (frame) {
    B->has_frame = true;
    B->frame = *frame;
    FrameDev& F = B->F;
    F.mat_id = frame->mat_id;
    F.w = frame->width;
    F.h = frame->height;
    F.nmat = count;
    F.chunk_tiles = 16;
    const int pixels = frame->width * frame->height;
    const int max_tiles = pixels / kTileK + 1;
    B->plist_ints = (size_t)(pixels / kTileK + count + 1) * kTileK;
    const size_t ints = (size_t)2 * count + 3 /* counts + stats */ + 4 * (size_t)count /* cursors, offsets */ +
                        2 * (size_t)max_tiles /* kind, mat */ + max_tiles /* ulist */ + B->plist_ints + 1;
    NBTC_TRY(cuda_check(cudaMalloc(&B->frame_block, ints * sizeof(int)), "frame buffers"));
    int* q = B->frame_block;
    F.ucount = q; q += count;
    F.pcount = q; q += count;
    F.stats = q; q += 3;
    F.ucur = q; q += count;
    F.pcur = q; q += count;
    F.uoff = q; q += count;
    F.poff = q; q += count;
    F.tkind = q; q += max_tiles;
    F.tmat = q; q += max_tiles;
    F.ulist = q; q += max_tiles;
    F.nchunks = q; q += 1;
    F.plist = q;
    F.ulist_cap = max_tiles;
    F.plist_cap = (int64_t)B->plist_ints;
    F.status = ctx->status_dev;
    F.chunk_cap = 2 * (max_tiles + count) + 16;
    NBTC_TRY(cuda_check(cudaMalloc(&B->fchunks, sizeof(WorkChunk) * F.chunk_cap), "frame chunks"));
    NBTC_TRY(cuda_check(cudaMalloc(&B->fcounter, sizeof(int)), "frame counter"));
    F.chunks = B->fchunks;
    NBTC_TRY(set_tile_shape(B, 16, 8));
  }
  NBTC_TRY(cuda_check(cudaStreamSynchronize(s), "plan set-up"));
  // ---- autotune: warpgroups x chunk size (decode); warpgroups x tile shape (frame)
  if (flags & NBTC_BATCH_AUTOTUNE) {
    float best = 1e30f;
    int bw = B->W, bc = B->chunk, bta = B->ta;
    // candidates: 3 or 4 warpgroups of two slots with shared-memory operands,
    // or 4 warpgroups of one slot with TMEM operands (coded as W = 5 here)
    if (B->decode_tiles > 0) {
      for (int W : {3, 4, 5})
        for (int c : {8, 32, 128}) {
          B->W = W == 5 ? 4 : W;
          B->ta = W == 5;
          NBTC_TRY(set_decode_chunk(B, c, B->cap));
          const float ms = time_ms([&] { return enqueue_decode(ctx, B, B->cap); }, B->cap, 3, st);
          if (st) {
            free_plan(B);
            return st;
          }
          if (ms < best) {
            best = ms;
            bw = B->W;
            bta = B->ta;
            bc = c;
          }
        }
      B->W = bw;
      B->ta = bta;
      NBTC_TRY(set_decode_chunk(B, bc, B->cap));
      B->info.tuned_decode_ms = best;
    }
    if (B->has_frame) {
      float bestf = 1e30f;
      int fw = B->Wf, fta = B->taf, ftw = 16, fth = 8;
      const int shapes[4][2] = {{16, 8}, {32, 4}, {8, 16}, {128, 1}};
      for (int W : {3, 4, 5})
        for (auto& sh : shapes) {
          if (set_tile_shape(B, sh[0], sh[1])) continue;
          B->Wf = W == 5 ? 4 : W;
          B->taf = W == 5;
          const float ms = time_ms([&] { return enqueue_render(ctx, B, B->cap); }, B->cap, 3, st);
          if (st) {
            free_plan(B);
            return st;
          }
          if (ms < bestf) {
            bestf = ms;
            fw = B->Wf;
            fta = B->taf;
            ftw = sh[0];
            fth = sh[1];
          }
        }
      NBTC_TRY(set_tile_shape(B, ftw, fth));
      B->Wf = fw;
      B->taf = fta;
      B->info.tuned_render_ms = bestf;
    }
  }
  // ---- graphs
  if (B->decode_tiles > 0) NBTC_TRY(capture(ctx, B, false, &B->g_decode));
  if (B->has_frame) NBTC_TRY(capture(ctx, B, true, &B->g_render));
#undef NBTC_TRY
  B->info.warpgroups = B->W;
  B->info.render_warpgroups = B->Wf;
  B->info.decode_tmem_operands = B->ta;
  B->info.render_tmem_operands = B->taf;
  B->info.chunk_tiles = B->chunk;
  B->info.tile_w = B->tw;
  B->info.tile_h = B->th;
  B->info.decode_tiles = B->decode_tiles;
  *plan = B;
  return NBTC_OK;
}

nbtc_status nbtc_decode_batched(nbtc_context* ctx, nbtc_batch* B, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if (!B) return fail(NBTC_ERR_INVALID_ARG, "plan NULL");
  if (!B->g_decode) return NBTC_OK;  // no material has a full-decode output
  return cuda_check(cudaGraphLaunch(B->g_decode, (cudaStream_t)stream), "launch decode graph");
}

nbtc_status nbtc_render_frame(nbtc_context* ctx, nbtc_batch* B, void* stream) {
  NBTC_RANGE();
  nbtc_status st = enter(ctx);
  if (st) return st;
  if (!B) return fail(NBTC_ERR_INVALID_ARG, "plan NULL");
  if (!B->g_render) return fail(NBTC_ERR_INVALID_ARG, "the plan has no frame");
  return cuda_check(cudaGraphLaunch(B->g_render, (cudaStream_t)stream), "launch render graph");
}

nbtc_status nbtc_batch_info_get(nbtc_batch* B, nbtc_batch_info* info) {
  if (!B || !info) return fail(NBTC_ERR_INVALID_ARG, "NULL argument");
  nbtc_status st = cuda_check(cudaSetDevice(B->device), "cudaSetDevice");
  if (st) return st;
  *info = B->info;
  if (B->has_frame) {
    int stats[3] = {0, 0, 0};
    if ((st = cuda_check(cudaDeviceSynchronize(), "sync")) ||
        (st = cuda_check(cudaMemcpy(stats, B->F.stats, sizeof(stats), cudaMemcpyDeviceToHost), "read stats")))
      return st;
    info->frame_uniform_tiles = stats[0];
    info->frame_mixed_tiles = stats[1];
    info->frame_packed_tiles = stats[2];
  }
  return NBTC_OK;
}

nbtc_status nbtc_batch_destroy(nbtc_batch* B) {
  free_plan(B);
  return NBTC_OK;
}

}  // extern "C"
