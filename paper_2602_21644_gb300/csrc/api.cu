// C ABI of libdags.so (declared in include/dags.h): context and workspace,
// host-side argument checks, and the launch sequence of each entry point.
#include <math.h>
#include <new>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include <cuda.h>

#include "common.cuh"

#include <nvtx3/nvToolsExt.h>

using namespace dags;

// Opt-in per-kernel device timing: a pair of CUDA events around every
// kernel launch of the library, on the launch stream; read and reset by
// dags_timing_read. Skipped while the stream is being captured into a graph.
struct KernelTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> kid;      // kernel id per used pair
  size_t used = 0;           // pairs in use
  double ms[DAGS_KERNEL_COUNT] = {};
  int64_t launches[DAGS_KERNEL_COUNT] = {};

  bool active(cudaStream_t s) {
    if (!on) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    return true;
  }
  // returns the index of the begin event, or -1
  int begin(int k, cudaStream_t s) {
    if (!active(s)) return -1;
    if (2 * (used + 1) > pool.size()) {
      for (int i = 0; i < 512; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        pool.push_back(e);
      }
    }
    const int i = (int)used++;
    kid.resize(used);
    kid[i] = k;
    cudaEventRecord(pool[2 * i], s);
    return i;
  }
  void end(int i, cudaStream_t s) {
    if (i >= 0) cudaEventRecord(pool[2 * i + 1], s);
  }
  int collect() {
    for (size_t i = 0; i < used; ++i) {
      float t = 0.f;
      if (cudaEventSynchronize(pool[2 * i + 1]) != cudaSuccess) return DAGS_E_CUDA;
      if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) != cudaSuccess) return DAGS_E_CUDA;
      ms[kid[i]] += t;
      launches[kid[i]] += 1;
    }
    used = 0;
    return DAGS_OK;
  }
  void release() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

// A captured tracking iteration (exec) and a captured chunk of kTrackUnroll
// iterations (exec_chunk), and the arguments they were captured with.
constexpr int kTrackUnroll = 10;
struct TrackGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraphExec_t exec_chunk = nullptr;
  cudaStream_t cap = nullptr;       // private stream used for capture
  unsigned char key[512];
  size_t key_len = 0;
};

struct dags_ctx {
  int device = 0;
  int num_sms = 0;
  Workspace ws;
  KernelTimer timer;
  TrackGraph graph;
  TrackGraph graph_lm;            // captured LM iteration
  LmBuffers lm;                   // allocated by the first LM call
  uint32_t *warp_masks = nullptr; // [max_tiles][kMaskGroups][8] forward masks of the tracking loop
  uint32_t *cand_ids = nullptr;   // [max_n] the tracking frame's culled candidates
  uint32_t *cand_n = nullptr;     // [1]
  float *cull_pose = nullptr;     // [12]
  uint32_t *track_order = nullptr;  // [max_tiles] the tracking loop's render order (ranked one iteration late)
  uint32_t *prev_count = nullptr;   // [max_tiles] the counts it is ranked from
  int track_order_tiles = 0;        // the tile count track_order is a permutation of (0: none yet)
  double *reg_partial = nullptr;  // per-CTA sums of the regulariser (first call)
  double *edge_partial = nullptr; // per-CTA sums of the edge-warp term (first call)
  float *rel32 = nullptr;         // [12] FP32 relative pose of the regularisers (first call)
  EpiBuffers epi;                 // epipolar verification, grown on demand
  MpBuffers mp;
  MpnetScratch net;
  cudaStream_t last_stream = nullptr;
  // the buffers of the latest forward (backward must follow its forward)
  const void *fwd_image = nullptr;
  const void *fwd_last = nullptr;
  const void *fwd_gauss = nullptr;
  int64_t fwd_n = -1;
  int fwd_views = 0, fwd_w = 0, fwd_h = 0, fwd_tiles = 0;
};

namespace {

template <class T>
cudaError_t alloc(T **p, size_t count) {
  return cudaMalloc((void **)p, (count > 0 ? count : 1) * sizeof(T));
}

void free_ws(Workspace &w) {
  void *ptrs[] = {w.rec2d, w.rec_lo, w.rect, w.grad2d, w.tile_count, w.tile_start, w.tile_cursor, w.keys,
                  w.keys_tmp, w.sorted_ids, w.tile_order, w.loss_partial, w.pose_partial, w.pose32,
                  w.vis_ids, w.vis_append, w.vis_n, w.counters, w.evals};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  w = Workspace();
}

void free_mp(MpBuffers &b) {
  void *ptrs[] = {b.e, b.mpf, b.acc, b.mhat, b.sige, b.U, b.Mt, b.Ut, b.obs, b.hist, b.sel};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  b = MpBuffers();
}

void free_lm(LmBuffers &b) {
  void *ptrs[] = {b.tan, b.partial, b.normal, b.pose_try};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  b = LmBuffers();
}

void free_epi(EpiBuffers &b) {
  void *ptrs[] = {b.count, b.off, b.block_sum, b.rank, b.vals, b.dist, b.F};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  b = EpiBuffers();
}

void free_net(MpnetScratch &b) {
  void *ptrs[] = {b.y, b.acts, b.dz2, b.grad, b.inv_n};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  b = MpnetScratch();
}

bool finite_pos(float x) { return isfinite(x) && x > 0.f; }

int check_camera(const dags_ctx *ctx, const dags_camera *cam) {
  if (!cam) return DAGS_E_INVAL;
  if (cam->width <= 0 || cam->height <= 0 || cam->width > ctx->ws.max_w || cam->height > ctx->ws.max_h)
    return DAGS_E_INVAL;
  if (!finite_pos(cam->fx) || !finite_pos(cam->fy) || !isfinite(cam->cx) || !isfinite(cam->cy))
    return DAGS_E_INVAL;
  return DAGS_OK;
}

int make_raster(const dags_camera *cam, const dags_raster_cfg *rc_in, Raster *r) {
  dags_raster_cfg rc;
  if (rc_in) rc = *rc_in;
  else dags_default_raster_cfg(&rc);
  if (rc.tile != kTile) return DAGS_E_INVAL;
  if (!(rc.alpha_min > 0.f) || !(rc.alpha_max <= 1.f) || !(rc.alpha_min < rc.alpha_max)) return DAGS_E_INVAL;
  if (!(rc.t_min > 0.f && rc.t_min < 1.f) || !(rc.dilation >= 0.f) || !(rc.z_near > 0.f) || !(rc.guard > 0.f))
    return DAGS_E_INVAL;
  r->fx = cam->fx; r->fy = cam->fy; r->cx = cam->cx; r->cy = cam->cy;
  r->W = cam->width; r->H = cam->height;
  r->tiles_x = (cam->width + kTile - 1) / kTile;
  r->tiles_y = (cam->height + kTile - 1) / kTile;
  r->T = r->tiles_x * r->tiles_y;
  r->alpha_min = rc.alpha_min; r->alpha_max = rc.alpha_max; r->t_min = rc.t_min;
  r->dilation = rc.dilation; r->z_near = rc.z_near;
  r->limx = rc.guard * 0.5f * (float)cam->width / cam->fx;
  r->limy = rc.guard * 0.5f * (float)cam->height / cam->fy;
  r->log2_alpha_min = log2f(rc.alpha_min);
  return DAGS_OK;
}

int make_loss(const dags_loss_cfg *lc_in, Loss *l) {
  dags_loss_cfg lc;
  if (lc_in) lc = *lc_in;
  else dags_default_loss_cfg(&lc);
  if (!isfinite(lc.lambda_pho) || !isfinite(lc.lambda_depth) || !(lc.o_eps >= 0.f)) return DAGS_E_INVAL;
  if (lc.weight_mode != 0 && lc.weight_mode != 1) return DAGS_E_INVAL;
  l->lambda_pho = lc.lambda_pho; l->lambda_depth = lc.lambda_depth; l->o_eps = lc.o_eps;
  l->weight_mode = lc.weight_mode; l->weight_grad = lc.weight_grad ? 1 : 0;
  return DAGS_OK;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? DAGS_OK : DAGS_E_CUDA; }

int common_args(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, const double *poses,
                int32_t n_views) {
  if (!ctx) return DAGS_E_INVAL;
  if (n < 0 || n > ctx->ws.max_n || (n > 0 && !gauss)) return DAGS_E_INVAL;
  if (n_views < 1 || n_views > ctx->ws.max_v || !poses) return DAGS_E_INVAL;
  if (((uintptr_t)gauss & 15u) != 0) return DAGS_E_INVAL;
  return check_camera(ctx, cam);
}

}  // namespace

// An NVTX range around each ABI call (header-only NVTX 3: a no-op unless a
// profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

extern "C" {

void dags_default_raster_cfg(dags_raster_cfg *c) {
  if (!c) return;
  c->tile = 16;
  c->alpha_min = 1.0f / 255.0f;
  c->alpha_max = 0.99f;
  c->t_min = 1e-4f;
  c->dilation = 0.3f;
  c->z_near = 0.2f;
  c->guard = 1.3f;
}

void dags_default_loss_cfg(dags_loss_cfg *c) {
  if (!c) return;
  c->lambda_pho = 0.9f;
  c->lambda_depth = 0.1f;
  c->weight_mode = 0;
  c->weight_grad = 0;
  c->o_eps = 1e-6f;
}

void dags_default_pose_cfg(dags_pose_cfg *c) {
  if (!c) return;
  for (int k = 0; k < 6; ++k) c->lr[k] = 1e-3;
  c->beta1 = 0.9;
  c->beta2 = 0.999;
  c->eps = 1e-8;
}

int dags_abi_version(void) { return DAGS_ABI_VERSION; }

const char *dags_status_string(int code) {
  switch (code) {
    case DAGS_OK: return "ok";
    case DAGS_E_INVAL: return "invalid argument";
    case DAGS_E_CUDA: return "CUDA runtime error";
    case DAGS_E_CAPACITY: return "tile/Gaussian pair capacity exceeded (see dags_sync_status)";
    case DAGS_E_TIMEOUT: return "a bounded device wait gave up";
    case DAGS_E_NOMEM: return "workspace allocation failed";
    case DAGS_E_ORDER: return "splat_backward does not follow its splat_forward on this context";
    case DAGS_E_BOUNDS: return "an index was out of range (a DAGS_CHECK build's check, or a caller's id; the access was skipped)";
    default: return "unknown status";
  }
}

int dags_create(dags_ctx **out, int64_t max_gaussians, int32_t max_width, int32_t max_height,
                int32_t max_views, int64_t max_pairs) {
  NvtxRange nv("dags_create");
  if (!out) return DAGS_E_INVAL;
  *out = nullptr;
  if (max_gaussians < 0 || max_gaussians > (int64_t)0x7FFFFFFF || max_width <= 0 || max_height <= 0 ||
      max_width > 32768 || max_height > 32768 || max_views < 1 || max_views > 64 || max_pairs < 0)
    return DAGS_E_INVAL;
  if (max_pairs == 0) {
    // 16 pairs per Gaussian and view, and at least min(N, 4096) slots per
    // tile for the fixed-capacity buckets of the tracking loop
    const int64_t tiles = (int64_t)((max_width + kTile - 1) / kTile) * ((max_height + kTile - 1) / kTile);
    const int64_t per_tile = max_gaussians < 4096 ? max_gaussians : 4096;
    max_pairs = 16 * max_gaussians * (int64_t)max_views;
    if (per_tile * tiles * max_views > max_pairs) max_pairs = per_tile * tiles * max_views;
  }
  if (max_pairs < 1024) max_pairs = 1024;
  if (max_pairs > (int64_t)0xFFFFFFFE) return DAGS_E_INVAL;
  dags_ctx *c = new (std::nothrow) dags_ctx();
  if (!c) return DAGS_E_NOMEM;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return DAGS_E_CUDA;
  }
  Workspace &w = c->ws;
  w.max_n = max_gaussians > 0 ? max_gaussians : 1;
  w.max_w = max_width;
  w.max_h = max_height;
  w.max_v = max_views;
  w.max_tiles = ((max_width + kTile - 1) / kTile) * ((max_height + kTile - 1) / kTile);
  w.max_pairs = max_pairs;
  w.bwd_prep_blocks = (int)((w.max_n + kBwdPrepBlock - 1) / kBwdPrepBlock);
  w.band = c->num_sms;
  const size_t vn = (size_t)w.max_v * (size_t)w.max_n;
  const size_t vt = (size_t)w.max_v * (size_t)w.max_tiles;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(alloc(&w.rec2d, vn * 3));
  A(alloc(&w.rec_lo, vn));
  A(alloc(&w.rect, vn));
  A(alloc(&w.grad2d, vn * kGradWords));
  A(alloc(&w.tile_count, vt));
  A(alloc(&w.tile_start, vt + 1));
  A(alloc(&w.tile_cursor, vt));
  A(alloc(&w.keys, (size_t)max_pairs));
  A(alloc(&w.keys_tmp, (size_t)max_pairs));
  A(alloc(&w.sorted_ids, (size_t)max_pairs));
  A(alloc(&w.tile_order, vt));
  A(alloc(&w.loss_partial, vt));
  A(alloc(&w.pose_partial, (size_t)w.bwd_prep_blocks * w.max_v * 6));
  A(alloc(&w.pose32, (size_t)w.max_v * 12));
  A(alloc(&w.vis_ids, vn));
  A(alloc(&w.vis_append, (size_t)w.max_v));
  A(alloc(&w.vis_n, (size_t)w.max_v));
  A(alloc(&w.counters, (size_t)CNT_N));
  A(alloc(&w.evals, (size_t)4));
  A(alloc(&c->warp_masks, (size_t)w.max_tiles * kMaskGroups * 8));
  A(alloc(&c->cand_ids, (size_t)w.max_n));
  A(alloc(&c->cand_n, (size_t)1));
  A(alloc(&c->cull_pose, (size_t)12));
  A(alloc(&c->track_order, (size_t)w.max_tiles));
  A(alloc(&c->prev_count, (size_t)w.max_tiles));
  if (e == cudaSuccess) e = cudaMemset(w.tile_count, 0, vt * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(w.tile_cursor, 0, vt * sizeof(uint32_t));
  MpBuffers &mb = c->mp;
  A(alloc(&mb.e, (size_t)max_width * max_height));
  A(alloc(&mb.mpf, (size_t)max_width * max_height));
  A(alloc(&mb.pyr, mp_pyramid_floats(max_width, max_height)));
  A(alloc(&mb.acc, (size_t)DAGS_MP_MAX_REGIONS * 4));
  A(alloc(&mb.mhat, (size_t)w.max_n));
  A(alloc(&mb.sige, (size_t)w.max_n));
  A(alloc(&mb.U, (size_t)w.max_n));
  A(alloc(&mb.Mt, (size_t)w.max_n));
  A(alloc(&mb.Ut, (size_t)w.max_n));
  A(alloc(&mb.obs, (size_t)w.max_n));
  A(alloc(&mb.hist, (size_t)2 * 2048));
  A(alloc(&mb.sel, (size_t)8));
  if (e == cudaSuccess) e = cudaMemset(w.counters, 0, CNT_N * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(w.evals, 0, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(w.vis_append, 0, (size_t)w.max_v * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(w.vis_n, 0, (size_t)w.max_v * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? DAGS_E_NOMEM : DAGS_E_CUDA;
    cudaGetLastError();
    free_mp(c->mp);
    free_ws(w);
    for (void *p : {(void *)c->warp_masks, (void *)c->cand_ids, (void *)c->cand_n, (void *)c->cull_pose,
                    (void *)c->track_order, (void *)c->prev_count})
      if (p) cudaFree(p);
    delete c;
    return code;
  }
  *out = c;
  return DAGS_OK;
}

void dags_destroy(dags_ctx *ctx) {
  NvtxRange nv("dags_destroy");
  if (!ctx) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  ctx->timer.release();
  if (ctx->graph.exec) cudaGraphExecDestroy(ctx->graph.exec);
  if (ctx->graph.exec_chunk) cudaGraphExecDestroy(ctx->graph.exec_chunk);
  if (ctx->graph.cap) cudaStreamDestroy(ctx->graph.cap);
  if (ctx->graph_lm.exec) cudaGraphExecDestroy(ctx->graph_lm.exec);
  if (ctx->graph_lm.exec_chunk) cudaGraphExecDestroy(ctx->graph_lm.exec_chunk);
  if (ctx->graph_lm.cap) cudaStreamDestroy(ctx->graph_lm.cap);
  free_lm(ctx->lm);
  for (void *p : {(void *)ctx->warp_masks, (void *)ctx->cand_ids, (void *)ctx->cand_n, (void *)ctx->cull_pose,
                  (void *)ctx->track_order, (void *)ctx->prev_count})
    if (p) cudaFree(p);
  if (ctx->reg_partial) cudaFree(ctx->reg_partial);
  if (ctx->edge_partial) cudaFree(ctx->edge_partial);
  if (ctx->rel32) cudaFree(ctx->rel32);
  free_epi(ctx->epi);
  free_mp(ctx->mp);
  free_net(ctx->net);
  free_ws(ctx->ws);
  cudaSetDevice(cur);
  delete ctx;
}

int dags_eval_counting(dags_ctx *ctx, int32_t enable) {
  NvtxRange nv("dags_eval_counting");
  if (!ctx) return DAGS_E_INVAL;
  ctx->ws.count_evals = enable ? 1 : 0;
  return DAGS_OK;
}

int dags_eval_read(dags_ctx *ctx, int64_t *counts) {
  NvtxRange nv("dags_eval_read");
  if (!ctx || !counts) return DAGS_E_INVAL;
  if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) return DAGS_E_CUDA;
  unsigned long long c[4];
  if (cudaMemcpy(c, ctx->ws.evals, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return DAGS_E_CUDA;
  if (cudaMemset(ctx->ws.evals, 0, sizeof(c)) != cudaSuccess) return DAGS_E_CUDA;
  for (int k = 0; k < 4; ++k) counts[k] = (int64_t)c[k];
  return DAGS_OK;
}

int dags_sync_status(dags_ctx *ctx, int64_t *required_pairs) {
  NvtxRange nv("dags_sync_status");
  if (!ctx) return DAGS_E_INVAL;
  if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) return DAGS_E_CUDA;
  uint32_t cnt[CNT_N];
  if (cudaMemcpy(cnt, ctx->ws.counters, sizeof(cnt), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DAGS_E_CUDA;
  if (required_pairs) *required_pairs = (int64_t)((uint64_t)cnt[CNT_REQ_LO] | ((uint64_t)cnt[CNT_REQ_HI] << 32));
  const uint32_t st = cnt[CNT_STATUS];
  if (st) {
    uint32_t zero = 0;
    if (cudaMemcpy(ctx->ws.counters + CNT_STATUS, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess)
      return DAGS_E_CUDA;
  }
  if (st & kStatusCapacity) return DAGS_E_CAPACITY;
  if (st & kStatusTimeout) return DAGS_E_TIMEOUT;
  if (st & kStatusBounds) return DAGS_E_BOUNDS;
  return DAGS_OK;
}

int splat_forward(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, const double *poses,
                  int32_t n_views, const float *targets, const dags_raster_cfg *rcfg,
                  const dags_loss_cfg *lcfg, float *image, int32_t *last, double *loss, void *stream) {
  NvtxRange nv("splat_forward");
  int rc = common_args(ctx, gauss, n, cam, poses, n_views);
  if (rc) return rc;
  if (!image || !last || (loss && !targets)) return DAGS_E_INVAL;
  if (((uintptr_t)targets & 15u) != 0) return DAGS_E_INVAL;
  Raster r;
  Loss l;
  if ((rc = make_raster(cam, rcfg, &r)) || (rc = make_loss(lcfg, &l))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  ctx->fwd_image = nullptr;
  const Workspace &w = ctx->ws;
  const float4 *g4 = reinterpret_cast<const float4 *>(gauss);
  KernelTimer &tm = ctx->timer;
  int ev = tm.begin(DAGS_K_PREPROCESS, s);
  cudaError_t e = launch_preprocess(w, g4, n, poses, n_views, r, kGradWords, s);
  tm.end(ev, s);
  if (e == cudaSuccess && n > 0) {
    ev = tm.begin(DAGS_K_EMIT, s);
    e = launch_emit(w, n, n_views, r, s);
    tm.end(ev, s);
  }
  if (e == cudaSuccess) {
    ev = tm.begin(DAGS_K_RENDER_FWD, s);
    e = launch_render_fwd(w, n_views, n, r, l, reinterpret_cast<const float4 *>(targets), image, last, loss, s);
    tm.end(ev, s);
  }
  if (e != cudaSuccess) return DAGS_E_CUDA;
  ctx->fwd_image = image;
  ctx->fwd_last = last;
  ctx->fwd_gauss = gauss;
  ctx->fwd_n = n;
  ctx->fwd_views = n_views;
  ctx->fwd_w = cam->width;
  ctx->fwd_h = cam->height;
  ctx->fwd_tiles = r.T;
  return DAGS_OK;
}

int dags_copy_bins(dags_ctx *ctx, uint32_t *tile_start, int64_t n_start, uint32_t *ids, int64_t cap,
                   int64_t *n_pairs) {
  NvtxRange nv("dags_copy_bins");
  if (!ctx || !tile_start || !ctx->fwd_image || cap < 0 || (cap > 0 && !ids)) return DAGS_E_INVAL;
  if (n_start != (int64_t)ctx->fwd_views * ctx->fwd_tiles + 1) return DAGS_E_INVAL;
  int64_t req = 0;
  int st = dags_sync_status(ctx, &req);
  if (n_pairs) *n_pairs = req;
  if (st != DAGS_OK) return st;
  if (cudaMemcpy(tile_start, ctx->ws.tile_start, (size_t)n_start * sizeof(uint32_t), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return DAGS_E_CUDA;
  const int64_t m = req < cap ? req : cap;
  if (m > 0 && cudaMemcpy(ids, ctx->ws.sorted_ids, (size_t)m * sizeof(uint32_t), cudaMemcpyDeviceToHost) !=
                   cudaSuccess)
    return DAGS_E_CUDA;
  return DAGS_OK;
}

int splat_backward(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, const double *poses,
                   int32_t n_views, const float *targets, const dags_raster_cfg *rcfg,
                   const dags_loss_cfg *lcfg, const float *image, const int32_t *last, uint32_t grad_flags,
                   float *grad_gauss, double *grad_pose, void *stream) {
  NvtxRange nv("splat_backward");
  int rc = common_args(ctx, gauss, n, cam, poses, n_views);
  if (rc) return rc;
  if (!targets || !image || !last) return DAGS_E_INVAL;
  if ((grad_flags & ~(DAGS_GRAD_GAUSS | DAGS_GRAD_POSE)) || !grad_flags) return DAGS_E_INVAL;
  if ((grad_flags & DAGS_GRAD_GAUSS) && !grad_gauss && n > 0) return DAGS_E_INVAL;
  if ((grad_flags & DAGS_GRAD_POSE) && !grad_pose) return DAGS_E_INVAL;
  if (((uintptr_t)targets & 15u) != 0 || ((uintptr_t)grad_gauss & 15u) != 0) return DAGS_E_INVAL;
  if (ctx->fwd_image != image || ctx->fwd_last != last || ctx->fwd_gauss != gauss || ctx->fwd_n != n ||
      ctx->fwd_views != n_views || ctx->fwd_w != cam->width || ctx->fwd_h != cam->height)
    return DAGS_E_ORDER;
  Raster r;
  Loss l;
  if ((rc = make_raster(cam, rcfg, &r)) || (rc = make_loss(lcfg, &l))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const bool full = (grad_flags & DAGS_GRAD_GAUSS) != 0;
  KernelTimer &tm = ctx->timer;
  int ev = tm.begin(DAGS_K_RENDER_BWD, s);
  cudaError_t e = launch_render_bwd(ctx->ws, n_views, n, r, l, reinterpret_cast<const float4 *>(targets),
                                    image, last, full, s);
  tm.end(ev, s);
  if (e == cudaSuccess) {
    ev = tm.begin(DAGS_K_PREPROCESS_BWD, s);
    e = launch_preprocess_bwd(ctx->ws, reinterpret_cast<const float4 *>(gauss), n, n_views, r,
                              full ? grad_gauss : nullptr, (grad_flags & DAGS_GRAD_POSE) ? grad_pose : nullptr,
                              PoseStep(), s);
    tm.end(ev, s);
  }
  return cuda_status(e);
}

int splat_backward_upstream(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam,
                            const double *poses, int32_t n_views, const dags_raster_cfg *rcfg, const float *image,
                            const int32_t *last, const float *grad_image, uint32_t grad_flags, float *grad_gauss,
                            double *grad_pose, void *stream) {
  NvtxRange nv("splat_backward_upstream");
  int rc = common_args(ctx, gauss, n, cam, poses, n_views);
  if (rc) return rc;
  if (!image || !last || !grad_image) return DAGS_E_INVAL;
  if ((grad_flags & ~(DAGS_GRAD_GAUSS | DAGS_GRAD_POSE)) || !grad_flags) return DAGS_E_INVAL;
  if ((grad_flags & DAGS_GRAD_GAUSS) && !grad_gauss && n > 0) return DAGS_E_INVAL;
  if ((grad_flags & DAGS_GRAD_POSE) && !grad_pose) return DAGS_E_INVAL;
  if (((uintptr_t)grad_gauss & 15u) != 0) return DAGS_E_INVAL;
  if (ctx->fwd_image != image || ctx->fwd_last != last || ctx->fwd_gauss != gauss || ctx->fwd_n != n ||
      ctx->fwd_views != n_views || ctx->fwd_w != cam->width || ctx->fwd_h != cam->height)
    return DAGS_E_ORDER;
  Raster r;
  Loss l;
  if ((rc = make_raster(cam, rcfg, &r)) || (rc = make_loss(nullptr, &l))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const bool full = (grad_flags & DAGS_GRAD_GAUSS) != 0;
  KernelTimer &tm = ctx->timer;
  int ev = tm.begin(DAGS_K_RENDER_BWD, s);
  cudaError_t e = launch_render_bwd(ctx->ws, n_views, n, r, l, nullptr, image, last, full, s, grad_image);
  tm.end(ev, s);
  if (e == cudaSuccess) {
    ev = tm.begin(DAGS_K_PREPROCESS_BWD, s);
    e = launch_preprocess_bwd(ctx->ws, reinterpret_cast<const float4 *>(gauss), n, n_views, r,
                              full ? grad_gauss : nullptr, (grad_flags & DAGS_GRAD_POSE) ? grad_pose : nullptr,
                              PoseStep(), s);
    tm.end(ev, s);
  }
  return cuda_status(e);
}

void dags_default_gauss_adam_cfg(dags_gauss_adam_cfg *c) {
  if (!c) return;
  c->lr_mean = 1e-3f;
  c->lr_opacity = 0.05f;
  c->lr_quat = 1e-3f;
  c->lr_scale = 5e-3f;
  c->lr_colour = 2.5e-3f;
  c->beta1 = 0.9f;
  c->beta2 = 0.999f;
  c->eps = 1e-8f;
}

int gauss_adam_init(dags_ctx *ctx, const float *gauss, int64_t n, float *colour, float *adam_m, float *adam_v,
                    void *stream) {
  NvtxRange nv("gauss_adam_init");
  if (!ctx || n < 0 || (n > 0 && (!gauss || !colour || !adam_m || !adam_v))) return DAGS_E_INVAL;
  if ((((uintptr_t)gauss | (uintptr_t)colour | (uintptr_t)adam_m | (uintptr_t)adam_v) & 15u) != 0)
    return DAGS_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  return cuda_status(launch_gauss_adam_init(gauss, colour, adam_m, adam_v, n, s));
}

int gauss_adam_step(dags_ctx *ctx, float *gauss, int64_t n, float *colour, float *adam_m, float *adam_v,
                    const float *grad, int64_t step, const dags_gauss_adam_cfg *cfg, void *stream) {
  NvtxRange nv("gauss_adam_step");
  if (!ctx || n < 0 || step < 1 || (n > 0 && (!gauss || !colour || !adam_m || !adam_v || !grad)))
    return DAGS_E_INVAL;
  if ((((uintptr_t)gauss | (uintptr_t)colour | (uintptr_t)adam_m | (uintptr_t)adam_v | (uintptr_t)grad) & 15u) != 0)
    return DAGS_E_INVAL;
  dags_gauss_adam_cfg c;
  if (cfg) c = *cfg;
  else dags_default_gauss_adam_cfg(&c);
  const float rates[5] = {c.lr_mean, c.lr_opacity, c.lr_quat, c.lr_scale, c.lr_colour};
  for (float x : rates)
    if (!isfinite(x) || x < 0.f) return DAGS_E_INVAL;
  if (!(c.beta1 >= 0.f && c.beta1 < 1.f) || !(c.beta2 >= 0.f && c.beta2 < 1.f) || !(c.eps > 0.f)) return DAGS_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ev = ctx->timer.begin(DAGS_K_GAUSS_ADAM, s);
  const cudaError_t e = launch_gauss_adam(gauss, colour, adam_m, adam_v, grad, n, step, c, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

int pose_step(dags_ctx *ctx, double *poses, const double *grad, double *adam_state, int32_t n_views,
              const dags_pose_cfg *cfg, void *stream) {
  NvtxRange nv("pose_step");
  if (!ctx || !poses || !grad || !adam_state || n_views < 1 || n_views > ctx->ws.max_v) return DAGS_E_INVAL;
  dags_pose_cfg c;
  if (cfg) c = *cfg;
  else dags_default_pose_cfg(&c);
  for (int k = 0; k < 6; ++k)
    if (!isfinite(c.lr[k]) || c.lr[k] < 0) return DAGS_E_INVAL;
  if (!(c.beta1 >= 0 && c.beta1 < 1) || !(c.beta2 >= 0 && c.beta2 < 1) || !(c.eps > 0)) return DAGS_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ev = ctx->timer.begin(DAGS_K_POSE_STEP, s);
  const cudaError_t e = launch_pose_step(poses, grad, adam_state, n_views, c, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

}  // extern "C"

namespace {

// The tracking loop's view of the workspace: the fixed-capacity bucket
// layout (max_pairs / tiles slots per tile) and the frame's culled
// candidates.
Workspace track_workspace(const dags_ctx *ctx, const Raster &r) {
  Workspace w = ctx->ws;
  const int64_t cap = w.max_pairs / r.T;
  w.bucket_cap = (uint32_t)(cap < 0xFFFFFFFFll ? cap : 0xFFFFFFFFll);
  w.cand_ids = ctx->cand_ids;
  w.cand_n = ctx->cand_n;
  w.cull_pose = ctx->cull_pose;
  // the renders launch in an order ranked from the previous iteration's
  // counts (a permutation of the tiles whatever the counts; ranking this
  // iteration's would add a serial step before the forward)
  w.tile_order = ctx->track_order;
  w.order_next = ctx->track_order;
  w.prev_count = ctx->prev_count;
  return w;
}

// Enqueues one tracking iteration: projection and binning into the
// fixed-capacity buckets, the forward with loss, the pose-only adjoint, and
// the chain to the pose twist with the pose step in its last CTA (arguments
// checked by the caller). follows_iteration: the launch just before is the
// previous iteration's last kernel, in the same stream or captured graph.
int track_iteration(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, double *pose,
                    const float *targets, const dags_raster_cfg *rcfg, const dags_loss_cfg *lcfg,
                    const dags_pose_cfg *pcfg, double *adam_state, float *image, int32_t *last, double *loss,
                    double *grad_pose, bool follows_iteration, cudaStream_t s) {
  Raster r;
  Loss l;
  int rc;
  if ((rc = make_raster(cam, rcfg, &r)) || (rc = make_loss(lcfg, &l))) return rc;
  ctx->last_stream = s;
  // the tile buckets take the fixed-capacity layout: max_pairs / tiles slots
  // per tile, filled by the preprocess directly (no scan or emit launch)
  Workspace w = track_workspace(ctx, r);
  if (w.bucket_cap == 0) return DAGS_E_INVAL;
  const float4 *g4 = reinterpret_cast<const float4 *>(gauss);
  KernelTimer &tm = ctx->timer;
  // the pose path accumulates 2D-gradient words G2_U .. G2_Z: two float4
  int ev = tm.begin(DAGS_K_PREPROCESS, s);
  // after an iteration, the candidate list is three launches old and the
  // preprocess may load it before waiting for the pose step; after the
  // culling launch it may not
  cudaError_t e = launch_preprocess_direct(w, g4, n, pose, r, 8, follows_iteration, s);
  tm.end(ev, s);
  // the forward records, per warp, which list entries its pixels took; the
  // adjoint visits only those
  w.warp_masks = ctx->warp_masks;
  if (e == cudaSuccess) {
    ev = tm.begin(DAGS_K_RENDER_FWD, s);
    e = launch_render_fwd(w, 1, n, r, l, reinterpret_cast<const float4 *>(targets), image, last, loss, s);
    tm.end(ev, s);
  }
  if (e == cudaSuccess) {
    ev = tm.begin(DAGS_K_RENDER_BWD, s);
    e = launch_render_bwd(w, 1, n, r, l, reinterpret_cast<const float4 *>(targets), image, last, false, s);
    tm.end(ev, s);
  }
  if (e == cudaSuccess) {
    // the pose step runs in the last CTA of the preprocess backward
    PoseStep ps;
    ps.poses = pose;
    ps.state = adam_state;
    ps.cfg = *pcfg;
    ev = tm.begin(DAGS_K_PREPROCESS_BWD, s);
    e = launch_preprocess_bwd(w, g4, n, 1, r, nullptr, grad_pose, ps, s);
    tm.end(ev, s);
  }
  // the workspace's lists are in the fixed-bucket layout: no splat_backward
  // or dags_copy_bins may follow
  ctx->fwd_image = nullptr;
  if (e != cudaSuccess) return DAGS_E_CUDA;
  return DAGS_OK;
}

template <class T>
void key_put(unsigned char *key, size_t &len, const T &v) {
  if (len + sizeof(T) <= 512) { memcpy(key + len, &v, sizeof(T)); }
  len += sizeof(T);
}

}  // namespace

extern "C" {

int splat_track(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, double *pose,
                const float *targets, const dags_raster_cfg *rcfg, const dags_loss_cfg *lcfg,
                const dags_pose_cfg *pcfg, int32_t iters, double *adam_state, float *image, int32_t *last,
                double *loss, double *grad_pose, int32_t use_graph, void *stream) {
  NvtxRange nv("splat_track");
  if (!ctx || iters < 0 || !pose || !targets || !adam_state || !image || !last || !loss || !grad_pose)
    return DAGS_E_INVAL;
  int rc = common_args(ctx, gauss, n, cam, pose, 1);
  if (rc) return rc;
  dags_raster_cfg rc_v;
  dags_loss_cfg lc_v;
  dags_pose_cfg pc_v;
  if (rcfg) rc_v = *rcfg; else dags_default_raster_cfg(&rc_v);
  if (lcfg) lc_v = *lcfg; else dags_default_loss_cfg(&lc_v);
  if (pcfg) pc_v = *pcfg; else dags_default_pose_cfg(&pc_v);
  for (int k = 0; k < 6; ++k)
    if (!isfinite(pc_v.lr[k]) || pc_v.lr[k] < 0) return DAGS_E_INVAL;
  if (!(pc_v.beta1 >= 0 && pc_v.beta1 < 1) || !(pc_v.beta2 >= 0 && pc_v.beta2 < 1) || !(pc_v.eps > 0))
    return DAGS_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // the frame's culling at its starting pose (the iterations fall back to
  // every Gaussian if their pose leaves the culling bounds)
  {
    Raster r;
    if ((rc = make_raster(cam, &rc_v, &r))) return rc;
    if (ctx->track_order_tiles != r.T) {
      // a new image size: the first iteration renders in tile order
      if (launch_order_identity(ctx->track_order, r.T, s) != cudaSuccess) return DAGS_E_CUDA;
      ctx->track_order_tiles = r.T;
    }
    const int ev = ctx->timer.begin(DAGS_K_PREPROCESS, s);
    const cudaError_t e = launch_cull(track_workspace(ctx, r), reinterpret_cast<const float4 *>(gauss), n, pose, r, s);
    ctx->timer.end(ev, s);
    if (e != cudaSuccess) return DAGS_E_CUDA;
  }
  if (!use_graph || ctx->timer.on) {
    for (int k = 0; k < iters; ++k) {
      rc = track_iteration(ctx, gauss, n, cam, pose, targets, &rc_v, &lc_v, &pc_v, adam_state, image, last, loss,
                           grad_pose, k > 0, s);
      if (rc) return rc;
    }
    return DAGS_OK;
  }
  // Graph path: capture one iteration on a private stream (the caller's may be
  // the legacy default stream, which cannot be captured), keyed by every
  // argument, and replay it on the caller's stream.
  unsigned char key[512];
  size_t kl = 0;
  key_put(key, kl, gauss); key_put(key, kl, n); key_put(key, kl, *cam); key_put(key, kl, pose);
  key_put(key, kl, targets); key_put(key, kl, rc_v); key_put(key, kl, lc_v); key_put(key, kl, pc_v);
  key_put(key, kl, adam_state); key_put(key, kl, image); key_put(key, kl, last); key_put(key, kl, loss);
  key_put(key, kl, grad_pose);
  TrackGraph &g = ctx->graph;
  if (!g.exec || g.key_len != kl || memcmp(g.key, key, kl) != 0) {
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    if (g.exec_chunk) { cudaGraphExecDestroy(g.exec_chunk); g.exec_chunk = nullptr; }
    if (!g.cap && cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking) != cudaSuccess) return DAGS_E_CUDA;
    // order the capture after the caller's pending work on the workspace
    if (cudaStreamSynchronize(s) != cudaSuccess) return DAGS_E_CUDA;
    // one iteration, and a chunk of kTrackUnroll iterations: inside a chunk
    // each iteration's first kernel overlaps the previous one's drain
    // (programmatic dependent launch), which a graph boundary prevents
    for (int pass = 0; pass < 2; ++pass) {
      const int reps = pass == 0 ? 1 : kTrackUnroll;
      if (cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DAGS_E_CUDA;
      for (int k = 0; k < reps && rc == DAGS_OK; ++k)
        rc = track_iteration(ctx, gauss, n, cam, pose, targets, &rc_v, &lc_v, &pc_v, adam_state, image, last, loss,
                             grad_pose, k > 0, g.cap);
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(g.cap, &graph);
      if (rc != DAGS_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != DAGS_OK ? rc : DAGS_E_CUDA;
      }
      cudaGraphExec_t *dst = pass == 0 ? &g.exec : &g.exec_chunk;
      const cudaError_t ie = cudaGraphInstantiate(dst, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) { *dst = nullptr; return DAGS_E_CUDA; }
    }
    memcpy(g.key, key, kl < 512 ? kl : 512);
    g.key_len = kl;
  }
  ctx->last_stream = s;
  int left = iters;
  for (; left >= kTrackUnroll; left -= kTrackUnroll)
    if (cudaGraphLaunch(g.exec_chunk, s) != cudaSuccess) return DAGS_E_CUDA;
  for (; left > 0; --left)
    if (cudaGraphLaunch(g.exec, s) != cudaSuccess) return DAGS_E_CUDA;
  return DAGS_OK;
}

}  // extern "C"

namespace {

// The LM buffers, allocated by the first LM call on the ctx.
int ensure_lm(dags_ctx *ctx) {
  LmBuffers &b = ctx->lm;
  if (b.tan) return DAGS_OK;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(alloc(&b.tan, (size_t)ctx->ws.max_n * 9));
  A(alloc(&b.partial, (size_t)ctx->ws.max_tiles * DAGS_LM_NORMAL));
  A(alloc(&b.normal, (size_t)DAGS_LM_NORMAL));
  A(alloc(&b.pose_try, (size_t)12));
  A(lm_kernel_setup());
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_lm(b);
    return e == cudaErrorMemoryAllocation ? DAGS_E_NOMEM : DAGS_E_CUDA;
  }
  return DAGS_OK;
}

int make_lm_cfg(const dags_lm_cfg *in, dags_lm_cfg *c) {
  if (in) *c = *in;
  else dags_default_lm_cfg(c);
  if (!(c->mu0 >= 0.0) || !(c->mu_min >= 0.0) || !(c->mu_max >= c->mu_min) || !(c->down > 0.0) ||
      !(c->down <= 1.0) || !(c->up >= 1.0) || !(c->delta > 0.0) || !(c->floor >= 0.0) || !isfinite(c->mu_max) ||
      !isfinite(c->up) || !isfinite(c->delta) || !isfinite(c->floor) || !isfinite(c->mu0))
    return DAGS_E_INVAL;
  return DAGS_OK;
}

// Enqueues the normal equations of one view at `pose` (arguments checked).
// track: the LM loop's iteration, on the frame's culled candidates and the
// fixed-capacity tile buckets of the first-order loop (a cull must precede
// the first such iteration of a frame); follows_iteration: the launch just
// before is the previous iteration's last kernel.
int normal_core(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, const double *pose,
                const float *targets, const Raster &r, const Loss &l, float delta, double *normal, float *jac,
                float *image, int32_t *last, const LmFuse &fuse, bool track, bool follows_iteration,
                cudaStream_t s) {
  ctx->last_stream = s;
  ctx->fwd_image = nullptr;     // the workspace no longer holds a forward for splat_backward
  const Workspace w = track ? track_workspace(ctx, r) : ctx->ws;
  if (track && w.bucket_cap == 0) return DAGS_E_INVAL;
  const float4 *g4 = reinterpret_cast<const float4 *>(gauss);
  KernelTimer &tm = ctx->timer;
  int ev = tm.begin(DAGS_K_PREPROCESS, s);
  cudaError_t e = track ? launch_preprocess_direct(w, g4, n, pose, r, 0, follows_iteration, s)
                        : launch_preprocess(w, g4, n, pose, 1, r, 0, s);
  tm.end(ev, s);
  if (e == cudaSuccess && n > 0 && !track) {
    ev = tm.begin(DAGS_K_EMIT, s);
    e = launch_emit(w, n, 1, r, s);
    tm.end(ev, s);
  }
  if (e == cudaSuccess) {
    ev = tm.begin(DAGS_K_POSE_TANGENT, s);
    e = launch_pose_tangents(w, g4, n, r, ctx->lm.tan, ctx->num_sms, s);
    tm.end(ev, s);
  }
  if (e == cudaSuccess) {
    ev = tm.begin(DAGS_K_RENDER_JAC, s);
    e = launch_render_jac(w, r, l, delta, reinterpret_cast<const float4 *>(targets), ctx->lm.tan, ctx->lm.partial,
                          normal, jac, image, last, fuse, s);
    tm.end(ev, s);
  }
  (void)cam;
  return cuda_status(e);
}

int lm_iteration(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, double *pose,
                 const float *targets, const Raster &r, const Loss &l, const dags_lm_cfg &c, double *state,
                 bool follows_iteration, cudaStream_t s) {
  // the LM step runs in the last CTA of the Jacobian render
  LmFuse fuse;
  fuse.state = state;
  fuse.pose_try = ctx->lm.pose_try;
  fuse.pose_best = pose;
  fuse.cfg = c;
  return normal_core(ctx, gauss, n, cam, ctx->lm.pose_try, targets, r, l, (float)c.delta, ctx->lm.normal, nullptr,
                     nullptr, nullptr, fuse, true, follows_iteration, s);
}

}  // namespace

extern "C" {

void dags_default_lm_cfg(dags_lm_cfg *c) {
  if (!c) return;
  c->mu0 = 1e-2;
  c->mu_min = 1e-9;
  c->mu_max = 1e9;
  c->down = 0.1;
  c->up = 10.0;
  c->delta = 0.01;
  c->floor = 1e-9;
}

int splat_normal_equations(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam,
                           const double *pose, const float *targets, const dags_raster_cfg *rcfg,
                           const dags_loss_cfg *lcfg, double delta, double *normal, float *jac, float *image,
                           int32_t *last, void *stream) {
  NvtxRange nv("splat_normal_equations");
  int rc = common_args(ctx, gauss, n, cam, pose, 1);
  if (rc) return rc;
  if (!targets || !normal || !(delta > 0.0) || !isfinite(delta)) return DAGS_E_INVAL;
  if (((uintptr_t)targets & 15u) != 0 || ((uintptr_t)jac & 15u) != 0) return DAGS_E_INVAL;
  Raster r;
  Loss l;
  if ((rc = make_raster(cam, rcfg, &r)) || (rc = make_loss(lcfg, &l))) return rc;
  if ((rc = ensure_lm(ctx))) return rc;
  return normal_core(ctx, gauss, n, cam, pose, targets, r, l, (float)delta, normal, jac, image, last, LmFuse(),
                     false, false, (cudaStream_t)stream);
}

int lm_init(dags_ctx *ctx, const double *pose, const dags_lm_cfg *cfg, double *state, double *pose_try,
            void *stream) {
  NvtxRange nv("lm_init");
  if (!ctx || !pose || !state || !pose_try) return DAGS_E_INVAL;
  dags_lm_cfg c;
  int rc = make_lm_cfg(cfg, &c);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  return cuda_status(launch_lm_init(pose, state, pose_try, c.mu0, s));
}

int lm_pose_step(dags_ctx *ctx, const double *normal, const dags_lm_cfg *cfg, double *state, double *pose_try,
                 double *pose_best, void *stream) {
  NvtxRange nv("lm_pose_step");
  if (!ctx || !normal || !state || !pose_try || !pose_best) return DAGS_E_INVAL;
  dags_lm_cfg c;
  int rc = make_lm_cfg(cfg, &c);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ev = ctx->timer.begin(DAGS_K_LM_STEP, s);
  const cudaError_t e = launch_lm_step(normal, state, pose_try, pose_best, c, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

int splat_track_lm(dags_ctx *ctx, const float *gauss, int64_t n, const dags_camera *cam, double *pose,
                   const float *targets, const dags_raster_cfg *rcfg, const dags_loss_cfg *lcfg,
                   const dags_lm_cfg *lmcfg, int32_t iters, double *state, int32_t use_graph, void *stream) {
  NvtxRange nv("splat_track_lm");
  if (!ctx || iters < 0 || !pose || !targets || !state) return DAGS_E_INVAL;
  int rc = common_args(ctx, gauss, n, cam, pose, 1);
  if (rc) return rc;
  if (((uintptr_t)targets & 15u) != 0) return DAGS_E_INVAL;
  Raster r;
  Loss l;
  dags_lm_cfg c;
  if ((rc = make_raster(cam, rcfg, &r)) || (rc = make_loss(lcfg, &l)) || (rc = make_lm_cfg(lmcfg, &c))) return rc;
  if ((rc = ensure_lm(ctx))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  if (launch_lm_init(pose, state, ctx->lm.pose_try, c.mu0, s) != cudaSuccess) return DAGS_E_CUDA;
  // the frame's culling at its starting pose, as in the first-order loop
  // (an iteration whose pose leaves the culling bounds takes every Gaussian)
  if (ctx->track_order_tiles != r.T) {
    if (launch_order_identity(ctx->track_order, r.T, s) != cudaSuccess) return DAGS_E_CUDA;
    ctx->track_order_tiles = r.T;
  }
  {
    const int ev = ctx->timer.begin(DAGS_K_PREPROCESS, s);
    const cudaError_t e = launch_cull(track_workspace(ctx, r), reinterpret_cast<const float4 *>(gauss), n, pose, r, s);
    ctx->timer.end(ev, s);
    if (e != cudaSuccess) return DAGS_E_CUDA;
  }
  if (!use_graph || ctx->timer.on) {
    for (int k = 0; k < iters; ++k)
      if ((rc = lm_iteration(ctx, gauss, n, cam, pose, targets, r, l, c, state, k > 0, s))) return rc;
    return DAGS_OK;
  }
  dags_raster_cfg rc_v;
  dags_loss_cfg lc_v;
  if (rcfg) rc_v = *rcfg; else dags_default_raster_cfg(&rc_v);
  if (lcfg) lc_v = *lcfg; else dags_default_loss_cfg(&lc_v);
  unsigned char key[512];
  size_t kl = 0;
  key_put(key, kl, gauss); key_put(key, kl, n); key_put(key, kl, *cam); key_put(key, kl, pose);
  key_put(key, kl, targets); key_put(key, kl, rc_v); key_put(key, kl, lc_v); key_put(key, kl, c);
  key_put(key, kl, state);
  TrackGraph &g = ctx->graph_lm;
  if (!g.exec || g.key_len != kl || memcmp(g.key, key, kl) != 0) {
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    if (g.exec_chunk) { cudaGraphExecDestroy(g.exec_chunk); g.exec_chunk = nullptr; }
    if (!g.cap && cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking) != cudaSuccess) return DAGS_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DAGS_E_CUDA;
    // one iteration and a chunk of kTrackUnroll, as for the first-order loop
    for (int pass = 0; pass < 2; ++pass) {
      const int reps = pass == 0 ? 1 : kTrackUnroll;
      if (cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DAGS_E_CUDA;
      for (int k = 0; k < reps && rc == DAGS_OK; ++k)
        rc = lm_iteration(ctx, gauss, n, cam, pose, targets, r, l, c, state, k > 0, g.cap);
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(g.cap, &graph);
      if (rc != DAGS_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != DAGS_OK ? rc : DAGS_E_CUDA;
      }
      cudaGraphExec_t *dst = pass == 0 ? &g.exec : &g.exec_chunk;
      const cudaError_t ie = cudaGraphInstantiate(dst, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) { *dst = nullptr; return DAGS_E_CUDA; }
    }
    memcpy(g.key, key, kl < 512 ? kl : 512);
    g.key_len = kl;
  }
  ctx->last_stream = s;
  int left = iters;
  for (; left >= kTrackUnroll; left -= kTrackUnroll)
    if (cudaGraphLaunch(g.exec_chunk, s) != cudaSuccess) return DAGS_E_CUDA;
  for (; left > 0; --left)
    if (cudaGraphLaunch(g.exec, s) != cudaSuccess) return DAGS_E_CUDA;
  return DAGS_OK;
}

int splat_mp_consistency(dags_ctx *ctx, const float *gauss, int64_t n, const float *prev, const double *rel_pose,
                         float lambda, float *grad_gauss, double *loss, void *stream) {
  NvtxRange nv("splat_mp_consistency");
  if (!ctx || n < 0 || n > ctx->ws.max_n || (n > 0 && (!gauss || !prev)) || !isfinite(lambda) || lambda < 0.f)
    return DAGS_E_INVAL;
  if (((uintptr_t)gauss & 15u) != 0 || ((uintptr_t)prev & 15u) != 0 || ((uintptr_t)grad_gauss & 15u) != 0)
    return DAGS_E_INVAL;
  if (!ctx->reg_partial || !ctx->rel32) {
    cudaError_t a = ctx->reg_partial ? cudaSuccess
                                     : alloc(&ctx->reg_partial, (size_t)mp_consistency_blocks(ctx->ws.max_n) + 1);
    if (a == cudaSuccess && !ctx->rel32) a = alloc(&ctx->rel32, (size_t)12);
    if (a != cudaSuccess) {
      cudaGetLastError();
      return a == cudaErrorMemoryAllocation ? DAGS_E_NOMEM : DAGS_E_CUDA;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ev = ctx->timer.begin(DAGS_K_REGULARISER, s);
  const cudaError_t e = launch_mp_consistency(reinterpret_cast<const float4 *>(gauss),
                                              reinterpret_cast<const float4 *>(prev), n, rel_pose, lambda,
                                              grad_gauss, ctx->reg_partial, ctx->ws.counters + CNT_DONE_REG, loss,
                                              ctx->rel32, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

void dags_default_edge_cfg(dags_edge_cfg *c) {
  if (!c) return;
  c->edge_rel = 0.05f;
  c->huber = 0.05f;
  c->z_near = 0.2f;
  c->literal = 0;
}

int splat_edge_warp(dags_ctx *ctx, const dags_camera *cam, const float *depth_i, const float *depth_j,
                    const float *weight_j, const double *pose_i, const double *pose_j, const dags_edge_cfg *cfg,
                    float lambda, double *out, void *stream) {
  NvtxRange nv("splat_edge_warp");
  if (!ctx || !depth_i || !depth_j || !weight_j || !pose_i || !pose_j || !out || !isfinite(lambda) || lambda < 0.f)
    return DAGS_E_INVAL;
  int rc = check_camera(ctx, cam);
  if (rc) return rc;
  dags_edge_cfg c;
  if (cfg) c = *cfg;
  else dags_default_edge_cfg(&c);
  if (!(c.edge_rel > 0.f) || !(c.huber > 0.f) || !(c.z_near > 0.f) || !isfinite(c.edge_rel) || !isfinite(c.huber))
    return DAGS_E_INVAL;
  Raster r;
  if ((rc = make_raster(cam, nullptr, &r))) return rc;
  if (!ctx->edge_partial || !ctx->rel32) {
    cudaError_t a = ctx->edge_partial
                        ? cudaSuccess
                        : alloc(&ctx->edge_partial, (size_t)edge_warp_blocks((int64_t)ctx->ws.max_w * ctx->ws.max_h) * 13);
    if (a == cudaSuccess && !ctx->rel32) a = alloc(&ctx->rel32, (size_t)12);
    if (a != cudaSuccess) {
      cudaGetLastError();
      return a == cudaErrorMemoryAllocation ? DAGS_E_NOMEM : DAGS_E_CUDA;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ev = ctx->timer.begin(DAGS_K_REGULARISER, s);
  const cudaError_t e = launch_edge_warp(r, depth_i, depth_j, weight_j, pose_i, pose_j, c, lambda,
                                         ctx->edge_partial, ctx->ws.counters + CNT_DONE_REG, out, ctx->rel32, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

int epipolar_verify(dags_ctx *ctx, const dags_camera *cam, const double *pose_1, const double *pose_2,
                    const float *p1, const float *p2, const int32_t *gid, int64_t m, float *gauss, int64_t n,
                    uint8_t *labels, float eps, float m_static, float *d_out, float *dbar_out, void *stream) {
  NvtxRange nv("epipolar_verify");
  if (!ctx || !pose_1 || !pose_2 || m < 0 || n < 0 || n > ctx->ws.max_n || m > (int64_t)0x7FFFFFFF) return DAGS_E_INVAL;
  if (m > 0 && (!p1 || !p2 || !gid)) return DAGS_E_INVAL;
  if (n > 0 && (!gauss || !labels)) return DAGS_E_INVAL;
  if (!(eps > 0.f) || !isfinite(eps) || !(m_static >= 0.f && m_static <= 1.f)) return DAGS_E_INVAL;
  if (((uintptr_t)p1 & 7u) != 0 || ((uintptr_t)p2 & 7u) != 0 || ((uintptr_t)gauss & 15u) != 0) return DAGS_E_INVAL;
  int rc = check_camera(ctx, cam);
  if (rc) return rc;
  Raster r;
  if ((rc = make_raster(cam, nullptr, &r))) return rc;
  EpiBuffers &b = ctx->epi;
  if (n > b.cap_n || m > b.cap_m) {
    const int64_t cn = n > b.cap_n ? n : b.cap_n, cm = m > b.cap_m ? m : b.cap_m;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DAGS_E_CUDA;
    free_epi(b);
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    A(alloc(&b.count, (size_t)cn));
    A(alloc(&b.off, (size_t)cn));
    A(alloc(&b.block_sum, (size_t)epi_scan_blocks(cn) + 1));
    A(alloc(&b.rank, (size_t)cm));
    A(alloc(&b.vals, (size_t)cm));
    A(alloc(&b.dist, (size_t)cm));
    A(alloc(&b.F, (size_t)9));
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_epi(b);
      return e == cudaErrorMemoryAllocation ? DAGS_E_NOMEM : DAGS_E_CUDA;
    }
    b.cap_n = cn;
    b.cap_m = cm;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ev = ctx->timer.begin(DAGS_K_EPIPOLAR, s);
  const cudaError_t e = launch_epipolar(r, pose_1, pose_2, reinterpret_cast<const float2 *>(p1),
                                        reinterpret_cast<const float2 *>(p2), gid, m, reinterpret_cast<float4 *>(gauss),
                                        n, labels, eps, m_static, d_out ? d_out : b.dist, dbar_out, b,
                                        ctx->ws.counters + CNT_STATUS, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

void dags_default_mp_cfg(dags_mp_cfg *c) {
  if (!c) return;
  c->kappa_c = 0.05f;
  c->lam = 2.f;
  c->sigma_min = 0.005f;
  c->e_floor = 0.05f;
  c->sigma_g = 0.05f;
  c->sigma_c = 0.05f;
  c->lam_u = 1.f;
  c->eps = 1e-6f;
  c->alpha_min = 0.05f;
  c->alpha_max = 0.6f;
  c->rho = 0.5f;
  c->r_s = 2.f;
  c->sigma_w = 1.f;
  c->vis_tol = 0.1f;
  c->z_near = 0.2f;
  c->tau_floor = 0.5f;
  c->fusion_mode = 0;
  c->scales = 1;
}

int mp_update(dags_ctx *ctx, float *gauss, int64_t n, const dags_camera *cam, const double *pose,
              const float *targets, const float *image, const uint8_t *inst, const float *table,
              int32_t n_regions, const dags_mp_cfg *cfg, int32_t seg_refreshed, uint8_t *labels,
              double *stats, const float *mp_map, float *mp_pixel, void *stream) {
  NvtxRange nv("mp_update");
  int rc = common_args(ctx, gauss, n, cam, pose, 1);
  if (rc) return rc;
  if (!targets || !image || !inst || !table || !labels || !stats) return DAGS_E_INVAL;
  if (n_regions < 1 || n_regions > DAGS_MP_MAX_REGIONS) return DAGS_E_INVAL;
  if (((uintptr_t)targets & 15u) != 0 || ((uintptr_t)table & 7u) != 0) return DAGS_E_INVAL;
  dags_mp_cfg c;
  if (cfg) c = *cfg;
  else dags_default_mp_cfg(&c);
  if (!(c.r_s > 0.f) || !(c.sigma_w > 0.f) || !(c.sigma_g > 0.f) || !(c.sigma_c > 0.f) || !(c.e_floor > 0.f) ||
      !(c.alpha_min >= 0.f && c.alpha_min <= c.alpha_max && c.alpha_max <= 1.f) || !(c.rho >= 0.f && c.rho <= 1.f) ||
      c.fusion_mode < 0 || c.fusion_mode > 2 || c.r_s > 64.f || c.scales < 1 || c.scales > DAGS_MP_MAX_SCALES)
    return DAGS_E_INVAL;
  Raster r;
  if ((rc = make_raster(cam, nullptr, &r))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ev = ctx->timer.begin(DAGS_K_MP_GAUSS, s);
  const cudaError_t e = launch_mp_update(ctx->mp, gauss, n, pose, r, reinterpret_cast<const float4 *>(targets),
                                         image, inst, table, n_regions, c, seg_refreshed ? 1 : 0, labels, stats,
                                         mp_map, mp_pixel, ctx->ws.counters + CNT_STATUS, ctx->num_sms, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

void dags_default_sched_cfg(dags_sched_cfg *c) {
  if (!c) return;
  c->w_u = 0.5;
  c->w_r = 0.5;
  c->theta = 0.35;
  c->e_ref = 0.05;
  c->n_max = 10;
}

int semantic_trigger(dags_ctx *ctx, const double *stats, const dags_sched_cfg *cfg, int32_t seg_refreshed,
                     int32_t *state, double *score, void *stream) {
  NvtxRange nv("semantic_trigger");
  if (!ctx || !stats || !state) return DAGS_E_INVAL;
  dags_sched_cfg c;
  if (cfg) c = *cfg;
  else dags_default_sched_cfg(&c);
  if (!(c.w_u >= 0.0) || !(c.w_r >= 0.0) || !(fabs(c.w_u + c.w_r - 1.0) <= 1e-6) || !(c.e_ref > 0.0) ||
      c.n_max < 1 || !(c.theta == c.theta))
    return DAGS_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  return cuda_status(launch_semantic_trigger(stats, c, seg_refreshed, state, score, s));
}

int mpnet_features(dags_ctx *ctx, const float *image, const float *targets, const uint8_t *inst,
                   const float *table, int32_t n_regions, int32_t width, int32_t height, uint16_t *feats,
                   void *stream) {
  NvtxRange nv("mpnet_features");
  if (!ctx || !image || !targets || !inst || !table || !feats || width < 1 || height < 1) return DAGS_E_INVAL;
  if (n_regions < 1 || n_regions > DAGS_MP_MAX_REGIONS) return DAGS_E_INVAL;
  if (((uintptr_t)targets & 15u) != 0 || ((uintptr_t)feats & 15u) != 0 || ((uintptr_t)table & 7u) != 0)
    return DAGS_E_INVAL;
  const long long P = (long long)width * height;
  if (P > INT32_MAX) return DAGS_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ev = ctx->timer.begin(DAGS_K_MPNET, s);
  const cudaError_t e = launch_mpnet_features(image, reinterpret_cast<const float4 *>(targets), inst, table,
                                              n_regions, (int)P, feats, ctx->ws.counters + CNT_STATUS, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

int mpnet_infer(dags_ctx *ctx, const void *weights, const uint16_t *feats, int32_t batch, int32_t width,
                int32_t height, float *mp_out, uint16_t *acts, void *stream) {
  NvtxRange nv("mpnet_infer");
  if (!ctx || !weights || !feats || !mp_out || batch < 1 || width < 1 || height < 1) return DAGS_E_INVAL;
  if (((uintptr_t)feats & 15u) != 0 || ((uintptr_t)weights & 15u) != 0 || ((uintptr_t)acts & 15u) != 0)
    return DAGS_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const int ev = ctx->timer.begin(DAGS_K_MPNET, s);
  const cudaError_t e = launch_mpnet_forward(weights, feats, batch, width, height, mp_out, acts,
                                             ctx->ws.counters + CNT_STATUS, ctx->num_sms, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

int mpnet_train_step(dags_ctx *ctx, void *weights, float *master, float *adam_m, float *adam_v, int32_t step,
                     const uint16_t *feats, const float *target, int32_t batch, int32_t width, int32_t height,
                     float lr, double *loss, float *grad_out, void *stream) {
  NvtxRange nv("mpnet_train_step");
  if (!ctx || !weights || !master || !adam_m || !adam_v || !feats || !target || !loss) return DAGS_E_INVAL;
  if (batch < 1 || width < 1 || height < 1 || step < 1 || !isfinite(lr) || lr < 0.f) return DAGS_E_INVAL;
  if (((uintptr_t)feats & 15u) != 0 || ((uintptr_t)weights & 15u) != 0) return DAGS_E_INVAL;
  const long long npix = (long long)batch * width * height;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  MpnetScratch &sc = ctx->net;
  if (sc.cap < npix) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    free_net(sc);
    e = alloc(&sc.y, (size_t)npix);
    if (e == cudaSuccess) e = alloc(&sc.acts, (size_t)npix * DAGS_MPNET_ACT_WORDS);
    if (e == cudaSuccess) e = alloc(&sc.dz2, (size_t)npix * 32);
    if (e == cudaSuccess) e = alloc(&sc.grad, DAGS_MPNET_PARAMS);
    if (e == cudaSuccess) e = alloc(&sc.inv_n, 2);
    if (e != cudaSuccess) {
      free_net(sc);
      cudaGetLastError();
      return DAGS_E_NOMEM;
    }
    sc.cap = npix;
  }
  const int ev = ctx->timer.begin(DAGS_K_MPNET_TRAIN, s);
  cudaError_t e = launch_mpnet_train(weights, master, adam_m, adam_v, step, feats, target, batch, width, height, lr,
                                     loss, sc, ctx->ws.counters + CNT_STATUS, ctx->num_sms, s);
  if (e == cudaSuccess && grad_out)
    e = cudaMemcpyAsync(grad_out, sc.grad, DAGS_MPNET_PARAMS * sizeof(float), cudaMemcpyDeviceToDevice, s);
  ctx->timer.end(ev, s);
  return cuda_status(e);
}

int dags_selftest_timeout(dags_ctx *ctx, int64_t spins, void *stream) {
  NvtxRange nv("dags_selftest_timeout");
  if (!ctx || spins < 0 || spins > (1ll << 24)) return DAGS_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  return cuda_status(launch_selftest_wait(ctx->ws.counters + CNT_STATUS, (long long)spins, s));
}

int dags_timing_enable(dags_ctx *ctx, int enable) {
  NvtxRange nv("dags_timing_enable");
  if (!ctx) return DAGS_E_INVAL;
  int rc = DAGS_OK;
  if (!enable && ctx->timer.used) rc = ctx->timer.collect();
  ctx->timer.on = enable != 0;
  return rc;
}

int dags_timing_read(dags_ctx *ctx, double *ms, int64_t *launches, int32_t count) {
  NvtxRange nv("dags_timing_read");
  if (!ctx || count < 0 || (count > 0 && (!ms || !launches))) return DAGS_E_INVAL;
  const int rc = ctx->timer.collect();
  if (rc != DAGS_OK) return rc;
  for (int k = 0; k < count && k < DAGS_KERNEL_COUNT; ++k) {
    ms[k] = ctx->timer.ms[k];
    launches[k] = ctx->timer.launches[k];
    ctx->timer.ms[k] = 0.0;
    ctx->timer.launches[k] = 0;
  }
  for (int k = DAGS_KERNEL_COUNT; k < count; ++k) { ms[k] = 0.0; launches[k] = 0; }
  return DAGS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free forward. The paper has no counterpart: this serves callers
// that must not allocate device memory once they are running (a real-time
// pipeline that forbids allocation after start-up, a plugin whose host owns
// all device memory). Its workspace is one file-scope device array of fixed
// size, shared by every call in the process; each GPU that loads the library
// holds it until the process exits.
namespace {

constexpr int64_t kStaticMaxN = 16384;
constexpr int kStaticMaxW = 256, kStaticMaxH = 256;
constexpr int64_t kStaticMaxPairs = 131072;
constexpr int kStaticTiles = (kStaticMaxW / kTile) * (kStaticMaxH / kTile);

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
// Regions, in order; the first four must be zero when a call starts.
constexpr size_t kOffCount = 0;
constexpr size_t kOffCursor = kOffCount + al256(kStaticTiles * 4);
constexpr size_t kOffVisAppend = kOffCursor + al256(kStaticTiles * 4);
constexpr size_t kOffCounters = kOffVisAppend + al256(4);
constexpr size_t kZeroBytes = kOffCounters + al256(CNT_N * 4);
constexpr size_t kOffStart = kZeroBytes;
constexpr size_t kOffOrder = kOffStart + al256((kStaticTiles + 1) * 4);
constexpr size_t kOffLossPartial = kOffOrder + al256(kStaticTiles * 4);
constexpr size_t kOffVisN = kOffLossPartial + al256(kStaticTiles * 8);
constexpr size_t kOffPose32 = kOffVisN + al256(4);
constexpr size_t kOffRec2d = kOffPose32 + al256(12 * 4);
constexpr size_t kOffRecLo = kOffRec2d + al256(kStaticMaxN * 3 * 16);
constexpr size_t kOffRect = kOffRecLo + al256(kStaticMaxN * 8);
constexpr size_t kOffGrad2d = kOffRect + al256(kStaticMaxN * 8);
constexpr size_t kOffVisIds = kOffGrad2d + al256(kStaticMaxN * kGradWords * 4);
constexpr size_t kOffKeys = kOffVisIds + al256(kStaticMaxN * 4);
constexpr size_t kOffKeysTmp = kOffKeys + al256(kStaticMaxPairs * 8);
constexpr size_t kOffSorted = kOffKeysTmp + al256(kStaticMaxPairs * 8);
constexpr size_t kStaticBytes = kOffSorted + al256(kStaticMaxPairs * 4);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Per-device device address of g_static_scratch (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory), with
// the context it was resolved in: a device reset or a new primary context
// loads the module again, and the address is then resolved again.
std::mutex g_static_mu;
unsigned char *g_static_addr[256] = {};
CUcontext g_static_ctx[256] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

int static_scratch(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return DAGS_E_CUDA;
  // the runtime makes the device's primary context current; its handle
  // comes from the driver entry point (no link against the driver library)
  static CtxGetCurrentFn get_current = nullptr;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!get_current) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return DAGS_E_CUDA;
    }
    get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
  }
  CUcontext cur = nullptr;
  if (get_current(&cur) != CUDA_SUCCESS) return DAGS_E_CUDA;
  if (!cur) {
    // no context current yet: cudaSetDevice initialises the primary context
    if (cudaSetDevice(dev) != cudaSuccess || get_current(&cur) != CUDA_SUCCESS || !cur) {
      cudaGetLastError();
      return DAGS_E_CUDA;
    }
  }
  if (!g_static_addr[dev] || g_static_ctx[dev] != cur) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return DAGS_E_CUDA;
    }
    g_static_addr[dev] = static_cast<unsigned char *>(p);
    g_static_ctx[dev] = cur;
  }
  *out = g_static_addr[dev];
  return DAGS_OK;
}

// status[0]: the call's outcome from the array's status word and pair count
// (capacity first, then a failed index check of a DAGS_CHECK build);
// status[1]: the pairs the call needed.
__global__ void static_status_kernel(const uint32_t *counters, int64_t *status, int64_t max_pairs) {
  const uint64_t req = (uint64_t)counters[CNT_REQ_LO] | ((uint64_t)counters[CNT_REQ_HI] << 32);
  const uint32_t st = counters[CNT_STATUS];
  int64_t code = DAGS_OK;
  if ((st & kStatusCapacity) || req > (uint64_t)max_pairs) code = DAGS_E_CAPACITY;
  else if (st & kStatusBounds) code = DAGS_E_BOUNDS;
  status[0] = code;
  status[1] = (int64_t)req;
}

}  // namespace

extern "C" int splat_forward_static(const float *gauss, int64_t n, const dags_camera *cam, const double *pose,
                                    const float *targets, const dags_raster_cfg *rcfg, const dags_loss_cfg *lcfg,
                                    float *image, int32_t *last, double *loss, int64_t *status, void *stream) {
  NvtxRange nv("splat_forward_static");
  if (n < 0 || n > kStaticMaxN || (n > 0 && !gauss) || !cam || !pose || !image || !last || (loss && !targets))
    return DAGS_E_INVAL;
  if (cam->width <= 0 || cam->height <= 0 || cam->width > kStaticMaxW || cam->height > kStaticMaxH)
    return DAGS_E_INVAL;
  if (!finite_pos(cam->fx) || !finite_pos(cam->fy) || !isfinite(cam->cx) || !isfinite(cam->cy))
    return DAGS_E_INVAL;
  if (((uintptr_t)gauss & 15u) != 0 || ((uintptr_t)targets & 15u) != 0) return DAGS_E_INVAL;
  Raster r;
  Loss l;
  int rc = make_raster(cam, rcfg, &r);
  if (rc) return rc;
  if ((rc = make_loss(lcfg, &l))) return rc;
  unsigned char *base = nullptr;
  if ((rc = static_scratch(&base))) return rc;
  Workspace w;
  w.max_n = kStaticMaxN;
  w.max_w = kStaticMaxW;
  w.max_h = kStaticMaxH;
  w.max_v = 1;
  w.max_tiles = kStaticTiles;
  w.max_pairs = kStaticMaxPairs;
  {
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      w.band = sms;
  }
  w.tile_count = reinterpret_cast<uint32_t *>(base + kOffCount);
  w.tile_cursor = reinterpret_cast<uint32_t *>(base + kOffCursor);
  w.vis_append = reinterpret_cast<uint32_t *>(base + kOffVisAppend);
  w.counters = reinterpret_cast<uint32_t *>(base + kOffCounters);
  w.tile_start = reinterpret_cast<uint32_t *>(base + kOffStart);
  w.tile_order = reinterpret_cast<uint32_t *>(base + kOffOrder);
  w.loss_partial = reinterpret_cast<double *>(base + kOffLossPartial);
  w.vis_n = reinterpret_cast<uint32_t *>(base + kOffVisN);
  w.pose32 = reinterpret_cast<float *>(base + kOffPose32);
  w.rec2d = reinterpret_cast<float4 *>(base + kOffRec2d);
  w.rec_lo = reinterpret_cast<float2 *>(base + kOffRecLo);
  w.rect = reinterpret_cast<uint2 *>(base + kOffRect);
  w.grad2d = reinterpret_cast<float *>(base + kOffGrad2d);
  w.vis_ids = reinterpret_cast<uint32_t *>(base + kOffVisIds);
  w.keys = reinterpret_cast<uint64_t *>(base + kOffKeys);
  w.keys_tmp = reinterpret_cast<uint64_t *>(base + kOffKeysTmp);
  w.sorted_ids = reinterpret_cast<uint32_t *>(base + kOffSorted);
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear the counters
  cudaError_t e = cudaMemsetAsync(base, 0, kZeroBytes, s);
  if (e == cudaSuccess) e = launch_preprocess(w, reinterpret_cast<const float4 *>(gauss), n, pose, 1, r, kGradWords, s);
  if (e == cudaSuccess && n > 0) e = launch_emit(w, n, 1, r, s);
  if (e == cudaSuccess)
    e = launch_render_fwd(w, 1, n, r, l, reinterpret_cast<const float4 *>(targets), image, last, loss, s);
  if (e == cudaSuccess && status) {
    static_status_kernel<<<1, 1, 0, s>>>(w.counters, status, kStaticMaxPairs);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? DAGS_OK : DAGS_E_CUDA;
}
