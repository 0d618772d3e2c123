// Internal declarations shared by the CUDA translation units of libdags.so.
// Not part of the public ABI (include/dags.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dags.h"

namespace dags {

constexpr int kTile = 16;               // tile edge in pixels
constexpr int kTilePix = kTile * kTile; // pixels (= threads) per render CTA
constexpr int kGradWords = 12;          // per (view, Gaussian) 2D gradient slots
constexpr int kSortSmallCap = 1024;     // tile lists up to this length are sorted by the render CTA
constexpr int kPrepBlock = 128;         // threads per preprocess / emit CTA
constexpr int kBwdPrepBlock = 128;      // threads per preprocess-backward CTA
constexpr int kMaskGroups = 32;         // list groups of 32 entries with a recorded forward mask (1024 entries)

// Status word bits (device).
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;
constexpr uint32_t kStatusBounds = 4u;

// Index checks of a DAGS_CHECK build (nvcc -DDAGS_CHECK=1): a failed check
// records kStatusBounds in the status word and the access is skipped (the
// caller takes the `false` branch). In the normal build the checks compile
// away to `true`.
#ifdef DAGS_CHECK
__device__ __forceinline__ bool dags_in_bounds(bool ok, uint32_t *status) {
  if (!ok) atomicOr(status, kStatusBounds);
  return ok;
}
#define DAGS_IN_BOUNDS(cond, status) dags_in_bounds((cond), (status))
#else
#define DAGS_IN_BOUNDS(cond, status) true
#endif

// 2D gradient slots per (view, Gaussian).
enum { G2_U = 0, G2_V, G2_A, G2_B, G2_C, G2_Z, G2_O, G2_R, G2_G, G2_BL };

// Counters in the workspace's counter array.
enum {
  CNT_DONE_PREP = 0,   // CTAs of the preprocess kernel that finished
  CNT_DONE_RENDER,     // CTAs of the forward render that finished
  CNT_DONE_BWDPREP,    // CTAs of the preprocess backward that finished
  CNT_DONE_REG,        // CTAs of the regulariser that finished
  CNT_STATUS,          // status bits
  CNT_PAD,             // (keeps the 64-bit requirement 8-byte aligned)
  CNT_REQ_LO,          // pairs required by the last forward (low / high word)
  CNT_REQ_HI,
  CNT_RECULL,          // tracking loop: the next preprocess re-culls at its pose
  CNT_N
};

// Projected Gaussian, 3 float4 per (view, Gaussian):
//   r0 = {u, v, ex, ey}      centre (px) and half extents of the bounding box
//                            of the alpha >= alpha_min ellipse
//   r1 = {a', b', c', lo}    exponent p(d) = a' dx^2 + b' dx dy + c' dy^2 + lo
//                            in log2 units: alpha = min(alpha_max, 2^p),
//                            a' = -a log2(e) / 2, b' = -b log2(e),
//                            c' = -c log2(e) / 2 for the conic (a, b, c), and
//                            lo = log2(opacity)
//   r2 = {z, M, rg, bl}      depth, motion probability, colour as the
//                            record's BF16 bit patterns
// The centre (u, v) is computed in FP64 from the FP64 pose and stored as
// u = r0.x + lo.x, v = r0.y + lo.y with the FP32 remainders in rec_lo, so
// that a pixel offset (u - px) = (r0.x - px) + lo.x carries a relative
// rounding of 2^-24 of the offset rather than an absolute ulp(u).
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

struct Workspace {
  int64_t max_n = 0;
  int max_w = 0, max_h = 0, max_v = 0, max_tiles = 0;
  int64_t max_pairs = 0;
  int bwd_prep_blocks = 0;
  int band = 1;                   // CTAs per dispatch round of the renders (the SM count)
  float4 *rec2d = nullptr;        // [V][N][3], see above
  float2 *rec_lo = nullptr;       // [V][N] FP32 remainders of the FP64 centre
  uint2 *rect = nullptr;          // [V][N]: {x0 | x1 << 16, y0 | y1 << 16}, candidate tiles [x0, x1) x [y0, y1)
  float *grad2d = nullptr;        // [V][N][kGradWords]
  uint32_t *tile_count = nullptr; // [V * T]
  uint32_t *tile_start = nullptr; // [V * T + 1]
  uint32_t *tile_cursor = nullptr;// [V * T]
  uint64_t *keys = nullptr;       // [max_pairs]: depth bits << 32 | Gaussian id
  uint64_t *keys_tmp = nullptr;   // [max_pairs]: merge ping-pong
  uint32_t *sorted_ids = nullptr; // [max_pairs]
  uint32_t *tile_order = nullptr; // [V * T] launch order of the renders (length-ranked, band-reversed)
  double *loss_partial = nullptr; // [V * T] per-tile loss sums (FP64)
  float2 *pose_partial = nullptr; // [bwd_prep_blocks][V][6] compensated (high, low) CTA sums
  float *pose32 = nullptr;        // [V][12] FP32 copy of the poses of the last forward
  uint32_t *vis_ids = nullptr;    // [V][N] ids of the Gaussians with a non-empty candidate range
  uint32_t *vis_append = nullptr; // [V] append cursors (zero between calls)
  uint32_t *vis_n = nullptr;      // [V] visible counts of the last forward
  uint32_t *counters = nullptr;   // [CNT_N]
  // Evaluation counts (when count_evals is set): pixel-Gaussian exponents
  // evaluated and contributions (alpha >= alpha_min) of the forward and the
  // backward compositing, [fwd eval, fwd contrib, bwd eval, bwd contrib].
  unsigned long long *evals = nullptr;
  int count_evals = 0;
  // Fixed-capacity layout of the tile buckets (the tracking loop, one view):
  // when non-zero, tile t's keys and sorted ids occupy [t cap, t cap +
  // min(count_t, cap)) and tile_count holds the counts; otherwise the
  // buckets are packed at tile_start offsets.
  uint32_t bucket_cap = 0;
  // Per tile, warp and 32-entry group of the first kMaskGroups groups: the
  // entries at least one pixel of the warp took in the forward (one bit
  // each), for the adjoint of the same iteration; null: not recorded.
  uint32_t *warp_masks = nullptr;   // [max_tiles][kMaskGroups][8]
  // Per-frame culling of the tracking loop: the candidates of the frame's
  // starting pose (cull_pose, FP32 3x4) and their count; null: no culling.
  uint32_t *cand_ids = nullptr;     // [max_n]
  uint32_t *cand_n = nullptr;       // [1]
  float *cull_pose = nullptr;       // [12]
  // Render order of the tracking loop: tile_order is ranked from the
  // previous iteration's counts (prev_count, written by the forward), by an
  // extra CTA of the pose chain, into order_next for the next iteration.
  uint32_t *prev_count = nullptr;   // [max_tiles]
  uint32_t *order_next = nullptr;   // [max_tiles]
};

// The list range [s, e) of tile t in the workspace's bucket layout.
__device__ __forceinline__ void tile_range(const Workspace &ws, int t, uint32_t &s, uint32_t &e) {
  if (ws.bucket_cap) {
    s = (uint32_t)t * ws.bucket_cap;
    e = s + min(ws.tile_count[t], ws.bucket_cap);
  } else {
    s = ws.tile_start[t];
    e = ws.tile_start[t + 1];
  }
}

// Adds a lane's evaluation counts to the workspace totals (one atomic per
// warp and counter); called by whole warps.
__device__ __forceinline__ void add_eval_counts(const Workspace &ws, int which, unsigned ne, unsigned nc) {
  if (!ws.count_evals) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ne += __shfl_xor_sync(0xffffffffu, ne, o);
    nc += __shfl_xor_sync(0xffffffffu, nc, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(ws.evals + 2 * which, (unsigned long long)ne);
    atomicAdd(ws.evals + 2 * which + 1, (unsigned long long)nc);
  }
}

// Per-call constants handed to kernels by value.
struct Raster {
  float fx, fy, cx, cy;
  int W, H, tiles_x, tiles_y, T;   // T = tiles per view
  float alpha_min, alpha_max, t_min, dilation, z_near, limx, limy;
  float log2_alpha_min;
};

struct Loss {
  float lambda_pho, lambda_depth, o_eps;
  int weight_mode, weight_grad;
};

// Optional pose step fused into the end of the preprocess backward.
struct PoseStep {
  double *poses = nullptr;     // [V][12], in/out; nullptr: no step
  double *state = nullptr;     // [V][13]
  dags_pose_cfg cfg;
};

// ---- launchers (defined in the .cu files) ----
cudaError_t launch_preprocess(const Workspace &ws, const float4 *gauss, int64_t n, const double *poses,
                              int views, const Raster &r, int zero_grad_words, cudaStream_t s);
cudaError_t launch_emit(const Workspace &ws, int64_t n, int views, const Raster &r, cudaStream_t s);
// Projection and binning of one view into fixed-capacity tile buckets
// (ws.bucket_cap > 0) over the frame's culled candidates: keys written
// directly (no scan or emit launch). prefetch: the candidate list was
// written two or more launches before this one (not by the launch just
// before it), so the kernel may read it before its pdl_wait.
cudaError_t launch_preprocess_direct(const Workspace &ws, const float4 *gauss, int64_t n, const double *pose,
                                     const Raster &r, int zero_grad_words, bool prefetch, cudaStream_t s);
// The frame's culling: candidates of `pose` into ws.cand_ids / cand_n and
// the pose into ws.cull_pose (the tracking loop's preprocess uses them while
// its pose stays within the culling bounds).
cudaError_t launch_cull(const Workspace &ws, const float4 *gauss, int64_t n, const double *pose, const Raster &r,
                        cudaStream_t s);
// The identity render order of `tiles` tiles (the tracking loop's first
// iteration at a new image size).
cudaError_t launch_order_identity(uint32_t *order, int tiles, cudaStream_t s);
cudaError_t launch_render_fwd(const Workspace &ws, int views, int64_t n, const Raster &r, const Loss &l,
                              const float4 *targets, float *image, int32_t *last, double *loss,
                              cudaStream_t s);
// upstream (V x 6 x P, or null): a caller's gradients of the composited
// channels (C_r, C_g, C_b, D, O, R_MP) used in place of the loss's
cudaError_t launch_render_bwd(const Workspace &ws, int views, int64_t n, const Raster &r, const Loss &l,
                              const float4 *targets, const float *image, const int32_t *last, bool full,
                              cudaStream_t s, const float *upstream = nullptr);
cudaError_t launch_preprocess_bwd(const Workspace &ws, const float4 *gauss, int64_t n, int views,
                                  const Raster &r, float *grad_gauss, double *grad_pose, const PoseStep &ps,
                                  cudaStream_t s);
cudaError_t launch_pose_step(double *poses, const double *grad, double *state, int views,
                             const dags_pose_cfg &cfg, cudaStream_t s);


// Mapping optimiser (gauss_adam.cu).
cudaError_t launch_gauss_adam_init(const float *gauss, float *colour, float *m, float *v, int64_t n, cudaStream_t s);
cudaError_t launch_gauss_adam(float *gauss, float *colour, float *m, float *v, const float *grad, int64_t n,
                              int64_t step, const dags_gauss_adam_cfg &c, cudaStream_t s);

// Levenberg-Marquardt pose refinement (lm.cu).
struct LmBuffers {
  float4 *tan = nullptr;      // [max_n][9] twist tangents of the projected records (view 0)
  float *partial = nullptr;   // [max_tiles][28] tile partials of the normal equations
  double *normal = nullptr;   // [28] the loop's normal equations
  double *pose_try = nullptr; // [12] the loop's linearisation point
};
cudaError_t lm_kernel_setup();
cudaError_t launch_pose_tangents(const Workspace &ws, const float4 *gauss, int64_t n, const Raster &r, float4 *tan,
                                 int num_sms, cudaStream_t s);
// Optional LM step fused into the last CTA of the Jacobian render.
struct LmFuse {
  double *state = nullptr;      // nullptr: no step
  double *pose_try = nullptr;
  double *pose_best = nullptr;
  dags_lm_cfg cfg;
};
cudaError_t launch_render_jac(const Workspace &ws, const Raster &r, const Loss &l, float delta,
                              const float4 *targets, const float4 *tan, float *partial, double *normal, float *jac,
                              float *image, int32_t *last, const LmFuse &fuse, cudaStream_t s);
cudaError_t launch_lm_init(const double *pose, double *state, double *pose_try, double mu0, cudaStream_t s);
cudaError_t launch_lm_step(const double *normal, double *state, double *pose_try, double *pose_best,
                           const dags_lm_cfg &c, cudaStream_t s);

// MP motion-consistency regulariser (regular.cu).
int64_t mp_consistency_blocks(int64_t n);
int64_t edge_warp_blocks(int64_t pixels);
cudaError_t launch_edge_warp(const Raster &r, const float *Di, const float *Dj, const float *wj, const double *pose_i,
                             const double *pose_j, const dags_edge_cfg &c, float lam, double *partial, uint32_t *done,
                             double *out, float *tji, cudaStream_t s);
cudaError_t launch_mp_consistency(const float4 *gauss, const float4 *prev, int64_t n, const double *rel, float lam,
                                  float *grad, double *partial, uint32_t *done, double *loss, float *rel32,
                                  cudaStream_t s);

// Epipolar verification (epipolar.cu): buffers owned by the ctx, grown on
// demand.
struct EpiBuffers {
  uint32_t *count = nullptr, *off = nullptr;   // [cap_n]
  uint32_t *block_sum = nullptr;               // [scan blocks of cap_n]
  uint32_t *rank = nullptr;                    // [cap_m]
  float *vals = nullptr, *dist = nullptr;      // [cap_m]
  double *F = nullptr;                         // [9]
  int64_t cap_n = 0, cap_m = 0;
};
int64_t epi_scan_blocks(int64_t n);
cudaError_t launch_epipolar(const Raster &r, const double *pose_1, const double *pose_2, const float2 *p1,
                            const float2 *p2, const int32_t *gid, int64_t m, float4 *gauss, int64_t n,
                            uint8_t *labels, float eps, float m_static, float *dist, float *dbar, const EpiBuffers &b,
                            uint32_t *status, cudaStream_t s);

cudaError_t launch_mpnet_forward(const void *weights, const uint16_t *feats, int batch, int W, int H, float *out,
                                 uint16_t *acts, uint32_t *status, int num_sms, cudaStream_t s);

// Scratch of a training step of the MP network (owned by the ctx).
struct MpnetScratch {
  float *y = nullptr;        // [pixels]
  uint16_t *acts = nullptr;  // [pixels][96] bf16
  uint16_t *dz2 = nullptr;   // [pixels][32] bf16
  float *grad = nullptr;     // [10881]
  float *inv_n = nullptr;    // [2]: 1 / valid pixels, valid count
  long long cap = 0;         // pixels
};
cudaError_t launch_selftest_wait(uint32_t *status, long long limit, cudaStream_t s);
cudaError_t launch_mpnet_train(void *weights, float *master, float *adam_m, float *adam_v, int step,
                               const uint16_t *feats, const float *target, int batch, int W, int H, float lr,
                               double *loss, const MpnetScratch &sc, uint32_t *status, int num_sms, cudaStream_t s);

// Buffers of the MP update (owned by the ctx).
// Floats of the association pyramid's levels 1 .. DAGS_MP_MAX_SCALES-1 for
// a W x H frame: three maps (M_p, e, rendered depth) per level, level s of
// (W >> s) x (H >> s) pixels.
inline size_t mp_pyramid_floats(int W, int H) {
  size_t t = 0;
  for (int s = 1; s < DAGS_MP_MAX_SCALES; ++s) t += 3 * (size_t)(W >> s) * (size_t)(H >> s);
  return t > 0 ? t : 1;
}

struct MpBuffers {
  float *e = nullptr;                 // [max_w * max_h]
  float *mpf = nullptr;               // [max_w * max_h] fused per-pixel M_p
  float *pyr = nullptr;               // [mp_pyramid_floats] levels 1.. of the association pyramid
  double *acc = nullptr;              // [DAGS_MP_MAX_REGIONS * 4]
  float *mhat = nullptr, *sige = nullptr, *U = nullptr, *Mt = nullptr, *Ut = nullptr;  // [max_n]
  uint8_t *obs = nullptr;             // [max_n]
  uint32_t *hist = nullptr;           // [2 * 2048]
  uint32_t *sel = nullptr;            // [8]
};
cudaError_t launch_semantic_trigger(const double *stats, const dags_sched_cfg &cfg, int seg_refreshed,
                                    int32_t *state, double *score, cudaStream_t s);
cudaError_t launch_mp_update(const MpBuffers &b, float *gauss, int64_t n, const double *pose, const Raster &r,
                             const float4 *targets, const float *image, const uint8_t *inst, const float *table,
                             int n_regions, const dags_mp_cfg &cfg, int seg_refreshed, uint8_t *labels,
                             double *stats, const float *mp_map, float *mp_pixel, uint32_t *status,
                             int num_sms, cudaStream_t s);
cudaError_t launch_mpnet_features(const float *image, const float4 *targets, const uint8_t *inst, const float *table,
                                  int n_regions, int P, uint16_t *feats, uint32_t *status, cudaStream_t s);

// ---- device helpers ----

// Programmatic dependent launch: the splatting kernels are launched with
// programmatic stream serialization, so that a kernel's CTAs may be scheduled
// while its predecessor drains; each of them waits for the predecessor's
// memory (griddepcontrol.wait) before its first global access, which keeps
// the stream order of all reads and writes. Without the launch attribute the
// wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Lets the next kernel's CTAs be scheduled before this one completes. Every
// kernel calls it only after its own pdl_wait, so when a successor starts,
// the launch before this one has completed: a successor may therefore read,
// before its own pdl_wait, data written two or more launches earlier (and
// nothing this kernel writes). Harmless without the launch attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Culling bounds of the tracking loop (the per-frame cull in splat_fwd.cu):
// poses within kCullRot rad and kCullTrans m of the pose the candidates were
// culled at.
constexpr float kCullRot = 0.01f, kCullTrans = 0.01f, kCullNear = 0.5f, kCullGrow = 1.25f;

// Whether pose P (FP32, 3x4) lies within the culling bounds of pose C:
// the relative motion p -> R_d p + t_d, R_d = R_P R_C^T, t_d = t_P - R_d t_C,
// with ||R_d - I||_F / (2 sqrt 2) = sin(theta / 2) <= sin(kCullRot / 2) and
// |t_d| <= kCullTrans (both with a rounding allowance).
__device__ __forceinline__ bool within_cull_bounds(const float *P, const float *C) {
  float Rd[9], fro = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Rd[3 * a + b] = P[4 * a] * C[4 * b] + P[4 * a + 1] * C[4 * b + 1] + P[4 * a + 2] * C[4 * b + 2];
      const float d = Rd[3 * a + b] - (a == b ? 1.f : 0.f);
      fro += d * d;
    }
  float t2 = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float td = P[4 * a + 3] - (Rd[3 * a] * C[3] + Rd[3 * a + 1] * C[7] + Rd[3 * a + 2] * C[11]);
    t2 += td * td;
  }
  const float s_max = 0.999f * sinf(0.5f * kCullRot);
  return sqrtf(fro) <= 2.f * 1.41421356f * s_max && sqrtf(t2) <= 0.999f * kCullTrans;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Hardware base-2 exponential and reciprocal (MUFU, flush-to-zero, about
// 2^-22 relative error). The compositing loops take the exponential only for
// exponents in [log2(1/255), 0] and the reciprocal of 1 - alpha in [0.01, 1].
__device__ __forceinline__ float hw_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float hw_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Rotation matrix (row-major) of q / |q|, Hamilton convention, scalar first.
__device__ __forceinline__ void quat_to_rot(float qw, float qx, float qy, float qz, float *R,
                                            float *n, float *qlen) {
  // every operation explicitly rounded (no contraction left to the
  // compiler), so that each kernel that inlines this computes the same bits
  const float len = __fsqrt_rn(__fmaf_rn(qz, qz, __fmaf_rn(qy, qy, __fmaf_rn(qx, qx, __fmul_rn(qw, qw)))));
  const float inv = __fdiv_rn(1.0f, len);
  const float w = __fmul_rn(qw, inv), x = __fmul_rn(qx, inv), y = __fmul_rn(qy, inv), z = __fmul_rn(qz, inv);
  auto diag = [](float a, float b) { return __fmaf_rn(-2.f, __fmaf_rn(a, a, __fmul_rn(b, b)), 1.f); };
  auto offd = [](float a, float b, float c, float d, float sg) {
    return __fmul_rn(2.f, __fmaf_rn(a, b, __fmul_rn(sg * c, d)));
  };
  R[0] = diag(y, z);               R[1] = offd(x, y, w, z, -1.f); R[2] = offd(x, z, w, y, 1.f);
  R[3] = offd(x, y, w, z, 1.f);    R[4] = diag(x, z);             R[5] = offd(y, z, w, x, -1.f);
  R[6] = offd(x, z, w, y, -1.f);   R[7] = offd(y, z, w, x, 1.f);  R[8] = diag(x, y);
  if (n) { n[0] = w; n[1] = x; n[2] = y; n[3] = z; }
  if (qlen) *qlen = len;
}

// Camera depth of the mean, which is also the depth-order key: evaluated in
// FP32 in exactly this order with no fused multiply-add, so that the order
// of two Gaussians closer than FP32 rounding is a defined function of the
// record and the FP32 pose (ties are broken by Gaussian id).
__device__ __forceinline__ float depth_key(const float4 &g0, const float *P) {
  const float a = __fmul_rn(P[8], g0.x), b = __fmul_rn(P[9], g0.y), c = __fmul_rn(P[10], g0.z);
  return __fadd_rn(__fadd_rn(__fadd_rn(a, b), c), P[11]);
}

// Everything the projection of one Gaussian into one view computes in FP32,
// kept so the backward can chain through it.
struct Proj {
  float x, y, z;          // camera-space mean
  float txz, tyz;         // x/z, y/z before the guard clamp
  float tx, ty;           // after the clamp
  float j00, j02, j11, j12;
  float Rq[9], nq[4], qlen, S[3];
  float K[9];             // R_cw Rq diag(S)
  float m0[3], m1[3];     // rows of J K
  float A, B, C, det;     // 2D covariance (dilated) and its determinant
  float ca, cb, cc;       // conic
  float o, u, v;
};

// Projects record (g0..g2) with the FP32 pose P (3x4 row-major). Returns
// false if the Gaussian is culled before the conic (behind the near plane,
// degenerate covariance, opacity at or below alpha_min). The screen rect is
// computed separately.
__device__ __forceinline__ bool project_gaussian(const float4 &g0, const float4 &g1, const float4 &g2,
                                                 const float *P, const Raster &r, Proj &q) {
  // every operation explicitly rounded (no contraction left to the
  // compiler), so that each kernel that inlines this computes the same bits
  q.x = __fadd_rn(__fmaf_rn(P[2], g0.z, __fmaf_rn(P[1], g0.y, __fmul_rn(P[0], g0.x))), P[3]);
  q.y = __fadd_rn(__fmaf_rn(P[6], g0.z, __fmaf_rn(P[5], g0.y, __fmul_rn(P[4], g0.x))), P[7]);
  q.z = depth_key(g0, P);
  if (!(q.z > r.z_near)) return false;
  q.txz = __fdiv_rn(q.x, q.z);
  q.tyz = __fdiv_rn(q.y, q.z);
  q.tx = q.txz > r.limx ? r.limx : (q.txz < -r.limx ? -r.limx : q.txz);
  q.ty = q.tyz > r.limy ? r.limy : (q.tyz < -r.limy ? -r.limy : q.tyz);
  q.j00 = __fdiv_rn(r.fx, q.z);
  q.j02 = __fdiv_rn(__fmul_rn(-r.fx, q.tx), q.z);
  q.j11 = __fdiv_rn(r.fy, q.z);
  q.j12 = __fdiv_rn(__fmul_rn(-r.fy, q.ty), q.z);
  quat_to_rot(g1.x, g1.y, g1.z, g1.w, q.Rq, q.nq, &q.qlen);
  q.S[0] = expf(g2.x);
  q.S[1] = expf(g2.y);
  q.S[2] = expf(g2.z);
  // K = R_cw Rq diag(S); the 2D covariance is (J K)(J K)^T + dilation I, and
  // its determinant is the squared cross product of the rows of J K plus
  // dilation terms, which has no cancellation.
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int s = 0; s < 3; ++s)
      q.K[3 * a + s] = __fmul_rn(__fmaf_rn(P[4 * a + 2], q.Rq[6 + s],
                                           __fmaf_rn(P[4 * a + 1], q.Rq[3 + s], __fmul_rn(P[4 * a], q.Rq[s]))),
                                 q.S[s]);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    q.m0[s] = __fmaf_rn(q.j02, q.K[6 + s], __fmul_rn(q.j00, q.K[s]));
    q.m1[s] = __fmaf_rn(q.j12, q.K[6 + s], __fmul_rn(q.j11, q.K[3 + s]));
  }
  auto dot3 = [](const float *a, const float *b) {
    return __fmaf_rn(a[2], b[2], __fmaf_rn(a[1], b[1], __fmul_rn(a[0], b[0])));
  };
  const float A0 = dot3(q.m0, q.m0), C0 = dot3(q.m1, q.m1);
  q.B = dot3(q.m0, q.m1);
  const float cx0 = __fmaf_rn(q.m0[1], q.m1[2], -__fmul_rn(q.m0[2], q.m1[1]));
  const float cx1 = __fmaf_rn(q.m0[2], q.m1[0], -__fmul_rn(q.m0[0], q.m1[2]));
  const float cx2 = __fmaf_rn(q.m0[0], q.m1[1], -__fmul_rn(q.m0[1], q.m1[0]));
  const float d = r.dilation;
  q.A = __fadd_rn(A0, d);
  q.C = __fadd_rn(C0, d);
  const float cc = __fmaf_rn(cx2, cx2, __fmaf_rn(cx1, cx1, __fmul_rn(cx0, cx0)));
  q.det = __fadd_rn(__fmaf_rn(d, __fadd_rn(A0, C0), cc), __fmul_rn(d, d));
  q.o = __fdiv_rn(1.f, __fadd_rn(1.f, expf(-g0.w)));
  if (!(q.det > 0.f) || !(q.o > r.alpha_min)) return false;
  const float idet = __fdiv_rn(1.f, q.det);
  q.ca = __fmul_rn(q.C, idet);
  q.cb = __fmul_rn(-q.B, idet);
  q.cc = __fmul_rn(q.A, idet);
  q.u = __fadd_rn(__fdiv_rn(__fmul_rn(r.fx, q.x), q.z), r.cx);
  q.v = __fadd_rn(__fdiv_rn(__fmul_rn(r.fy, q.y), q.z), r.cy);
  return true;
}

// Error-free transformations of FP32 sums and products (Knuth's two-sum,
// and the fused multiply-add form of Dekker's two-product): a op b = s + e
// exactly. Every operation is explicitly rounded, so nothing is contracted.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// One row of the FP64 pose applied to an FP32 mean, in double-FP32
// arithmetic: (ph + pl) . m + (th + tl) = hi + lo with a relative error of a
// few 2^-44 of the largest term. ph, pl: the row's rotation entries split
// into FP32 high and low parts; th, tl: its translation.
__device__ __forceinline__ void df_row(const float *ph, const float *pl, float th, float tl, float mx, float my,
                                       float mz, float &hi, float &lo) {
  float p0, e0, p1, e1, p2, e2, s, t;
  two_prod(ph[0], mx, p0, e0);
  two_prod(ph[1], my, p1, e1);
  two_prod(ph[2], mz, p2, e2);
  float acc = __fadd_rn(__fadd_rn(e0, e1), e2);
  acc = __fadd_rn(acc, __fadd_rn(__fadd_rn(__fmul_rn(pl[0], mx), __fmul_rn(pl[1], my)), __fmul_rn(pl[2], mz)));
  two_sum(p0, p1, s, t);
  acc = __fadd_rn(acc, t);
  two_sum(s, p2, s, t);
  acc = __fadd_rn(acc, t);
  two_sum(s, th, s, t);
  acc = __fadd_rn(acc, __fadd_rn(t, tl));
  two_sum(s, acc, hi, lo);
}

// The projected centre u = f x / z + c in double-FP32 from x = xh + xl,
// z = zh + zl: the quotient's high part, its remainder through a fused
// multiply-add, then f q + c with two-product and two-sum.
__device__ __forceinline__ void df_project(float xh, float xl, float zh, float zl, float f, float c, float &uh,
                                           float &ul) {
  const float qh = __fdiv_rn(xh, zh);
  // x - qh z = (xh - qh zh) + xl - qh zl; the first term is exact by FMA
  const float rem = __fadd_rn(__fsub_rn(__fmaf_rn(-qh, zh, xh), __fmul_rn(qh, zl)), xl);
  const float ql = __fdiv_rn(rem, zh);
  float p, pe, s, se;
  two_prod(f, qh, p, pe);
  two_sum(p, c, s, se);
  const float lo = __fadd_rn(__fadd_rn(pe, __fmul_rn(f, ql)), se);
  two_sum(s, lo, uh, ul);
}

// Does the ellipse Q(d) = A2 dx^2 + B2 dx dy + C2 dy^2 <= thr (centre (u, v);
// A2 = -a', B2 = -b', C2 = -c', thr = lo - log2(alpha_min)) reach the
// pixel-centre rectangle [x0, x1] x [y0, y1]? The minimum of the positive
// definite Q over the rectangle is 0 if the centre is inside, else it is on
// an edge, where Q is a 1-D quadratic whose minimiser is clamped to the edge.
// Every operation is explicitly rounded (no contraction), so that the kernel
// that counts pairs and the kernel that emits them decide identically.
__device__ __forceinline__ bool ellipse_reaches_rect(float u, float v, float A2, float B2, float C2, float thr,
                                                     float x0, float x1, float y0, float y1) {
  const float xl = __fsub_rn(x0, u), xh = __fsub_rn(x1, u);
  const float yl = __fsub_rn(y0, v), yh = __fsub_rn(y1, v);
  if (xl <= 0.f && xh >= 0.f && yl <= 0.f && yh >= 0.f) return true;
  float best = INFINITY;
  const float xs[2] = {xl, xh}, ys[2] = {yl, yh};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float x = xs[k];
    float y = __fdiv_rn(__fmul_rn(-B2, x), __fmul_rn(2.f, C2));
    y = fminf(fmaxf(y, yl), yh);
    float q = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(A2, x), x), __fmul_rn(__fmul_rn(B2, x), y)),
                        __fmul_rn(__fmul_rn(C2, y), y));
    best = fminf(best, q);
    const float yy = ys[k];
    float xx = __fdiv_rn(__fmul_rn(-B2, yy), __fmul_rn(2.f, A2));
    xx = fminf(fmaxf(xx, xl), xh);
    q = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(A2, xx), xx), __fmul_rn(__fmul_rn(B2, xx), yy)),
                  __fmul_rn(__fmul_rn(C2, yy), yy));
    best = fminf(best, q);
  }
  return best <= thr;
}

// Reduce-scatter of K values over the 32 lanes of a warp. Each of the five
// xor levels (16, 8, 4, 2, 1) halves the lane's list: the lane keeps one half
// and adds its partner's copy of that half; an odd last entry is summed whole
// and stays with both partners. On return every lane holds the full warp sum
// of one component, rs_component<K>(lane). Shuffles: 8 for K = 6, 9 for
// K = 8, 12 for K = 10 (against 5 K for separate warp sums).
template <int K, int M = 16>
__device__ __forceinline__ float warp_reduce_scatter(const float (&cur)[K], int lane) {
  constexpr int P = K / 2, K2 = P + (K & 1);
  static_assert(M > 1 || K2 == 1, "at most 32 components");
  const bool hi = (lane & M) != 0;
  float nxt[K2];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    const float keep = hi ? cur[i + P] : cur[i];
    const float send = hi ? cur[i] : cur[i + P];
    nxt[i] = keep + __shfl_xor_sync(0xffffffffu, send, M);
  }
  if constexpr ((K & 1) != 0) nxt[P] = cur[K - 1] + __shfl_xor_sync(0xffffffffu, cur[K - 1], M);
  if constexpr (M == 1) {
    return nxt[0];
  } else {
    return warp_reduce_scatter<K2, M / 2>(nxt, lane);
  }
}

// The component whose sum warp_reduce_scatter<K> leaves in lane `lane`: the
// same selections applied to the component indices.
template <int K, int M = 16>
__device__ __forceinline__ int rs_component_of(const int (&cur)[K], int lane) {
  constexpr int P = K / 2, K2 = P + (K & 1);
  const bool hi = (lane & M) != 0;
  int nxt[K2];
#pragma unroll
  for (int i = 0; i < P; ++i) nxt[i] = hi ? cur[i + P] : cur[i];
  if constexpr ((K & 1) != 0) nxt[P] = cur[K - 1];
  if constexpr (M == 1) {
    return nxt[0];
  } else {
    return rs_component_of<K2, M / 2>(nxt, lane);
  }
}

template <int K>
__device__ __forceinline__ int rs_component(int lane) {
  int ids[K];
#pragma unroll
  for (int i = 0; i < K; ++i) ids[i] = i;
  return rs_component_of<K>(ids, lane);
}

// FP64 Adam step on the twist of one pose followed by T <- exp(xi^) T, with
// no transcendental on the common path (GB300's FP64 units are few): the
// bias corrections beta^k by binary powering, and sin/cos of |phi| < 0.25 by
// their Taylor series to |phi|^12 (omitted terms below 1e-17).
__device__ inline double pow_int(double b, double kd) {
  unsigned long long k = (unsigned long long)kd;
  double r = 1.0;
  while (k) {
    if (k & 1ull) r *= b;
    b *= b;
    k >>= 1;
  }
  return r;
}

// T <- exp(xi^) T for the twist xi = (rho, phi) (translation first), FP64:
// Rodrigues' formula for the rotation and the left Jacobian of SO(3) for the
// translation, with series forms for small angles.
__device__ inline void se3_exp_left(double *T, const double *xi) {
  const double px = xi[3], py = xi[4], pz = xi[5];
  const double t2 = px * px + py * py + pz * pz;
  double a, b, c;
  if (t2 < 0.0625) {
    // sin(t)/t, (1-cos t)/t^2, (t-sin t)/t^3 as series in t^2
    a = 1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880 + t2 * (-1.0 / 39916800 +
        t2 * (1.0 / 6227020800.0))))));
    b = 0.5 + t2 * (-1.0 / 24 + t2 * (1.0 / 720 + t2 * (-1.0 / 40320 + t2 * (1.0 / 3628800 + t2 * (-1.0 / 479001600 +
        t2 * (1.0 / 87178291200.0))))));
    c = 1.0 / 6 + t2 * (-1.0 / 120 + t2 * (1.0 / 5040 + t2 * (-1.0 / 362880 + t2 * (1.0 / 39916800 +
        t2 * (-1.0 / 6227020800.0 + t2 * (1.0 / 1307674368000.0))))));
  } else {
    const double t = sqrt(t2);
    a = sin(t) / t;
    b = (1.0 - cos(t)) / t2;
    c = (t - sin(t)) / (t2 * t);
  }
  const double Kh[9] = {0.0, -pz, py, pz, 0.0, -px, -py, px, 0.0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      K2[3 * i + j] = Kh[3 * i] * Kh[j] + Kh[3 * i + 1] * Kh[3 + j] + Kh[3 * i + 2] * Kh[6 + j];
  double Re[9], V[9];
  for (int e = 0; e < 9; ++e) {
    const double I = (e % 4 == 0) ? 1.0 : 0.0;
    Re[e] = I + a * Kh[e] + b * K2[e];
    V[e] = I + b * Kh[e] + c * K2[e];
  }
  double te[3];
  for (int i = 0; i < 3; ++i) te[i] = V[3 * i] * xi[0] + V[3 * i + 1] * xi[1] + V[3 * i + 2] * xi[2];
  double out[12];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) out[4 * i + j] = Re[3 * i] * T[j] + Re[3 * i + 1] * T[4 + j] + Re[3 * i + 2] * T[8 + j];
    out[4 * i + 3] = Re[3 * i] * T[3] + Re[3 * i + 1] * T[7] + Re[3 * i + 2] * T[11] + te[i];
  }
  for (int e = 0; e < 12; ++e) T[e] = out[e];
}

__device__ inline void pose_adam_exp(double *T, const double *grad, double *st, const dags_pose_cfg &cfg) {
  const double k = st[12] + 1.0;
  const double bc1 = 1.0 - pow_int(cfg.beta1, k), bc2 = 1.0 - pow_int(cfg.beta2, k);
  double xi[6];
  for (int c = 0; c < 6; ++c) {
    const double g = grad[c];
    const double m = cfg.beta1 * st[c] + (1.0 - cfg.beta1) * g;
    const double s2 = cfg.beta2 * st[6 + c] + (1.0 - cfg.beta2) * g * g;
    st[c] = m;
    st[6 + c] = s2;
    xi[c] = -cfg.lr[c] * (m / bc1) / (sqrt(s2 / bc2) + cfg.eps);
  }
  st[12] = k;
  se3_exp_left(T, xi);
}

// The same pose step spread over the first 12 threads of a CTA (dependent
// FP64 chains are what costs on GB300): threads 0-5 update one twist
// component's Adam moments each, thread 0 the scalar series, threads 0-11
// one entry of the new 3x4 pose each. Must be called by all threads of the
// CTA (it synchronises); xi_s, sc_s are shared scratch of 6 and 3 doubles.
// The bias corrections 1 / (1 - beta1^k) and 1 / sqrt(1 - beta2^k) of the
// step that follows state st (they depend on its step count only).
__device__ inline double adam_bias1(const dags_pose_cfg &cfg, double k) { return 1.0 / (1.0 - pow_int(cfg.beta1, k)); }
__device__ inline double adam_bias2(const dags_pose_cfg &cfg, double k) {
  return 1.0 / sqrt(1.0 - pow_int(cfg.beta2, k));
}

// pre_sc: the two bias corrections when the caller formed them already
// (from the same step count), or null.
__device__ inline void pose_adam_exp_cta(double *T, const double *grad, double *st, const dags_pose_cfg &cfg,
                                         double *xi_s, double *sc_s, const double *pre_sc = nullptr) {
  const int t = threadIdx.x;
  const double k = st[12] + 1.0;
  // threads 6 and 7 form the bias corrections (unless given) while threads
  // 0-5 update the moments and take sqrt(s2): the step is then
  // -lr (m / bc1) / (sqrt(s2) / sqrt(bc2) + eps), one division deep
  double m = 0.0, rs = 0.0;
  if (t < 6) {
    const double g = grad[t];
    m = cfg.beta1 * st[t] + (1.0 - cfg.beta1) * g;
    const double s2 = cfg.beta2 * st[6 + t] + (1.0 - cfg.beta2) * g * g;
    st[t] = m;
    st[6 + t] = s2;
    rs = sqrt(s2);
  } else if (t == 6) {
    sc_s[0] = pre_sc ? pre_sc[0] : adam_bias1(cfg, k);
  } else if (t == 7) {
    sc_s[1] = pre_sc ? pre_sc[1] : adam_bias2(cfg, k);
  }
  __syncthreads();
  if (t < 6) xi_s[t] = -cfg.lr[t] * (m * sc_s[0]) / (rs * sc_s[1] + cfg.eps);
  __syncthreads();
  if (t == 0) {
    st[12] = k;
    const double t2 = xi_s[3] * xi_s[3] + xi_s[4] * xi_s[4] + xi_s[5] * xi_s[5];
    double a, b, c;
    if (t2 < 0.0625) {
      a = 1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880 + t2 * (-1.0 / 39916800 +
          t2 * (1.0 / 6227020800.0))))));
      b = 0.5 + t2 * (-1.0 / 24 + t2 * (1.0 / 720 + t2 * (-1.0 / 40320 + t2 * (1.0 / 3628800 + t2 * (-1.0 / 479001600 +
          t2 * (1.0 / 87178291200.0))))));
      c = 1.0 / 6 + t2 * (-1.0 / 120 + t2 * (1.0 / 5040 + t2 * (-1.0 / 362880 + t2 * (1.0 / 39916800 +
          t2 * (-1.0 / 6227020800.0 + t2 * (1.0 / 1307674368000.0))))));
    } else {
      const double th = sqrt(t2);
      a = sin(th) / th;
      b = (1.0 - cos(th)) / t2;
      c = (th - sin(th)) / (t2 * th);
    }
    sc_s[0] = a; sc_s[1] = b; sc_s[2] = c;
  }
  __syncthreads();
  double out = 0.0;
  if (t < 12) {
    const int i = t >> 2, j = t & 3;
    const double px = xi_s[3], py = xi_s[4], pz = xi_s[5];
    const double Kh[9] = {0.0, -pz, py, pz, 0.0, -px, -py, px, 0.0};
    double Re[3], V[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const double K2 = Kh[3 * i] * Kh[kk] + Kh[3 * i + 1] * Kh[3 + kk] + Kh[3 * i + 2] * Kh[6 + kk];
      const double I = (i == kk) ? 1.0 : 0.0;
      Re[kk] = I + sc_s[0] * Kh[3 * i + kk] + sc_s[1] * K2;
      V[kk] = I + sc_s[1] * Kh[3 * i + kk] + sc_s[2] * K2;
    }
    out = Re[0] * T[j] + Re[1] * T[4 + j] + Re[2] * T[8 + j];
    if (j == 3) out += V[0] * xi_s[0] + V[1] * xi_s[1] + V[2] * xi_s[2];
  }
  __syncthreads();
  if (t < 12) T[t] = out;
}

}  // namespace dags
