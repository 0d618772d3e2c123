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
constexpr int kSortSmallCap = 4096;     // per-tile list length sorted in one pass
constexpr int kSortBigChunk = 16384;    // chunk of the out-of-core merge sort
constexpr int kPrepBlock = 256;         // threads per preprocess CTA
constexpr int kBwdPrepBlock = 128;      // threads per preprocess-backward CTA

// Status word bits (device).
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;

// 2D gradient slots per (view, Gaussian).
enum { G2_U = 0, G2_V, G2_A, G2_B, G2_C, G2_Z, G2_O, G2_R, G2_G, G2_BL };

// Counters in the workspace's counter array.
enum {
  CNT_DONE_PREP = 0,   // CTAs of the preprocess kernel that finished
  CNT_DONE_RENDER,     // CTAs of the forward render that finished
  CNT_DONE_BWDPREP,    // CTAs of the preprocess backward that finished
  CNT_BIG_TILES,       // tiles whose lists exceed kSortSmallCap
  CNT_STATUS,          // status bits
  CNT_REQ_LO,          // pairs required by the last forward (low / high word)
  CNT_REQ_HI,
  CNT_N
};

struct Workspace {
  int64_t max_n = 0;
  int max_w = 0, max_h = 0, max_v = 0, max_tiles = 0;
  int64_t max_pairs = 0;
  int bwd_prep_blocks = 0;
  float4 *rec2d = nullptr;        // [V][N][3]: {u, v, z, o}, {a, b, c, M}, {r, g, b, -}
  uint2 *rect = nullptr;          // [V][N]: {x0 | x1 << 16, y0 | y1 << 16}, tiles [x0, x1) x [y0, y1)
  float *grad2d = nullptr;        // [V][N][kGradWords]
  uint32_t *tile_count = nullptr; // [V * T]
  uint32_t *tile_start = nullptr; // [V * T + 1]
  uint32_t *tile_cursor = nullptr;// [V * T]
  uint64_t *keys = nullptr;       // [max_pairs]: depth bits << 32 | Gaussian id
  uint64_t *keys_tmp = nullptr;   // [max_pairs]: merge ping-pong
  uint32_t *sorted_ids = nullptr; // [max_pairs]
  uint32_t *big_tiles = nullptr;  // [V * T]
  float *loss_partial = nullptr;  // [V * T]
  double *pose_partial = nullptr; // [bwd_prep_blocks][V][6]
  float *pose32 = nullptr;        // [V][12] FP32 copy of the poses of the last forward
  uint32_t *counters = nullptr;   // [CNT_N]
};

// Per-call constants handed to kernels by value.
struct Raster {
  float fx, fy, cx, cy;
  int W, H, tiles_x, tiles_y, T;   // T = tiles per view
  float alpha_min, alpha_max, t_min, dilation, z_near, limx, limy;
};

struct Loss {
  float lambda_pho, lambda_depth, o_eps;
  int weight_mode, weight_grad;
};

// ---- launchers (defined in the .cu files) ----
cudaError_t configure_fwd_kernels();  // once per device, at context creation
cudaError_t launch_preprocess(const Workspace &ws, const float4 *gauss, int64_t n, const double *poses,
                              int views, const Raster &r, int zero_grad_words, cudaStream_t s);
cudaError_t launch_emit(const Workspace &ws, int64_t n, int views, const Raster &r, cudaStream_t s);
cudaError_t launch_tile_sort(const Workspace &ws, int views, const Raster &r, cudaStream_t s);
cudaError_t launch_render_fwd(const Workspace &ws, int views, int64_t n, const Raster &r, const Loss &l,
                              const float4 *targets, float *image, int32_t *last, double *loss,
                              cudaStream_t s);
cudaError_t launch_render_bwd(const Workspace &ws, int views, int64_t n, const Raster &r, const Loss &l,
                              const float4 *targets, const float *image, const int32_t *last, bool full,
                              cudaStream_t s);
cudaError_t launch_preprocess_bwd(const Workspace &ws, const float4 *gauss, int64_t n, int views,
                                  const Raster &r, float *grad_gauss, double *grad_pose, cudaStream_t s);
cudaError_t launch_pose_step(double *poses, const double *grad, double *state, int views,
                             const dags_pose_cfg &cfg, cudaStream_t s);

// ---- device helpers ----

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
  float len = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  float inv = 1.0f / len;
  float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
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
  q.x = P[0] * g0.x + P[1] * g0.y + P[2] * g0.z + P[3];
  q.y = P[4] * g0.x + P[5] * g0.y + P[6] * g0.z + P[7];
  q.z = depth_key(g0, P);
  if (!(q.z > r.z_near)) return false;
  q.txz = q.x / q.z;
  q.tyz = q.y / q.z;
  q.tx = q.txz > r.limx ? r.limx : (q.txz < -r.limx ? -r.limx : q.txz);
  q.ty = q.tyz > r.limy ? r.limy : (q.tyz < -r.limy ? -r.limy : q.tyz);
  q.j00 = r.fx / q.z;
  q.j02 = -r.fx * q.tx / q.z;
  q.j11 = r.fy / q.z;
  q.j12 = -r.fy * q.ty / q.z;
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
      q.K[3 * a + s] = (P[4 * a] * q.Rq[s] + P[4 * a + 1] * q.Rq[3 + s] + P[4 * a + 2] * q.Rq[6 + s]) * q.S[s];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    q.m0[s] = q.j00 * q.K[s] + q.j02 * q.K[6 + s];
    q.m1[s] = q.j11 * q.K[3 + s] + q.j12 * q.K[6 + s];
  }
  const float A0 = q.m0[0] * q.m0[0] + q.m0[1] * q.m0[1] + q.m0[2] * q.m0[2];
  const float C0 = q.m1[0] * q.m1[0] + q.m1[1] * q.m1[1] + q.m1[2] * q.m1[2];
  q.B = q.m0[0] * q.m1[0] + q.m0[1] * q.m1[1] + q.m0[2] * q.m1[2];
  const float cx0 = q.m0[1] * q.m1[2] - q.m0[2] * q.m1[1];
  const float cx1 = q.m0[2] * q.m1[0] - q.m0[0] * q.m1[2];
  const float cx2 = q.m0[0] * q.m1[1] - q.m0[1] * q.m1[0];
  const float d = r.dilation;
  q.A = A0 + d;
  q.C = C0 + d;
  q.det = (cx0 * cx0 + cx1 * cx1 + cx2 * cx2) + d * (A0 + C0) + d * d;
  q.o = 1.f / (1.f + expf(-g0.w));
  if (!(q.det > 0.f) || !(q.o > r.alpha_min)) return false;
  const float idet = 1.f / q.det;
  q.ca = q.C * idet;
  q.cb = -q.B * idet;
  q.cc = q.A * idet;
  q.u = r.fx * q.x / q.z + r.cx;
  q.v = r.fy * q.y / q.z + r.cy;
  return true;
}

}  // namespace dags
