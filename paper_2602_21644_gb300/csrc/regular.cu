// MP-based motion-consistency regulariser (Sec. IV-D, Eqs. (23), (24)) on
// sm_103a:
//
//   mu_hat_k = T_rel mu_k^{t-1}   (T_rel the relative pose; identity for a
//                                  world-frame map)
//   lambda L_MP = lambda sum_k (1 - M_k) |mu_k - mu_hat_k|^2
//   d/d mu_k    = 2 lambda (1 - M_k) (mu_k - mu_hat_k)
//
// One thread per Gaussian, HBM-bound (the first and third float4 of the
// record, the first of the previous record, a read-modify-write of the first
// float4 of the gradient). The loss is summed per warp in FP32 (fixed
// shuffle order), across a CTA's warps in FP64 by one thread, and across CTAs
// in a fixed order by the last CTA.
//
// MP-guided edge-warp regulariser (Sec. IV-D, Eqs. (25), (26)): one thread
// per pixel u of frame i. An edge pixel (a valid 4-neighbour differs by more
// than edge_rel times its depth) is back-projected with its observed depth, moved by
// T_ji = T_jW T_iW^-1 (formed once in FP64 by a one-thread kernel) and projected into frame
// j; D_j and w^j are sampled bilinearly at u', r = w^j (D_j - z_ref) enters
// the Huber kernel, and the gradients with respect to both poses' left
// twists follow by the chain rule through the bilinear cell, the projection
// and the rigid motion. The 13 sums go per CTA in FP32 (warp shuffles, then
// the CTA's 8 warps in order), and across CTAs in FP64 in a fixed order by
// the last CTA.
#include "common.cuh"

namespace dags {

namespace {

constexpr int kRegBlock = 256;

__global__ void __launch_bounds__(kRegBlock)
mp_consistency_kernel(const float4 *__restrict__ gauss, const float4 *__restrict__ prev, int64_t n,
                      const float *__restrict__ rel, float lam, float *__restrict__ grad,
                      double *__restrict__ partial, uint32_t *__restrict__ done, double *__restrict__ loss) {
  pdl_wait();
  __shared__ double s_sum[kRegBlock];
  __shared__ float s_warp[kRegBlock / 32];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * kRegBlock + tid;
  float term = 0.f;
  if (i < n) {
    const float4 g0 = __ldg(gauss + 4 * i), g2 = __ldg(gauss + 4 * i + 2);
    const float4 p0 = __ldg(prev + 4 * i);
    float hx = p0.x, hy = p0.y, hz = p0.z;
    if (rel) {
      hx = rel[0] * p0.x + rel[1] * p0.y + rel[2] * p0.z + rel[3];
      hy = rel[4] * p0.x + rel[5] * p0.y + rel[6] * p0.z + rel[7];
      hz = rel[8] * p0.x + rel[9] * p0.y + rel[10] * p0.z + rel[11];
    }
    const float mbar = 1.f - g2.w;
    const float dx = g0.x - hx, dy = g0.y - hy, dz = g0.z - hz;
    term = mbar * (dx * dx + dy * dy + dz * dz);
    if (grad) {
      float4 *gp = reinterpret_cast<float4 *>(grad) + 4 * i;
      float4 gv = *gp;
      const float c = 2.f * lam * mbar;
      gv.x += c * dx;
      gv.y += c * dy;
      gv.z += c * dz;
      *gp = gv;
    }
  }
  if (!loss) return;
  // FP32 warp sums (fixed shuffle order), then the CTA's warps in FP64 by one
  // thread: FP64 instructions are scarce on GB300, so none per element
  const float ws = warp_sum(term);
  if ((tid & 31) == 0) s_warp[tid >> 5] = ws;
  __syncthreads();
  if (tid == 0) {
    double b = 0.0;
#pragma unroll
    for (int w = 0; w < kRegBlock / 32; ++w) b += (double)s_warp[w];
    partial[blockIdx.x] = b;
    __threadfence();
    s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  // the CTA sums in a fixed order: 256 strided threads, four accumulators
  // each, then a fixed tree
  double a4[4] = {0.0, 0.0, 0.0, 0.0};
  int j = 0;
  for (int k = tid; k < (int)gridDim.x; k += kRegBlock, ++j) a4[j & 3] += __ldcg(partial + k);
  s_sum[tid] = (a4[0] + a4[1]) + (a4[2] + a4[3]);
  __syncthreads();
  for (int o = kRegBlock / 2; o > 0; o >>= 1) {
    if (tid < o) s_sum[tid] += s_sum[tid + o];
    __syncthreads();
  }
  if (tid == 0) {
    *loss = (double)lam * s_sum[0];
    *done = 0u;
  }
}

// T_ji = T_jW T_iW^-1 (R = Rj Ri^T, t = tj - R ti) of two world-to-camera
// poses, or pose_j itself when pose_i is NULL, in FP64 by one thread, rounded
// to FP32 for the per-element kernels.
__global__ void rel_pose_kernel(const double *__restrict__ pose_i, const double *__restrict__ pose_j,
                                float *__restrict__ out) {
  if (threadIdx.x != 0) return;
  if (!pose_i) {
    for (int k = 0; k < 12; ++k) out[k] = (float)pose_j[k];
    return;
  }
  double R[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      R[3 * a + b] = pose_j[4 * a] * pose_i[4 * b] + pose_j[4 * a + 1] * pose_i[4 * b + 1] +
                     pose_j[4 * a + 2] * pose_i[4 * b + 2];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) out[4 * a + b] = (float)R[3 * a + b];
    out[4 * a + 3] =
        (float)(pose_j[4 * a + 3] - (R[3 * a] * pose_i[3] + R[3 * a + 1] * pose_i[7] + R[3 * a + 2] * pose_i[11]));
  }
}

constexpr int kEdgeBlock = 256;
constexpr int kEdgeOut = 13;     // lambda L_edge, d/d xi_i (6), d/d xi_j (6)

__global__ void __launch_bounds__(kEdgeBlock)
edge_warp_kernel(Raster r, const float *__restrict__ Di, const float *__restrict__ Dj,
                 const float *__restrict__ wj, const float *__restrict__ Tji, dags_edge_cfg c, float lam,
                 double *__restrict__ partial, uint32_t *__restrict__ done, double *__restrict__ out) {
  pdl_wait();
  __shared__ float s_T[12];
  __shared__ float s_red[kEdgeBlock / 32][kEdgeOut];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 12) s_T[tid] = Tji[tid];
  __syncthreads();
  const int W = r.W, H = r.H;
  const int p = blockIdx.x * kEdgeBlock + tid;
  float v[kEdgeOut];
#pragma unroll
  for (int k = 0; k < kEdgeOut; ++k) v[k] = 0.f;
  if (p < W * H) {
    const int y = p / W, x = p - y * W;
    const float d = Di[p];
    bool edge = false;
    if (d > 0.f) {
      const int nx[4] = {x + 1, x - 1, x, x}, ny[4] = {y, y, y + 1, y - 1};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (nx[k] < 0 || nx[k] >= W || ny[k] < 0 || ny[k] >= H) continue;
        const float dn = Di[ny[k] * W + nx[k]];
        if (dn > 0.f && fabsf(dn - d) > c.edge_rel * d) edge = true;
      }
    }
    if (edge) {
      const float X0 = d * ((float)x - r.cx) / r.fx, X1 = d * ((float)y - r.cy) / r.fy, X2 = d;
      const float Y0 = s_T[0] * X0 + s_T[1] * X1 + s_T[2] * X2 + s_T[3];
      const float Y1 = s_T[4] * X0 + s_T[5] * X1 + s_T[6] * X2 + s_T[7];
      const float Y2 = s_T[8] * X0 + s_T[9] * X1 + s_T[10] * X2 + s_T[11];
      if (Y2 > c.z_near) {
        const float iz = 1.f / Y2;
        const float u = r.fx * Y0 * iz + r.cx, vv = r.fy * Y1 * iz + r.cy;
        const float fx0 = floorf(u), fy0 = floorf(vv);
        if (fx0 >= 0.f && fy0 >= 0.f && fx0 + 1.f <= (float)(W - 1) && fy0 + 1.f <= (float)(H - 1)) {
          const int x0 = (int)fx0, y0 = (int)fy0;
          const int q0 = y0 * W + x0;
          const float d00 = Dj[q0], d01 = Dj[q0 + 1], d10 = Dj[q0 + W], d11 = Dj[q0 + W + 1];
          if (d00 > 0.f && d01 > 0.f && d10 > 0.f && d11 > 0.f) {
            const float w00 = wj[q0], w01 = wj[q0 + 1], w10 = wj[q0 + W], w11 = wj[q0 + W + 1];
            const float fu = u - fx0, fv = vv - fy0;
            const float a0 = (1.f - fu) * (1.f - fv), a1 = fu * (1.f - fv), a2 = (1.f - fu) * fv, a3 = fu * fv;
            const float Ds = a0 * d00 + a1 * d01 + a2 * d10 + a3 * d11;
            const float ws = a0 * w00 + a1 * w01 + a2 * w10 + a3 * w11;
            const float zref = c.literal ? d : Y2;
            const float res = ws * (Ds - zref);
            const float ar = fabsf(res);
            const float rho = ar <= c.huber ? 0.5f * res * res : c.huber * (ar - 0.5f * c.huber);
            const float drho = ar <= c.huber ? res : copysignf(c.huber, res);
            // bilinear slopes along u and v
            const float dDu = (1.f - fv) * (d01 - d00) + fv * (d11 - d10);
            const float dDv = (1.f - fu) * (d10 - d00) + fu * (d11 - d01);
            const float dwu = (1.f - fv) * (w01 - w00) + fv * (w11 - w10);
            const float dwv = (1.f - fu) * (w10 - w00) + fu * (w11 - w01);
            const float e = Ds - zref;
            const float dru = dwu * e + ws * dDu, drv = dwv * e + ws * dDv;
            // d(u, v)/dY, then dr/dY (the reference depth Y_z contributes -ws)
            float g0 = dru * r.fx * iz, g1 = drv * r.fy * iz;
            float g2 = -(dru * r.fx * Y0 + drv * r.fy * Y1) * iz * iz;
            if (!c.literal) g2 -= ws;
            g0 *= drho; g1 *= drho; g2 *= drho;
            v[0] = rho;
            // pose j: rho_j += gY, phi_j += Y x gY
            v[7] = g0; v[8] = g1; v[9] = g2;
            v[10] = Y1 * g2 - Y2 * g1; v[11] = Y2 * g0 - Y0 * g2; v[12] = Y0 * g1 - Y1 * g0;
            // pose i: gR = R^T gY; rho_i -= gR, phi_i -= X x gR
            const float r0 = s_T[0] * g0 + s_T[4] * g1 + s_T[8] * g2;
            const float r1 = s_T[1] * g0 + s_T[5] * g1 + s_T[9] * g2;
            const float r2 = s_T[2] * g0 + s_T[6] * g1 + s_T[10] * g2;
            v[1] = -r0; v[2] = -r1; v[3] = -r2;
            v[4] = -(X1 * r2 - X2 * r1); v[5] = -(X2 * r0 - X0 * r2); v[6] = -(X0 * r1 - X1 * r0);
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kEdgeOut; ++k) {
    const float sw = warp_sum(v[k]);
    if (lane == 0) s_red[warp][k] = sw;
  }
  __syncthreads();
  if (tid < kEdgeOut) {
    float a = 0.f;
#pragma unroll
    for (int w = 0; w < kEdgeBlock / 32; ++w) a += s_red[w][tid];
    partial[(size_t)blockIdx.x * kEdgeOut + tid] = (double)a;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  // 16 threads per output with a fixed stride, four independent accumulators
  // each (dependent FP64 additions are slow on GB300), then the 16 in order
  __shared__ double s_col[kEdgeOut * 16];
  if (tid < kEdgeOut * 16) {
    const int c = tid >> 4, part = tid & 15;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    int j = 0;
    for (int b = part; b < (int)gridDim.x; b += 16, ++j) a[j & 3] += __ldcg(partial + (size_t)b * kEdgeOut + c);
    s_col[tid] = (a[0] + a[1]) + (a[2] + a[3]);
  }
  __syncthreads();
  if (tid < kEdgeOut) {
    double a = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) a += s_col[tid * 16 + k];
    out[tid] = (double)lam * a;
  }
  __syncthreads();
  if (tid == 0) *done = 0u;
}

}  // namespace

int64_t edge_warp_blocks(int64_t pixels) { return (pixels + kEdgeBlock - 1) / kEdgeBlock; }

cudaError_t launch_edge_warp(const Raster &r, const float *Di, const float *Dj, const float *wj, const double *pose_i,
                             const double *pose_j, const dags_edge_cfg &c, float lam, double *partial, uint32_t *done,
                             double *out, float *tji, cudaStream_t s) {
  rel_pose_kernel<<<1, 32, 0, s>>>(pose_i, pose_j, tji);
  // a programmatic launch: the warp's launch overlaps the one-thread kernel
  const cudaError_t e = launch_pdl(edge_warp_kernel, dim3((unsigned)edge_warp_blocks((int64_t)r.W * r.H)),
                                   dim3(kEdgeBlock), 0, s, r, Di, Dj, wj, (const float *)tji, c, lam, partial, done,
                                   out);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int64_t mp_consistency_blocks(int64_t n) { return (n + kRegBlock - 1) / kRegBlock; }

cudaError_t launch_mp_consistency(const float4 *gauss, const float4 *prev, int64_t n, const double *rel, float lam,
                                  float *grad, double *partial, uint32_t *done, double *loss, float *rel32,
                                  cudaStream_t s) {
  if (n == 0) {
    if (loss) return cudaMemsetAsync(loss, 0, sizeof(double), s);
    return cudaSuccess;
  }
  if (rel) rel_pose_kernel<<<1, 32, 0, s>>>(nullptr, rel, rel32);
  const cudaError_t e = launch_pdl(mp_consistency_kernel, dim3((unsigned)mp_consistency_blocks(n)), dim3(kRegBlock), 0, s,
                                   gauss, prev, n, (const float *)(rel ? rel32 : nullptr), lam, grad, partial, done, loss);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace dags
