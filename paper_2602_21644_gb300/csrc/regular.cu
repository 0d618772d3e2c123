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
// float4 of the gradient). The loss is summed per CTA in FP64 by a fixed tree
// and across CTAs in a fixed order by the last CTA.
#include "common.cuh"

namespace dags {

namespace {

constexpr int kRegBlock = 256;

__global__ void __launch_bounds__(kRegBlock)
mp_consistency_kernel(const float4 *__restrict__ gauss, const float4 *__restrict__ prev, int64_t n,
                      const double *__restrict__ rel, float lam, float *__restrict__ grad,
                      double *__restrict__ partial, uint32_t *__restrict__ done, double *__restrict__ loss) {
  __shared__ double s_sum[kRegBlock];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * kRegBlock + tid;
  double term = 0.0;
  if (i < n) {
    const float4 g0 = __ldg(gauss + 4 * i), g2 = __ldg(gauss + 4 * i + 2);
    const float4 p0 = __ldg(prev + 4 * i);
    float hx = p0.x, hy = p0.y, hz = p0.z;
    if (rel) {
      hx = (float)(rel[0] * p0.x + rel[1] * p0.y + rel[2] * p0.z + rel[3]);
      hy = (float)(rel[4] * p0.x + rel[5] * p0.y + rel[6] * p0.z + rel[7]);
      hz = (float)(rel[8] * p0.x + rel[9] * p0.y + rel[10] * p0.z + rel[11]);
    }
    const float mbar = 1.f - g2.w;
    const float dx = g0.x - hx, dy = g0.y - hy, dz = g0.z - hz;
    term = (double)(mbar * (dx * dx + dy * dy + dz * dz));
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
  s_sum[tid] = term;
  __syncthreads();
  for (int o = kRegBlock / 2; o > 0; o >>= 1) {
    if (tid < o) s_sum[tid] += s_sum[tid + o];
    __syncthreads();
  }
  if (tid == 0) {
    partial[blockIdx.x] = s_sum[0];
    __threadfence();
    s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  double acc = 0.0;
  for (int k = tid; k < (int)gridDim.x; k += kRegBlock) acc += __ldcg(partial + k);
  s_sum[tid] = acc;
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

}  // namespace

int64_t mp_consistency_blocks(int64_t n) { return (n + kRegBlock - 1) / kRegBlock; }

cudaError_t launch_mp_consistency(const float4 *gauss, const float4 *prev, int64_t n, const double *rel, float lam,
                                  float *grad, double *partial, uint32_t *done, double *loss, cudaStream_t s) {
  if (n == 0) {
    if (loss) return cudaMemsetAsync(loss, 0, sizeof(double), s);
    return cudaSuccess;
  }
  mp_consistency_kernel<<<(unsigned)mp_consistency_blocks(n), kRegBlock, 0, s>>>(gauss, prev, n, rel, lam, grad,
                                                                                 partial, done, loss);
  return cudaGetLastError();
}

}  // namespace dags
