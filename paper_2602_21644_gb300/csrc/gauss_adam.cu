// Mapping optimiser step on the Gaussian parameters (sm_103a): Adam per
// parameter (Kingma and Ba, Algorithm 1) with one learning rate per group,
// the joint optimisation of Eq. (27) applied to the map.
//
//   gauss_adam_init_kernel  per Gaussian: the FP32 master colour from the
//                           record's BF16 colour, and zero moments
//   gauss_adam_kernel       per Gaussian: moments and the step of the 14
//                           optimised parameters (mean, opacity logit,
//                           quaternion, log-scale, colour); the record's FP32
//                           words are their own master copy, the colour is
//                           stepped in the FP32 master and written back to
//                           the record as BF16 (round to nearest, ties to
//                           even). The MP word is the MP update's and is not
//                           touched. HBM-bound: 272 bytes read and 208 written
//                           per Gaussian, all as float4.
#include <cuda_bf16.h>

#include "common.cuh"

namespace dags {

namespace {

constexpr int kAdamBlock = 256;

struct AdamStep {
  float lr[4][4];        // per record float4 word and component (0: not optimised)
  float lr_colour;
  float beta1, beta2, eps;
  float bc1, bc2_sqrt;   // 1 - beta1^t, sqrt(1 - beta2^t)
};

__device__ __forceinline__ float adam_one(float p, float g, float &m, float &v, float lr, const AdamStep &a) {
  m = a.beta1 * m + (1.f - a.beta1) * g;
  v = a.beta2 * v + (1.f - a.beta2) * g * g;
  const float denom = sqrtf(v) / a.bc2_sqrt + a.eps;
  return p - (lr / a.bc1) * m / denom;
}

__device__ __forceinline__ float comp(const float4 &x, int c) { return c == 0 ? x.x : c == 1 ? x.y : c == 2 ? x.z : x.w; }
__device__ __forceinline__ void set_comp(float4 &x, int c, float v) {
  if (c == 0) x.x = v; else if (c == 1) x.y = v; else if (c == 2) x.z = v; else x.w = v;
}

__global__ void __launch_bounds__(kAdamBlock)
gauss_adam_kernel(float4 *__restrict__ gauss, float4 *__restrict__ colour, float4 *__restrict__ m4,
                  float4 *__restrict__ v4, const float4 *__restrict__ grad, int64_t n, AdamStep a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 rec[3], g[4], m[4], v[4];
#pragma unroll
  for (int w = 0; w < 3; ++w) rec[w] = gauss[4 * i + w];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    g[w] = __ldg(grad + 4 * i + w);
    m[w] = m4[4 * i + w];
    v[w] = v4[4 * i + w];
  }
  float4 col = colour[i];
  // record words 0-10 (mean, logit, quaternion, log-scale)
#pragma unroll
  for (int w = 0; w < 3; ++w)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (w == 2 && c == 3) continue;   // the MP word
      const float lr = a.lr[w][c];
      float mm = comp(m[w], c), vv = comp(v[w], c);
      const float p = adam_one(comp(rec[w], c), comp(g[w], c), mm, vv, lr, a);
      set_comp(rec[w], c, p);
      set_comp(m[w], c, mm);
      set_comp(v[w], c, vv);
    }
  // colour: gradient slots 12-14, master copy, BF16 refresh
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float mm = comp(m[3], c), vv = comp(v[3], c);
    set_comp(col, c, adam_one(comp(col, c), comp(g[3], c), mm, vv, a.lr_colour, a));
    set_comp(m[3], c, mm);
    set_comp(v[3], c, vv);
  }
#pragma unroll
  for (int w = 0; w < 3; ++w) gauss[4 * i + w] = rec[w];
  const uint32_t r = __bfloat16_as_ushort(__float2bfloat16_rn(col.x));
  const uint32_t gg = __bfloat16_as_ushort(__float2bfloat16_rn(col.y));
  const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(col.z));
  float4 w3 = gauss[4 * i + 3];
  w3.x = __uint_as_float(r | (gg << 16));
  w3.y = __uint_as_float(b);
  gauss[4 * i + 3] = w3;
  colour[i] = col;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    m4[4 * i + w] = m[w];
    v4[4 * i + w] = v[w];
  }
}

__global__ void __launch_bounds__(kAdamBlock)
gauss_adam_init_kernel(const float4 *__restrict__ gauss, float4 *__restrict__ colour, float4 *__restrict__ m4,
                       float4 *__restrict__ v4, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 w3 = __ldg(gauss + 4 * i + 3);
  const uint32_t rg = __float_as_uint(w3.x), bl = __float_as_uint(w3.y);
  colour[i] = make_float4(bf16_lo(rg), bf16_hi(rg), bf16_lo(bl), 0.f);
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    m4[4 * i + w] = z;
    v4[4 * i + w] = z;
  }
}

}  // namespace

cudaError_t launch_gauss_adam_init(const float *gauss, float *colour, float *m, float *v, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gauss_adam_init_kernel<<<(unsigned)((n + kAdamBlock - 1) / kAdamBlock), kAdamBlock, 0, s>>>(
      reinterpret_cast<const float4 *>(gauss), reinterpret_cast<float4 *>(colour), reinterpret_cast<float4 *>(m),
      reinterpret_cast<float4 *>(v), n);
  return cudaGetLastError();
}

cudaError_t launch_gauss_adam(float *gauss, float *colour, float *m, float *v, const float *grad, int64_t n,
                              int64_t step, const dags_gauss_adam_cfg &c, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  AdamStep a;
  const float lrs[11] = {c.lr_mean, c.lr_mean, c.lr_mean, c.lr_opacity, c.lr_quat, c.lr_quat, c.lr_quat,
                         c.lr_quat, c.lr_scale, c.lr_scale, c.lr_scale};
  for (int k = 0; k < 16; ++k) a.lr[k / 4][k % 4] = k < 11 ? lrs[k] : 0.f;
  a.lr_colour = c.lr_colour;
  a.beta1 = c.beta1;
  a.beta2 = c.beta2;
  a.eps = c.eps;
  a.bc1 = (float)(1.0 - pow((double)c.beta1, (double)step));
  a.bc2_sqrt = (float)sqrt(1.0 - pow((double)c.beta2, (double)step));
  gauss_adam_kernel<<<(unsigned)((n + kAdamBlock - 1) / kAdamBlock), kAdamBlock, 0, s>>>(
      reinterpret_cast<float4 *>(gauss), reinterpret_cast<float4 *>(colour), reinterpret_cast<float4 *>(m),
      reinterpret_cast<float4 *>(v), reinterpret_cast<const float4 *>(grad), n, a);
  return cudaGetLastError();
}

}  // namespace dags
