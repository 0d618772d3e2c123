// Throughput probes of the SM's FP32 and special-function pipes (sm_103a),
// used to measure the peaks that the compositing kernels are compared with.
// Not part of the method: the bench reports its ALU-bound kernels against
// these measured rates instead of peaks derived from unit counts and clocks.
//
//   alu_probe_kernel<0>   eight independent FP32 fused multiply-add chains
//                         per thread (one lane operation per FMA)
//   alu_probe_kernel<1>   eight independent ex2.approx.ftz chains per thread
//                         (x <- 2^-x keeps every value in [0.5, 1])
#include "common.cuh"

namespace dags {

namespace {

template <int KIND>
__global__ void __launch_bounds__(256) alu_probe_kernel(float *out, long long iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 0.5f + 0.01f * (float)((threadIdx.x + k) & 31);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (KIND == 0) x[k] = fmaf(x[k], a, b);
      else x[k] = hw_exp2(-x[k]);
    }
  }
  float t = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += x[k];
  // never true for the arguments the host passes; keeps the chains alive
  if (t == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace

}  // namespace dags

using namespace dags;

extern "C" int dags_measure_alu(int32_t kind, int64_t iters, double *ops_per_s, double *ms) {
  if ((kind != 0 && kind != 1) || iters < 1 || iters > (1ll << 24) || !ops_per_s) return DAGS_E_INVAL;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DAGS_E_CUDA;
  void (*kern)(float *, long long, float, float) = kind == 0 ? alu_probe_kernel<0> : alu_probe_kernel<1>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1)
    return DAGS_E_CUDA;
  const int grid = sms * per_sm;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return DAGS_E_CUDA;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // a = 1, b = 0 keeps the FMA chains at their start values
  if (e == cudaSuccess) { kern<<<grid, 256, 0, s>>>(nullptr, iters, 1.0f, 0.0f); e = cudaGetLastError(); }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) { kern<<<grid, 256, 0, s>>>(nullptr, iters, 1.0f, 0.0f); e = cudaGetLastError(); }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (e != cudaSuccess || !(t > 0.f)) return DAGS_E_CUDA;
  *ops_per_s = (double)grid * 256.0 * 8.0 * (double)iters / ((double)t * 1e-3);
  if (ms) *ms = t;
  return DAGS_OK;
}
