// Throughput probes of the SM's FP32 and special-function pipes (sm_103a),
// used to measure the peaks that the compositing kernels are compared with.
// Not part of the method: the bench reports its ALU-bound kernels against
// these measured rates instead of peaks derived from unit counts and clocks.
//
//   alu_probe_kernel<0>   eight independent FP32 fused multiply-add chains
//                         per thread (one lane operation per FMA)
//   alu_probe_kernel<1>   eight independent ex2.approx.ftz chains per thread
//                         (x <- 2^-x keeps every value in [0.5, 1])
//   mma_probe_kernel      back-to-back tcgen05.mma kind::f16 (M = 64 or 128,
//                         N = n_cols, K = 16, BF16 operands in shared memory,
//                         FP32 accumulators in tensor memory), issued by one
//                         thread of each of 1..4 warpgroups of one CTA: the
//                         tensor core's rate as a function of N
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

__device__ __forceinline__ uint32_t probe_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle, 8-row core matrices
// of 16-byte lines (LBO between the two core matrices along K, SBO between
// 8-row groups), the sm_100-class descriptor version bit.
__device__ __forceinline__ uint64_t probe_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

constexpr int kProbeSmem = 40960;

// One CTA of 128 x groups threads. Thread 0 of warpgroup g issues `reps`
// accumulating MMAs into its own TMEM columns, commits them to its mbarrier
// and waits (bounded); cycles[2g] = the issue loop's SM cycles, cycles[2g +
// 1] = issue to completion. The operands are zeros.
__global__ void mma_probe_kernel(int groups, int m_rows, int n_cols, int reps, unsigned long long *cycles,
                                 uint32_t *status) {
  __shared__ __align__(1024) uint8_t sm[kProbeSmem];
  __shared__ uint64_t bars[4];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, g = tid >> 7, t = tid & 127;
  for (int k = tid; k < kProbeSmem / 16; k += blockDim.x) reinterpret_cast<uint4 *>(sm)[k] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int k = 0; k < 4; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(probe_smem_u32(bars + k)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(probe_smem_u32(&s_tmem)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (t == 0) {
    const uint32_t tmem = s_tmem + (uint32_t)(g * (512 / groups));
    const uint32_t a = probe_smem_u32(sm + g * (kProbeSmem / groups)), b = a + 4096;
    const uint64_t ad = probe_sdesc(a, 128, 256), bd = probe_sdesc(b, 128, 256);
    // kind::f16: D FP32, A and B BF16, both K-major; N >> 3 at bit 17, M >> 4 at bit 24
    const uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n_cols >> 3) << 17) |
                        ((uint32_t)(m_rows >> 4) << 24);
    const uint32_t mb = probe_smem_u32(bars + g);
    for (int pass = 0; pass < 2; ++pass) {
      const unsigned long long c0 = clock64();
      for (int r = 0; r < reps; ++r) {
        const uint32_t acc = r ? 1u : 0u;
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                     "l"(ad), "l"(bd), "r"(id), "r"(acc));
      }
      const unsigned long long c1 = clock64();
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
      bool done = false;
      for (long long it = 0; it < (1ll << 24) && !done; ++it) {
        uint32_t d;
        asm volatile("{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, P;\n\t}\n"
                     : "=r"(d) : "r"(mb), "r"((uint32_t)pass) : "memory");
        done = d != 0;
      }
      const unsigned long long c2 = clock64();
      if (!done) { atomicOr(status, kStatusTimeout); break; }
      if (pass == 1) { cycles[2 * g] = c1 - c0; cycles[2 * g + 1] = c2 - c0; }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(512));
}

}  // namespace

}  // namespace dags

using namespace dags;

extern "C" int dags_measure_mma(int32_t m_rows, int32_t n_cols, int32_t groups, int32_t reps, double *mac_per_cycle,
                                double *cycles_per_mma) {
  if (!(m_rows == 64 || m_rows == 128) || !(groups == 1 || groups == 2 || groups == 4) || n_cols < 16 || n_cols > 256 || n_cols % 16 ||
      n_cols > 512 / groups || 4096 + n_cols * 32 > kProbeSmem / groups || reps < 1 || reps > 4096 ||
      !mac_per_cycle)
    return DAGS_E_INVAL;
  unsigned long long *d_cyc = nullptr;
  uint32_t *d_status = nullptr;
  if (cudaMalloc(&d_cyc, 8 * sizeof(unsigned long long)) != cudaSuccess) return DAGS_E_CUDA;
  cudaError_t e = cudaMalloc(&d_status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(d_cyc, 0, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(uint32_t));
  if (e == cudaSuccess) {
    mma_probe_kernel<<<1, 128 * groups>>>(groups, m_rows, n_cols, reps, d_cyc, d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  unsigned long long h[8] = {0};
  uint32_t st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(h, d_cyc, sizeof(h), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&st, d_status, sizeof(st), cudaMemcpyDeviceToHost);
  cudaFree(d_cyc);
  cudaFree(d_status);
  if (e != cudaSuccess) return DAGS_E_CUDA;
  if (st) return DAGS_E_TIMEOUT;
  double tot = 0.0, iss = 0.0;
  for (int g = 0; g < groups; ++g) { iss += (double)h[2 * g]; tot += (double)h[2 * g + 1]; }
  tot /= groups;
  iss /= groups;
  if (!(tot > 0.0)) return DAGS_E_CUDA;
  *mac_per_cycle = (double)m_rows * n_cols * 16.0 * reps * groups / tot;
  if (cycles_per_mma) *cycles_per_mma = iss / reps;
  return DAGS_OK;
}

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
