// Learned per-pixel MP proposal network on the 5th-generation tensor cores
// (tcgen05, sm_103a): BF16 operands staged in shared memory, FP32
// accumulators in tensor memory (TMEM), one elected thread issuing the MMAs,
// completion tracked by an mbarrier.
//
// Network (per pixel, NHWC): z1 = W1 x + b1 (1x1, 8 -> 32), a1 = bf16(relu);
// z2 = conv3x3(a1) + b2 (32 -> 32, zero pad), a2 = bf16(relu); z3 = W3 a2 +
// b3, a3 = bf16(relu); y = sigmoid(w4 . a3 + b4).
//
// mpnet_fwd_kernel: persistent, one CTA (4 warps) per SM; a tile is 128
// consecutive pixels of one image row. Per tile:
//   1. the 3 x 130 halo pixels' inputs (8 channels, padded to K = 16) are
//      staged as a K-major operand; 4 MMAs (M = 128, N = 32, K = 16) give z1;
//   2. the epilogue applies bias, ReLU and BF16 rounding (zero outside the
//      image: the convolution pads a1 with zeros) into a halo buffer, from
//      which the im2col operand (128 x 288) is gathered; 18 MMAs give z2;
//   3. a2 is staged (128 x 32); 2 MMAs give z3;
//   4. the last epilogue computes a3, the 32-term dot product with w4 and
//      the sigmoid in FP32 and writes y (and, for training, a1 a2 a3).
// Shared-memory operands use the canonical no-swizzle K-major layout: 8x16-
// byte core matrices, row groups of 8 rows, LBO = 128 B between core
// matrices along K, SBO = (K / 8) * 128 B between row groups.
#include <cuda_bf16.h>

#include "common.cuh"

namespace dags {

namespace {

constexpr int kNetThreads = 128;          // 4 warps = one warpgroup over the 128 TMEM lanes
constexpr int kTileW = 128;               // pixels per tile (MMA M)
constexpr int kHaloW = kTileW + 2;        // 130
constexpr int kHaloRows = 3 * kHaloW;     // 390
constexpr int kHaloPad = 512;             // rows of the first operand (4 M-blocks)
constexpr int kCh = 32;
constexpr int kK2 = 9 * kCh;              // 288
constexpr uint32_t kTmemCols = 256;       // D1: 0..127, D2: 128..159, D3: 160..191
constexpr long long kSpinLimit = 1ll << 22;

// Byte offsets inside the weight blob (declared in dags.h).
constexpr int kOffW1 = 0, kOffW2 = 1024, kOffW3 = 19456, kOffW4 = 21504, kOffB1 = 21568, kOffB2 = 21696,
              kOffB3 = 21824, kOffB4 = 21952;

// Dynamic shared-memory layout (bytes, 128-aligned).
constexpr int kSW1 = 0;                                   // 32 x 16 bf16
constexpr int kSW2 = kSW1 + 1024;                         // 32 x 288
constexpr int kSW3 = kSW2 + 32 * kK2 * 2;                 // 32 x 32
constexpr int kSA1 = kSW3 + 2048;                         // 512 x 16
constexpr int kSH1 = kSA1 + kHaloPad * 16 * 2;            // 390 x 32 (plain rows of 64 B)
constexpr int kSA2 = kSH1 + ((kHaloRows * 64 + 127) / 128) * 128;  // 128 x 288
constexpr int kSA3 = kSA2 + kTileW * kK2 * 2;             // 128 x 32
constexpr int kSPar = kSA3 + kTileW * kCh * 2;            // b1 b2 b3 w4 (fp32) b4
constexpr int kSBar = kSPar + (4 * kCh + 4) * 4;          // mbarrier + tmem address
constexpr int kSmemBytes = kSBar + 64;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) of a K-major bf16 operand with K columns
// in the no-swizzle core-matrix layout.
__device__ __forceinline__ uint32_t core_off(int row, int k, int K) {
  return (uint32_t)(((row >> 3) * (K >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of sm_100-class tcgen05
  return d;                 // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Bounded wait on an mbarrier phase; false if the limit ran out.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ float bf16_round_f(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Writes 32 bf16 (as 16 packed words) into row `row` of a K-major operand
// with K columns, at column offset k0 (multiple of 8).
__device__ __forceinline__ void store_row32(uint8_t *base, int row, int k0, int K, const uint32_t *w) {
#pragma unroll
  for (int g = 0; g < 4; ++g)
    *reinterpret_cast<uint4 *>(base + core_off(row, k0 + 8 * g, K)) =
        make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
}

__global__ void __launch_bounds__(kNetThreads, 1)
mpnet_fwd_kernel(const uint8_t *__restrict__ weights, const uint4 *__restrict__ feats, int batch, int W, int H,
                 float *__restrict__ out, uint16_t *__restrict__ acts, uint32_t *__restrict__ status) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t *sW1 = smem + kSW1, *sW2 = smem + kSW2, *sW3 = smem + kSW3;
  uint8_t *sA1 = smem + kSA1, *sH1 = smem + kSH1, *sA2 = smem + kSA2, *sA3 = smem + kSA3;
  float *sb1 = reinterpret_cast<float *>(smem + kSPar), *sb2 = sb1 + kCh, *sb3 = sb2 + kCh, *sw4 = sb3 + kCh;
  float *sb4 = sw4 + kCh;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kSBar);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + kSBar + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights into the K-major operand layouts; biases and w4 as FP32
  const uint16_t *gw1 = reinterpret_cast<const uint16_t *>(weights + kOffW1);
  const uint16_t *gw2 = reinterpret_cast<const uint16_t *>(weights + kOffW2);
  const uint16_t *gw3 = reinterpret_cast<const uint16_t *>(weights + kOffW3);
  for (int e = tid; e < 32 * 16; e += kNetThreads)
    *reinterpret_cast<uint16_t *>(sW1 + core_off(e / 16, e % 16, 16)) = gw1[e];
  for (int e = tid; e < 32 * kK2; e += kNetThreads)
    *reinterpret_cast<uint16_t *>(sW2 + core_off(e / kK2, e % kK2, kK2)) = gw2[e];
  for (int e = tid; e < 32 * 32; e += kNetThreads)
    *reinterpret_cast<uint16_t *>(sW3 + core_off(e / 32, e % 32, 32)) = gw3[e];
  if (tid < kCh) {
    sb1[tid] = reinterpret_cast<const float *>(weights + kOffB1)[tid];
    sb2[tid] = reinterpret_cast<const float *>(weights + kOffB2)[tid];
    sb3[tid] = reinterpret_cast<const float *>(weights + kOffB3)[tid];
    sw4[tid] = __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(weights + kOffW4)[tid]);
  }
  if (tid == 0) {
    sb4[0] = reinterpret_cast<const float *>(weights + kOffB4)[0];
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the zero half of the first operand (input channels 8-15) never changes
  for (int h = tid; h < kHaloPad; h += kNetThreads)
    *reinterpret_cast<uint4 *>(sA1 + core_off(h, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = *s_tmem;
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
  uint32_t phase = 0;
  bool ok = true;

  const int tiles_x = (W + kTileW - 1) / kTileW;
  const long long ntiles = (long long)batch * H * tiles_x;
  for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int tx = (int)(t % tiles_x);
    const int y = (int)((t / tiles_x) % H);
    const int b = (int)(t / ((long long)tiles_x * H));
    const int x0 = tx * kTileW;
    const uint4 *fb = feats + (size_t)b * H * W;

    // 1. halo inputs -> first operand (rows h = r * 130 + c; x = x0 - 1 + c)
    for (int h = tid; h < kHaloPad; h += kNetThreads) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (h < kHaloRows) {
        const int r = h / kHaloW, c = h % kHaloW;
        const int yy = y - 1 + r, xx = x0 - 1 + c;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = __ldg(fb + (size_t)yy * W + xx);
      }
      *reinterpret_cast<uint4 *>(sA1 + core_off(h, 0, 16)) = v;
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
#pragma unroll
      for (int mb = 0; mb < 4; ++mb)
        mma_bf16(tmem + mb * 32, sdesc(smem_u32(sA1) + mb * 4096, 128, 256), sdesc(smem_u32(sW1), 128, 256),
                 idesc_bf16(128, 32), 0u);
      mma_commit(bar);
    }
    ok = bar_wait(bar, phase);
    phase ^= 1u;
    tc_after_sync();

    // 2. z1 -> a1 (zero outside the image) -> halo buffer
    for (int mb = 0; mb < 4; ++mb) {
      float z[32];
      tmem_ld32(tmem + lane_base + mb * 32, z);
      const int h = mb * 128 + 32 * warp + lane;
      if (h < kHaloRows) {
        const int r = h / kHaloW, c = h % kHaloW;
        const int yy = y - 1 + r, xx = x0 - 1 + c;
        const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
        uint32_t w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k)
          w[k] = in ? pack_bf16x2(fmaxf(z[2 * k] + sb1[2 * k], 0.f), fmaxf(z[2 * k + 1] + sb1[2 * k + 1], 0.f)) : 0u;
        uint4 *dst = reinterpret_cast<uint4 *>(sH1 + (size_t)h * 64);
#pragma unroll
        for (int g = 0; g < 4; ++g) dst[g] = make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
        if (acts && r == 1 && c >= 1 && c <= kTileW && xx < W) {
          uint4 *ga = reinterpret_cast<uint4 *>(acts + (((size_t)b * H + y) * W + xx) * 96);
#pragma unroll
          for (int g = 0; g < 4; ++g) ga[g] = make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
        }
      }
    }
    tc_before_sync();
    __syncthreads();
    // im2col: row p, columns tap * 32 + channel, tap = ky * 3 + kx -> halo
    // pixel (ky, p + kx)
    {
      const int p = tid;
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        const uint4 *src = reinterpret_cast<const uint4 *>(sH1 + (size_t)(ky * kHaloW + p + kx) * 64);
#pragma unroll
        for (int g = 0; g < 4; ++g)
          *reinterpret_cast<uint4 *>(sA2 + core_off(p, tap * 32 + 8 * g, kK2)) = src[g];
      }
    }
    fence_async_smem();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
      for (int c = 0; c < kK2 / 16; ++c)
        mma_bf16(tmem + 128, sdesc(smem_u32(sA2) + c * 256, 128, (kK2 / 8) * 128),
                 sdesc(smem_u32(sW2) + c * 256, 128, (kK2 / 8) * 128), idesc_bf16(128, 32), c > 0 ? 1u : 0u);
      mma_commit(bar);
    }
    ok = ok && bar_wait(bar, phase);
    phase ^= 1u;
    tc_after_sync();

    // 3. z2 -> a2 -> third operand
    const int p = 32 * warp + lane;
    {
      float z[32];
      tmem_ld32(tmem + lane_base + 128, z);
      uint32_t w[16];
#pragma unroll
      for (int k = 0; k < 16; ++k)
        w[k] = pack_bf16x2(fmaxf(z[2 * k] + sb2[2 * k], 0.f), fmaxf(z[2 * k + 1] + sb2[2 * k + 1], 0.f));
      store_row32(sA3, p, 0, 32, w);
      if (acts && x0 + p < W) {
        uint4 *ga = reinterpret_cast<uint4 *>(acts + (((size_t)b * H + y) * W + x0 + p) * 96 + 32);
#pragma unroll
        for (int g = 0; g < 4; ++g) ga[g] = make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
      }
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
      for (int c = 0; c < 2; ++c)
        mma_bf16(tmem + 160, sdesc(smem_u32(sA3) + c * 256, 128, 512), sdesc(smem_u32(sW3) + c * 256, 128, 512),
                 idesc_bf16(128, 32), c > 0 ? 1u : 0u);
      mma_commit(bar);
    }
    ok = ok && bar_wait(bar, phase);
    phase ^= 1u;
    tc_after_sync();

    // 4. z3 -> a3 -> y
    {
      float z[32];
      tmem_ld32(tmem + lane_base + 160, z);
      float acc = sb4[0];
      uint32_t w[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float a0 = bf16_round_f(fmaxf(z[2 * k] + sb3[2 * k], 0.f));
        const float a1v = bf16_round_f(fmaxf(z[2 * k + 1] + sb3[2 * k + 1], 0.f));
        acc += a0 * sw4[2 * k] + a1v * sw4[2 * k + 1];
        w[k] = pack_bf16x2(a0, a1v);
      }
      if (x0 + p < W) {
        const size_t pix = ((size_t)b * H + y) * W + x0 + p;
        out[pix] = 1.f / (1.f + expf(-acc));
        if (acts) {
          uint4 *ga = reinterpret_cast<uint4 *>(acts + pix * 96 + 64);
#pragma unroll
          for (int g = 0; g < 4; ++g) ga[g] = make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
        }
      }
    }
    tc_before_sync();
    __syncthreads();
  }
  if (!ok) {
    // a wait gave up: record it and give in-flight MMAs one more bounded wait
    // before the tensor memory is released
    if (tid == 0) atomicOr(status, kStatusTimeout);
    bar_wait(bar, phase ^ 1u);
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

cudaError_t launch_mpnet_forward(const void *weights, const uint16_t *feats, int batch, int W, int H, float *out,
                                 uint16_t *acts, uint32_t *status, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(mpnet_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)batch * H * ((W + kTileW - 1) / kTileW);
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  if (grid <= 0) return cudaSuccess;
  mpnet_fwd_kernel<<<grid, kNetThreads, kSmemBytes, s>>>(static_cast<const uint8_t *>(weights),
                                                         reinterpret_cast<const uint4 *>(feats), batch, W, H, out,
                                                         acts, status);
  return cudaGetLastError();
}

}  // namespace dags
