// Learned per-pixel MP proposal network on the 5th-generation tensor cores
// (tcgen05, sm_103a): BF16 operands staged in shared memory, FP32
// accumulators in tensor memory (TMEM), one elected thread per warpgroup
// issuing the MMAs, completion tracked by mbarriers, inputs fetched by TMA or
// cp.async.
//
// Network (per pixel, NHWC): z1 = W1 x + b1 (1x1, 8 -> 32), a1 = bf16(relu);
// z2 = conv3x3(a1) + b2 (32 -> 32, zero pad), a2 = bf16(relu); z3 = W3 a2 +
// b3, a3 = bf16(relu); y = sigmoid(w4 . a3 + b4).
//
// mpnet_fwd_kernel   inference (and the training forward): three warpgroups
//                    per CTA (four epilogue warps and one MMA-issuing
//                    control warp each) walk 128-pixel column strips row by
//                    row in a software pipeline (see its comment).
// mpnet_bwd1_kernel  training: BCE gradient, dz3, da2 = dz3 W3 and dz2; the
//                    weight gradients dW3, dw4 accumulated in TMEM.
// mpnet_bwd2_kernel  training: da1 by the transposed 3x3 convolution, dz1;
//                    dW2 per tap and dW1 accumulated in TMEM.
// mpnet_adam_kernel  Adam on the FP32 master weights, BF16 blob refresh.
//
// Weights are staged once per CTA in the canonical no-swizzle K-major
// layout (8x16-byte core matrices, LBO = 128 B between core matrices along K,
// SBO = (K / 8) * 128 B between 8-row groups); activations use the
// row-contiguous chunk layout described at the forward kernel.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace dags {

namespace {

constexpr int kNetThreads = 128;          // 4 warps = one warpgroup over the 128 TMEM lanes
constexpr int kTileW = 128;               // pixels per tile (MMA M)
constexpr int kHaloW = kTileW + 2;        // 130
constexpr int kHaloRows = 3 * kHaloW;     // 390
constexpr int kCh = 32;
constexpr int kK2 = 9 * kCh;              // 288
constexpr long long kSpinLimit = 1ll << 22;

// Byte offsets inside the weight blob (declared in dags.h).
constexpr int kOffW1 = 0, kOffW2 = 1024, kOffW3 = 19456, kOffW4 = 21504, kOffB1 = 21568, kOffB2 = 21696,
              kOffB3 = 21824, kOffB4 = 21952;

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
__device__ __forceinline__ bool bar_wait_n(uint64_t *bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
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
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) { return bar_wait_n(bar, parity, kSpinLimit); }

// Failure-path self-test: one thread waits, with the given iteration limit,
// on an mbarrier phase that nothing completes, then records the timeout in
// the status word as every kernel's bounded waits do.
__global__ void selftest_wait_kernel(uint32_t *status, long long limit) {
  __shared__ uint64_t bar;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!bar_wait_n(&bar, 0u, limit)) atomicOr(status, kStatusTimeout);
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



// Forward kernel: kGroups warpgroups per CTA, each running its own stream
// of work units with its own operands, TMEM columns and mbarriers. A
// warpgroup is four epilogue warps (TMEM lane quadrants 0..3: 128 pixels)
// and one control warp whose lane 0 issues the MMAs and the TMA fetches.
//
// Work unit: a 128-pixel-wide column strip of one image over a segment of
// output rows [y0, y1). The warpgroup walks down the strip computing a1 for
// one 130-pixel halo row at a time (rows y0 - 1 .. y1; x0 - 1 .. x0 + 128);
// every a1 row is computed once per unit (plus two boundary rows).
//
// The 3 x 3 convolution reads each a1 row once: a1 row k meets all three
// kernel rows in one N = 96 product (K = the three column taps x 32
// channels), whose 32-column thirds go to the outputs k, k - 1 and k - 2
// (kernel rows 0, 1, 2). Output j accumulates in TMEM slot j mod 3 of a ring
// of three; because the thirds of one MMA are contiguous columns, the kernel
// rows are stacked in the order that puts each into the slot of its output
// (one of three row permutations of the weights, chosen by k mod 3). A slot
// starts as the layer-2 bias: a K = 16 MMA of per-row constants (1, 1, 0, ...)
// with the bias as a BF16 column pair (hi, lo), before the first product
// that reaches it. The A operand of an MMA is read from shared memory once
// per instruction, so one N = 96 product per row costs about as much as
// 1.4 products of N = 32 instead of three.
//
// Pipeline, step s of a unit with nO output rows (nA = nO + 2 a1 rows):
//   control: wait for the previous step's epilogues; fetch the input of a1
//     row s + 2; z1 of a1 row s (s < nA), commit; the bias of slot
//     (s - 1) mod 3 and the product of a1 row s - 1 (1 <= s <= nA) with
//     z3 of output row s - 4 (4 <= s <= nA + 1) issued between its first
//     MMAs, commit after z3, commit after the product.
//   epilogues: epilogue 1 once z1 is done (a1 row s into buffer s mod 2; the
//     halo pixels 128 and 129 on the CUDA cores); epilogue 3 once z3 is done
//     (a3, the dot product with w4 and the sigmoid of output row s - 4);
//     epilogue 2 once the product is done (output row s - 3 complete in slot
//     s mod 3: a2 into its buffer).
// The product runs on the tensor core while epilogues 1 and 3 run. Every
// buffer is rewritten only after the barrier that follows its last reader:
// the a1 buffer s mod 2 was last read by the product of step s - 1, which
// the commits of step s cover; the a2 buffer by the z3 of step s; a slot
// is re-biased one step after epilogue 2 read it. Out-of-image rows and
// columns read as zero.
//
// Operand layouts (no swizzle): "row-contiguous chunks" - chunk c holds
// channels 8c..8c+7 of every row as one 16-byte line, rows consecutive (SBO =
// 128 B between 8-row groups, LBO = the chunk stride). An MMA may then start
// at any row, which makes the 3 x 3 convolution an implicit GEMM: column tap
// kx reads the a1 row at rows kx + p directly, no im2col.
//
// The first layer's bias rides in its MMA the same way as the second's:
// a K-chunk of per-row constants (1, 1, 0, ..., 0) meets a B column pair
// (hi, lo) with hi = bf16(b), lo = bf16(b - hi) (|hi + lo - b| <= 2^-17 |b|).
// The third layer's bias is added in FP32 in its epilogue.
constexpr int kGroups = 3;
constexpr int kFwdThreads = 160 * kGroups;              // 4 epilogue warps + 1 control warp per warpgroup
constexpr int kBars = 8;                                // mbarriers per warpgroup
constexpr int kRowBytes = kHaloW * 16;                  // 2080 = the TMA box (8 x 130 x 1 x 1 bf16)
constexpr int kInBuf = 2176;                            // one input row (+ pad)
constexpr int kInBufs = 3;
constexpr int kSlotRows = 136;
constexpr int kSlotChunk = kSlotRows * 16;              // 2176
constexpr int kSlotBytes = 4 * kSlotChunk;              // 8704: one a1 row, four chunks
constexpr int kA1Bufs = 2;
constexpr int kA2Bytes = 4 * kTileW * 16;               // 8192
// per warpgroup: three input rows, ones (the bias chunks: 256 rows of
// (1, 1, 0, ...), of which an MMA reads 128 per K-chunk), two a1 rows, a2.
constexpr int kWgOnes = kInBufs * kInBuf, kWgA1 = kWgOnes + 4096;
constexpr int kWgA2 = kWgA1 + kA1Bufs * kSlotBytes;
constexpr int kWgBytes = kWgA2 + kA2Bytes;              // 36224
constexpr int kW2Perm = 96 * 96 * 2;                    // 18432: one stacking of the three kernel rows
constexpr int kFW1 = kGroups * kWgBytes, kFW2 = kFW1 + 1024, kFW3 = kFW2 + 3 * kW2Perm, kFB2 = kFW3 + 2048,
              kFB3 = kFB2 + 1024, kFW1f = kFB3 + 512, kFPar = kFW1f + 1024;
constexpr int kFBar = kFPar + 256;
constexpr int kFwdSmem = kFBar + 256 + 1024;            // + alignment slack
constexpr uint32_t kWgCols = 160;                       // D1 +0..31, D3 +32..63, ring +64..159
constexpr uint32_t kColD1 = 0, kColD3 = 32, kColRing = 64;
static_assert(kGroups * kWgCols <= 512, "TMEM columns");
static_assert(kFwdSmem <= 227 * 1024, "shared memory");

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// BF16 pair (lo, hi) of relu(lo), relu(hi), round to nearest even.
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void tma_row(const CUtensorMap *map, uint32_t dst, uint64_t *bar, int x, int y, int b) {
  const uint32_t mb = smem_u32(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(kRowBytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(y), "r"(b), "r"(mb)
      : "memory");
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

struct FwdUnits {
  int tiles_x, segs, seg_rows;
  long long count;
};

__global__ void __launch_bounds__(kFwdThreads, 1)
mpnet_fwd_kernel(const __grid_constant__ CUtensorMap in_map, const uint8_t *__restrict__ weights, int batch, int W,
                 int H, FwdUnits units, float *__restrict__ out, uint16_t *__restrict__ acts,
                 uint32_t *__restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *sW1 = smem + kFW1, *sW2 = smem + kFW2, *sW3 = smem + kFW3, *sB2 = smem + kFB2;
  // FP32 copies: b3 (added in its epilogue), b1 as its BF16 (hi, lo) pair and
  // W1, for the two halo pixels computed on the CUDA cores
  float *sb3f = reinterpret_cast<float *>(smem + kFB3), *sb1h = sb3f + kCh, *sb1l = sb3f + 2 * kCh;
  float *sw1f = reinterpret_cast<float *>(smem + kFW1f);  // [32][8]
  float *sw4 = reinterpret_cast<float *>(smem + kFPar), *sb4 = sw4 + kCh;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kFBar);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + kFBar + 8 * kBars * kGroups);
  volatile uint32_t *s_fail = reinterpret_cast<volatile uint32_t *>(smem + kFBar + 8 * kBars * kGroups + 8);
  // threads 0..4*32*kGroups-1: the warpgroups' epilogue warps (warp w reads
  // TMEM lane quadrant w % 4); then one control warp per warpgroup
  const int tid = threadIdx.x, lane = tid & 31;
  const bool ctl = tid >= 4 * kGroups * 32;
  const int g = ctl ? (tid - 4 * kGroups * 32) >> 5 : tid >> 7, t = tid & 127, warp = t >> 5;
  uint8_t *wg = smem + g * kWgBytes;
  uint8_t *sA1 = wg + kWgA1, *sA2 = wg + kWgA2;
  // per warpgroup: in0..in2 (TMA), z1, z3, prod (MMA commits), ep (all
  // epilogues done), drain (the final wait)
  uint64_t *bar_in = bars + kBars * g, *bar_z1 = bar_in + 3, *bar_z3 = bar_in + 4, *bar_prod = bar_in + 5,
           *bar_ep = bar_in + 6, *bar_drain = bar_in + 7;

  // weights into the K-major core-matrix layouts; bias columns (hi, lo)
  const uint16_t *gw1 = reinterpret_cast<const uint16_t *>(weights + kOffW1);
  const uint16_t *gw2 = reinterpret_cast<const uint16_t *>(weights + kOffW2);
  const uint16_t *gw3 = reinterpret_cast<const uint16_t *>(weights + kOffW3);
  const float *gb1 = reinterpret_cast<const float *>(weights + kOffB1);
  const float *gb2 = reinterpret_cast<const float *>(weights + kOffB2);
  const float *gb3 = reinterpret_cast<const float *>(weights + kOffB3);
  for (int e = tid; e < 32 * 16; e += kFwdThreads) {
    const int o = e / 16, k = e % 16;
    const float bias = gb1[o], hi = __bfloat162float(__float2bfloat16_rn(bias));
    const uint16_t v = k < 8 ? gw1[e] : k == 8 ? bf16_bits(bias) : k == 9 ? bf16_bits(bias - hi) : (uint16_t)0;
    *reinterpret_cast<uint16_t *>(sW1 + core_off(o, k, 16)) = v;
    const float b2 = gb2[o], h2 = __bfloat162float(__float2bfloat16_rn(b2));
    const uint16_t v2 = k == 0 ? bf16_bits(b2) : k == 1 ? bf16_bits(b2 - h2) : (uint16_t)0;
    *reinterpret_cast<uint16_t *>(sB2 + core_off(o, k, 16)) = v2;
  }
  // the three stackings of the kernel rows: in stacking p, rows 32c + o hold
  // output channel o of kernel row ky = (p - c) mod 3; K = kx * 32 + channel
  for (int e = tid; e < 3 * 96 * 96; e += kFwdThreads) {
    const int p = e / (96 * 96), n = (e / 96) % 96, kk = e % 96;
    const int c = n >> 5, o = n & 31, kx = kk >> 5, ci = kk & 31, ky = (p - c + 3) % 3;
    *reinterpret_cast<uint16_t *>(sW2 + p * kW2Perm + core_off(n, kk, 96)) = gw2[o * kK2 + (ky * 3 + kx) * kCh + ci];
  }
  for (int e = tid; e < 32 * 32; e += kFwdThreads)
    *reinterpret_cast<uint16_t *>(sW3 + core_off(e / 32, e % 32, 32)) = gw3[e];
  for (int e = tid; e < kCh; e += kFwdThreads) {
    sb3f[e] = gb3[e];
    const float hi = __bfloat162float(__float2bfloat16_rn(gb1[e]));
    sb1h[e] = hi;
    sb1l[e] = __bfloat162float(__float2bfloat16_rn(gb1[e] - hi));
  }
  for (int e = tid; e < kCh * 8; e += kFwdThreads)
    sw1f[e] = __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(gw1)[(e / 8) * 16 + e % 8]);
  if (tid < kCh) sw4[tid] = __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(weights + kOffW4)[tid]);
  // the whole warpgroup area starts at zero (don't-care rows stay finite);
  // then the bias constants (1, 1, 0, ..., 0) of every row
  if (!ctl)
    for (int e = t; e < kWgBytes / 16; e += 128) {
      const bool one = e >= kWgOnes / 16 && e < kWgOnes / 16 + 256;   // one writer per line
      *reinterpret_cast<uint4 *>(wg + 16 * e) = make_uint4(one ? 0x3F803F80u : 0u, 0u, 0u, 0u);
    }
  if (tid == 0) {
    sb4[0] = reinterpret_cast<const float *>(weights + kOffB4)[0];
    for (int k = 0; k < kBars * kGroups; ++k) {
      const int kind = k % kBars;   // ep: one arrival per epilogue warp
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bars + k)), "r"(kind == 6 ? 4 : 1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int k = 0; k < kGroups; ++k) s_fail[k] = 0u;
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = *s_tmem + kWgCols * (uint32_t)g;
  const uint32_t wg_u32 = smem_u32(wg);
  const uint32_t ones = wg_u32 + kWgOnes;
  const long long stride = (long long)kGroups * gridDim.x;
  // unit u -> image b, strip x0, rows [y0, y1)
  auto unit = [&](long long u, int *b, int *x0, int *y0, int *y1) {
    const int seg = (int)(u % units.segs);
    const long long rest = u / units.segs;
    *x0 = (int)(rest % units.tiles_x) * kTileW;
    *b = (int)(rest / units.tiles_x);
    *y0 = seg * units.seg_rows;
    *y1 = min(*y0 + units.seg_rows, H);
  };
  uint32_t qbase = 0;          // a1 rows of the earlier units (input buffer and phase)
  uint32_t sc = 0;             // steps of the earlier units (epilogue barrier phase)
  uint32_t n_z1 = 0, n_z3 = 0, n_prod = 0;   // commits so far on each MMA barrier
  if (ctl) {
    // ------------------------------------------------------------ control
    if (lane == 0) {
      // bits 0..2 = TMA into in0..in2 pending (bits 8..10 = the parity of
      // that fetch's phase), bit 3 = MMAs issued since the last waited commit
      uint32_t in_flight = 0;
      bool ok = true;
      auto fetch = [&](uint32_t q, int x0, int r, int b) {   // input of the q-th a1 row of this warpgroup
        const uint32_t buf = q % kInBufs;
        tma_row(&in_map, wg_u32 + buf * kInBuf, bar_in + buf, x0 - 1, r, b);
        in_flight = (in_flight & ~(0x101u << buf)) | (1u << buf) | (((q / kInBufs) & 1u) << (8 + buf));
      };
      long long u = (long long)kGroups * blockIdx.x + g;
      if (u < units.count) {
        int b, x0, y0, y1;
        unit(u, &b, &x0, &y0, &y1);
        fetch(0, x0, y0 - 1, b);
        fetch(1, x0, y0, b);
      }
      for (; u < units.count && ok; u += stride) {
        int b, x0, y0, y1;
        unit(u, &b, &x0, &y0, &y1);
        const int nO = y1 - y0, nA = nO + 2;
        int nb = 0, nx0 = 0, ny0 = 0, ny1 = 0;
        const bool has_next = u + stride < units.count;
        if (has_next) unit(u + stride, &nb, &nx0, &ny0, &ny1);
        for (int s = 0; s < nA + 2; ++s, ++sc) {
          const bool d1 = s < nA, dp = s >= 1 && s <= nA, d3 = s >= 4;
          const uint32_t q = qbase + (uint32_t)s;
          if (s_fail[g]) { ok = false; break; }
          // the previous step's epilogues have read D1, D3 and their slot and
          // written a1 and a2; the input buffer of a1 row s - 1 is free
          if (sc > 0) ok = bar_wait(bar_ep, (sc - 1) & 1u);
          if (!ok) break;
          tc_after_sync();
          if (s + 2 < nA) fetch(q + 2, x0, y0 + s + 1, b);
          else if (has_next && s + 2 - nA < 2) fetch(q + 2, nx0, ny0 - 1 + (s + 2 - nA), nb);
          // The MMAs of one accumulator run one after another (about 68
          // cycles apart); the three independent groups are interleaved so
          // that the tensor core overlaps them: the bias of slot (s - 1) mod 3
          // and the product of a1 row s - 1 (1 <= s <= nA), with z1 of a1 row
          // s (s < nA; halo pixels 0..127, the last two on the CUDA cores)
          // and z3 of output row s - 4 (4 <= s <= nA + 1) between its steps.
          // A commit covers everything issued before it.
          const int k = s - 1, pk = (k + 3) % 3;
          const uint32_t a1 = smem_u32(sA1) + (uint32_t)(k & 1) * kSlotBytes;
          auto prod = [&](int j) {   // j = 2 * kx + hh
            const int kx = j >> 1, hh = j & 1;
            mma_bf16(tmem + kColRing, sdesc(a1 + 2 * hh * kSlotChunk + kx * 16, kSlotChunk, 128),
                     sdesc(smem_u32(sW2) + pk * kW2Perm + j * 256, 128, 1536), idesc_bf16(128, 96), 1u);
          };
          auto z3 = [&](int h) {
            const uint32_t a2 = smem_u32(sA2);
            mma_bf16(tmem + kColD3, sdesc(a2 + 2 * h * (kTileW * 16), kTileW * 16, 128),
                     sdesc(smem_u32(sW3) + h * 256, 128, 512), idesc_bf16(128, 32), h ? 1u : 0u);
          };
          if (d1) {
            const uint32_t buf = q % kInBufs;
            ok = bar_wait(bar_in + buf, (q / kInBufs) & 1u);
            if (!ok) break;
            in_flight = (in_flight & ~(1u << buf)) | 8u;
            const uint32_t in = wg_u32 + buf * kInBuf, lbo = ones - in;
            mma_bf16(tmem + kColD1, sdesc(in, lbo, 128), sdesc(smem_u32(sW1), 128, 256), idesc_bf16(128, 32), 0u);
            mma_commit(bar_z1);
            ++n_z1;
          }
          in_flight |= 8u;
          if (dp) {
            mma_bf16(tmem + kColRing + 32 * (uint32_t)pk, sdesc(ones, 2048, 128), sdesc(smem_u32(sB2), 128, 256),
                     idesc_bf16(128, 32), 0u);
            prod(0);
          }
          if (d3) z3(0);
          if (dp) prod(1);
          if (d3) {
            z3(1);
            mma_commit(bar_z3);
            ++n_z3;
          }
          if (dp) {
#pragma unroll
            for (int j = 2; j < 6; ++j) prod(j);
            mma_commit(bar_prod);
            ++n_prod;
          }
        }
        qbase += (uint32_t)nA;
      }
      if (!ok) {
        // a wait gave up: record it, stop the epilogue warps, and give what
        // may still be in flight one more bounded wait before the tensor
        // memory is released
        s_fail[g] = 1u;
        atomicOr(status, kStatusTimeout);
        for (uint32_t buf = 0; buf < kInBufs; ++buf)
          if (in_flight & (1u << buf)) bar_wait(bar_in + buf, (in_flight >> (8 + buf)) & 1u);
      }
      // the last commit (and everything before it) completes
      if (in_flight & 8u) {
        mma_commit(bar_drain);
        bar_wait(bar_drain, 0u);
      }
    }
  } else {
    // ---------------------------------------------------------- epilogues
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int p = 32 * warp + lane;
    bool ok = true;
    for (long long u = (long long)kGroups * blockIdx.x + g; u < units.count && ok; u += stride) {
      int b, x0, y0, y1;
      unit(u, &b, &x0, &y0, &y1);
      const int nO = y1 - y0, nA = nO + 2;
      for (int s = 0; s < nA + 2; ++s, ++sc) {
        const bool d1 = s < nA, d2 = s >= 3 && s <= nA, d3 = s >= 4;
        const uint32_t q = qbase + (uint32_t)s;
        if (s_fail[g]) { ok = false; break; }
        // epilogue 1: a1 row r = y0 - 1 + s (zero outside the image) -> a1
        // buffer s mod 2; buffer pixel i <-> x = x0 - 1 + i
        if (d1) {
          ok = bar_wait(bar_z1, n_z1 & 1u);
          ++n_z1;
          if (!ok) break;
          tc_after_sync();
          const int r = y0 - 1 + s;
          const bool row_in = r >= 0 && r < H, own_row = r >= y0 && r < y1;
          uint8_t *a1 = sA1 + (s & 1) * kSlotBytes;
          {
            float z[32];
            tmem_ld32(tmem + lane_base + kColD1, z);
            const int i = p, xx = x0 - 1 + i;
            const bool in = row_in && xx >= 0 && xx < W;
            uint32_t w[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) w[e] = in ? relu_bf16x2(z[2 * e], z[2 * e + 1]) : 0u;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              *reinterpret_cast<uint4 *>(a1 + c * kSlotChunk + i * 16) =
                  make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
            if (acts && own_row && i >= 1 && xx < W) {
              uint4 *ga = reinterpret_cast<uint4 *>(acts + (((size_t)b * H + r) * W + xx) * 96);
#pragma unroll
              for (int c = 0; c < 4; ++c) ga[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
            }
          }
          // halo pixels i = 128 (warp 1) and 129 (warp 2): lane = output
          // channel, z1 = W1 x + hi + lo in FP32 from the row's input buffer
          // (refilled only after this step's epilogues)
          if (warp == 1 || warp == 2) {
            ok = bar_wait(bar_in + q % kInBufs, (q / kInBufs) & 1u);
            const int i = kTileW - 1 + warp, xx = x0 - 1 + i, c = lane;
            const bool in = row_in && xx >= 0 && xx < W;
            const uint4 xv = *reinterpret_cast<const uint4 *>(wg + (q % kInBufs) * kInBuf + i * 16);
            const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
            float zc = 0.f;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              const uint32_t bits = (kk & 1) ? (xw[kk >> 1] & 0xFFFF0000u) : (xw[kk >> 1] << 16);
              zc = fmaf(__uint_as_float(bits), sw1f[c * 8 + kk], zc);
            }
            zc = (zc + sb1h[c]) + sb1l[c];
            const uint16_t a = in ? bf16_bits(fmaxf(zc, 0.f)) : (uint16_t)0;
            *reinterpret_cast<uint16_t *>(a1 + (c >> 3) * kSlotChunk + i * 16 + (c & 7) * 2) = a;
            if (acts && own_row && i <= kTileW && xx < W) acts[(((size_t)b * H + r) * W + xx) * 96 + c] = a;
          }
          fence_async_smem();
        }
        // epilogue 3: a3, the dot product with w4 and the sigmoid of output
        // row y0 + s - 4
        if (ok && d3) {
          ok = bar_wait(bar_z3, n_z3 & 1u);
          ++n_z3;
          if (!ok) break;
          tc_after_sync();
          const int y = y0 + s - 4;
          float z[32];
          tmem_ld32(tmem + lane_base + kColD3, z);
          float acc = sb4[0];
          uint32_t w[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            w[e] = relu_bf16x2(z[2 * e] + sb3f[2 * e], z[2 * e + 1] + sb3f[2 * e + 1]);
            acc += __uint_as_float(w[e] << 16) * sw4[2 * e] + __uint_as_float(w[e] & 0xFFFF0000u) * sw4[2 * e + 1];
          }
          if (x0 + p < W) {
            const size_t pix = ((size_t)b * H + y) * W + x0 + p;
            out[pix] = __fdividef(1.f, 1.f + __expf(-acc));
            if (acts) {
              uint4 *ga = reinterpret_cast<uint4 *>(acts + pix * 96 + 64);
#pragma unroll
              for (int c = 0; c < 4; ++c) ga[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
            }
          }
        }
        // epilogue 2: output row y0 + s - 3 is complete in slot s mod 3 (its
        // bias included) -> a2 buffer
        if (ok && d2) {
          ok = bar_wait(bar_prod, n_prod & 1u);
          ++n_prod;
          if (!ok) break;
          tc_after_sync();
          const int y = y0 + s - 3;
          float z[32];
          tmem_ld32(tmem + lane_base + kColRing + 32 * (uint32_t)(s % 3), z);
          uint32_t w[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) w[e] = relu_bf16x2(z[2 * e], z[2 * e + 1]);
#pragma unroll
          for (int c = 0; c < 4; ++c)
            *reinterpret_cast<uint4 *>(sA2 + c * (kTileW * 16) + p * 16) =
                make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
          if (acts && x0 + p < W) {
            uint4 *ga = reinterpret_cast<uint4 *>(acts + (((size_t)b * H + y) * W + x0 + p) * 96 + 32);
#pragma unroll
            for (int c = 0; c < 4; ++c) ga[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
          }
          fence_async_smem();
        } else if (ok && s >= 1 && s <= nA) {
          // a product without a complete output row: its commit still has a
          // phase to pass
          ok = bar_wait(bar_prod, n_prod & 1u);
          ++n_prod;
          if (!ok) break;
        }
        tc_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_ep);
        if (!ok) break;
      }
      qbase += (uint32_t)nA;
    }
    if (!ok) s_fail[g] = 1u;
  }
  if (!ctl && s_fail[g] && t == 0) atomicOr(status, kStatusTimeout);
  tc_before_sync();
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*s_tmem), "r"(512));
}

// ----------------------------------------------------------------- training
//
// Mean binary cross-entropy over pixels with target >= 0; the backward
// treats the BF16 rounding of activations as the identity. Weight gradients
// reduce over pixels: per 128-pixel tile they are UMMAs with the pixels as
// the K dimension (A = activations channel-major, B = upstream gradients
// channel-major), accumulated in TMEM across all tiles of a persistent CTA
// and added to the global FP32 gradient once per CTA. A row of ones appended
// to A gives the bias gradients from the same MMAs. The weight-gradient MMAs
// are M = 64, the data MMAs M = 128; A rows past the real ones are
// don't-care rows whose D rows are ignored.

constexpr int kGW1 = 0, kGW2 = 512, kGW3 = 512 + 9216, kGw4 = 512 + 9216 + 1024, kGb1 = kGw4 + 32,
              kGb2 = kGb1 + 32, kGb3 = kGb2 + 32, kGb4 = kGb3 + 32, kGTotal = kGb4 + 1;   // 10881 floats


__global__ void mpnet_count_kernel(const float *__restrict__ target, long long n, float *__restrict__ inv_n,
                                   float *__restrict__ loss_acc) {
  __shared__ unsigned s_cnt;
  if (threadIdx.x == 0) s_cnt = 0u;
  __syncthreads();
  unsigned c = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c += target[i] >= 0.f ? 1u : 0u;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned *>(inv_n) + 1, s_cnt);   // count in word 1
  (void)loss_acc;
}

__global__ void mpnet_count_finish_kernel(float *inv_n) {
  const unsigned c = reinterpret_cast<unsigned *>(inv_n)[1];
  inv_n[0] = c ? 1.f / (float)c : 0.f;
}

// Backward operand layouts. All activations and gradients are staged as
// row-contiguous chunks (chunk c = channels 8c..8c+7 of every pixel as one
// 16-byte line, pixels consecutive), straight from their pixel-major (NHWC)
// form with 16-byte copies. The same buffer is read two ways:
//   K-major, M = pixels, K = channels: SBO = 128 B (8 pixels), LBO = chunk
//     stride (the next 8 channels) - the data GEMMs (da2, the transposed
//     convolution for da1, with shifted start rows as in the forward);
//   MN-major, MN = channels, K = pixels (instruction-descriptor bits 15/16):
//     SBO = chunk stride (the next 8 channels), LBO = 128 B (the next 8
//     pixels) - the weight-gradient GEMMs, which reduce over pixels.
// Weight-gradient MMAs are M = 64 over 32 (+1) real channel rows (M = 64
// reads half the A operand of M = 128, and at N = 32 the MMA rate is bound
// by the operands' shared-memory reads): the rows past them read whatever
// follows in shared memory (in bounds), and their D rows are never read. A
// chunk of (1, 0, ..., 0) after the real channels gives the bias gradient in
// D row 32.

// The D row an M = 64 accumulator keeps in TMEM lane `lane`: rows 16q ..
// 16q + 15 sit in lanes 32q .. 32q + 15 of lane quadrant q (measured on the
// device; lanes 16..31 of each quadrant hold none: -1).
__device__ __forceinline__ int m64_row(int lane) { return (lane & 31) < 16 ? 16 * (lane >> 5) + (lane & 31) : -1; }

__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N) {
  return idesc_bf16(M, N) | (1u << 15) | (1u << 16);   // A and B MN-major
}

constexpr int kChunkPx = kTileW * 16;                    // 2048: one chunk of a 128-pixel tile

// bwd1 shared memory: a2 and a3 (5 chunks each: 4 real + ones, then 11 more
// readable chunks for the M = 128 MMA), dz3 (4 chunks), dz4 (2 chunks), W3^T
constexpr int kB1A2 = 0;
constexpr int kB1A3 = kB1A2 + 5 * kChunkPx;
constexpr int kB1Dz3 = kB1A3 + 5 * kChunkPx;
constexpr int kB1Dz4 = kB1Dz3 + 4 * kChunkPx;
constexpr int kB1W3T = kB1Dz4 + 2 * kChunkPx;
constexpr int kB1Par = kB1W3T + 2048;
constexpr int kB1Bar = kB1Par + 128;
constexpr int kB1Span = 16 * kChunkPx;                    // the farthest MN-major read from kB1A3
constexpr int kB1Smem = (kB1A3 + kB1Span > kB1Bar + 64 ? kB1A3 + kB1Span : kB1Bar + 64);

__device__ __forceinline__ void st_chunks(uint8_t *base, int stride, int row, const uint32_t *w) {
#pragma unroll
  for (int c = 0; c < 4; ++c)
    *reinterpret_cast<uint4 *>(base + c * stride + row * 16) = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
}

__global__ void __launch_bounds__(kNetThreads)
mpnet_bwd1_kernel(const uint8_t *__restrict__ weights, const float *__restrict__ y, const float *__restrict__ target,
                  const uint16_t *__restrict__ acts, int batch, int W, int H, const float *__restrict__ inv_n,
                  uint16_t *__restrict__ dz2_out, float *__restrict__ grad, double *__restrict__ loss,
                  uint32_t *__restrict__ status) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t *sA2 = smem + kB1A2, *sA3 = smem + kB1A3, *sDz3 = smem + kB1Dz3, *sDz4 = smem + kB1Dz4;
  uint8_t *sW3T = smem + kB1W3T;
  float *sw4 = reinterpret_cast<float *>(smem + kB1Par);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kB1Bar);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + kB1Bar + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint16_t *gw3 = reinterpret_cast<const uint16_t *>(weights + kOffW3);
  // everything starts at zero (the M = 128 reads past the real rows see finite
  // values); the ones chunks; W3^T in the K-major core-matrix layout
  for (int e = tid; e < kB1Smem / 16; e += kNetThreads) reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int e = tid; e < 32 * 32; e += kNetThreads) {
    const int o = e / 32, i = e % 32;
    *reinterpret_cast<uint16_t *>(sW3T + core_off(i, o, 32)) = gw3[e];
  }
  *reinterpret_cast<uint4 *>(sA2 + 4 * kChunkPx + tid * 16) = make_uint4(0x3F80u, 0u, 0u, 0u);
  *reinterpret_cast<uint4 *>(sA3 + 4 * kChunkPx + tid * 16) = make_uint4(0x3F80u, 0u, 0u, 0u);
  if (tid < kCh) sw4[tid] = __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(weights + kOffW4)[tid]);
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)), "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = *s_tmem;   // D: da2 cols 0-31, dW3^T cols 32-63, dw4 cols 64-79
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
  uint32_t phase = 0;
  bool ok = true, first = true;
  float lsum = 0.f;
  const float invn = inv_n[0];
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const long long ntiles = (long long)batch * H * tiles_x;
  for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int tx = (int)(t % tiles_x), yy = (int)((t / tiles_x) % H), b = (int)(t / ((long long)tiles_x * H));
    const int p = tid, x = tx * kTileW + p;
    const bool in = x < W;
    const size_t pix = ((size_t)b * H + yy) * W + x;
    float dz4 = 0.f;
    uint32_t a2w[16], a3w[16];
    if (in) {
      const float tg = target[pix], yv = y[pix];
      if (tg >= 0.f) {
        dz4 = (yv - tg) * invn;
        const float yc = fminf(fmaxf(yv, 1e-12f), 0.99999994f);   // largest float below 1
        lsum -= (tg * logf(yc) + (1.f - tg) * logf(1.f - yc)) * invn;
      }
      const uint4 *ga = reinterpret_cast<const uint4 *>(acts + pix * 96);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const uint4 u2 = ga[4 + g], u3 = ga[8 + g];
        a2w[4 * g] = u2.x; a2w[4 * g + 1] = u2.y; a2w[4 * g + 2] = u2.z; a2w[4 * g + 3] = u2.w;
        a3w[4 * g] = u3.x; a3w[4 * g + 1] = u3.y; a3w[4 * g + 2] = u3.z; a3w[4 * g + 3] = u3.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) { a2w[k] = 0u; a3w[k] = 0u; }
    }
    // dz3 = dz4 w4 [a3 > 0]
    uint32_t dzw[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float a3lo = __uint_as_float(a3w[k] << 16), a3hi = __uint_as_float(a3w[k] & 0xFFFF0000u);
      dzw[k] = pack_bf16x2(a3lo > 0.f ? dz4 * sw4[2 * k] : 0.f, a3hi > 0.f ? dz4 * sw4[2 * k + 1] : 0.f);
    }
    st_chunks(sA2, kChunkPx, p, a2w);
    st_chunks(sA3, kChunkPx, p, a3w);
    st_chunks(sDz3, kChunkPx, p, dzw);
    *reinterpret_cast<uint4 *>(sDz4 + p * 16) = make_uint4(__bfloat16_as_ushort(__float2bfloat16_rn(dz4)), 0u, 0u, 0u);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
      // da2 = dz3 W3 (M = pixels, K = o)
      for (int c = 0; c < 2; ++c)
        mma_bf16(tmem + 0, sdesc(smem_u32(sDz3) + 2 * c * kChunkPx, kChunkPx, 128),
                 sdesc(smem_u32(sW3T) + c * 256, 128, 512), idesc_bf16(128, 32), c > 0 ? 1u : 0u);
      // dW3^T (M = i, N = o) and dw4 (M = i, N = 16) over the tile's pixels
      for (int s = 0; s < kTileW / 16; ++s) {
        const uint32_t acc = (!first || s > 0) ? 1u : 0u;
        mma_bf16(tmem + 32, sdesc(smem_u32(sA2) + s * 256, 128, kChunkPx),
                 sdesc(smem_u32(sDz3) + s * 256, 128, kChunkPx), idesc_bf16_mn(64, 32), acc);
        mma_bf16(tmem + 64, sdesc(smem_u32(sA3) + s * 256, 128, kChunkPx),
                 sdesc(smem_u32(sDz4) + s * 256, 128, kChunkPx), idesc_bf16_mn(64, 16), acc);
      }
      mma_commit(bar);
    }
    ok = bar_wait(bar, phase);
    phase ^= 1u;
    tc_after_sync();
    first = false;
    // dz2 = (dz3 W3) [a2 > 0] -> global (bf16) for the second backward kernel
    {
      float da[32];
      tmem_ld32(tmem + lane_base + 0, da);
      if (in) {
        uint32_t w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float a2lo = __uint_as_float(a2w[k] << 16), a2hi = __uint_as_float(a2w[k] & 0xFFFF0000u);
          w[k] = pack_bf16x2(a2lo > 0.f ? da[2 * k] : 0.f, a2hi > 0.f ? da[2 * k + 1] : 0.f);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(dz2_out + pix * 32);
#pragma unroll
        for (int g = 0; g < 4; ++g) dst[g] = make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
      }
    }
    tc_before_sync();
    ok = __syncthreads_and(ok) != 0;   // uniform loop exit
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, kStatusTimeout);
    bar_wait(bar, phase ^ 1u);
  }
  // the CTA's accumulated weight gradients: row r of D = input channel (or the
  // ones row), column = output channel; an M = 64 accumulator's row r is in
  // TMEM lane 32 (r / 16) + r % 16
  if (!first) {
    tc_after_sync();
    float d[32];
    tmem_ld32(tmem + lane_base + 32, d);
    const int r = m64_row(tid);
    if (r >= 0 && r < 32) {
      for (int o = 0; o < 32; ++o) atomicAdd(grad + kGW3 + o * 32 + r, d[o]);
    } else if (r == 32) {
      for (int o = 0; o < 32; ++o) atomicAdd(grad + kGb3 + o, d[o]);
    }
    tmem_ld32(tmem + lane_base + 64, d);
    if (r >= 0 && r < 32) atomicAdd(grad + kGw4 + r, d[0]);
    else if (r == 32) atomicAdd(grad + kGb4, d[0]);
  }
  lsum = warp_sum(lsum);
  if (lane == 0 && lsum != 0.f) atomicAdd(loss, (double)lsum);
  tc_before_sync();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

// bwd2 shared memory: two sets (double buffering) of the dz2 and a1 halos
// (3 rows x 130 pixels; a1 with its ones chunk 4) and of x (chunk 0, ones
// chunk 1), then dz1 and W2 rearranged as B[i][(tap, o)]. The M = 128
// MN-major reads of a1 and x run past their real chunks into what follows
// (in bounds, finite).
constexpr int kHaloChunk = 392 * 16;                     // 6272
constexpr int kB2SetA1 = 0, kB2SetDz2 = 5 * kHaloChunk, kB2SetBytes = 9 * kHaloChunk;   // 56448
constexpr int kB2X = 2 * kB2SetBytes;                    // 2 x (x chunk, ones chunk)
constexpr int kB2Dz1 = kB2X + 4 * kChunkPx;              // dz1: 4 chunks
constexpr int kB2W2t = kB2Dz1 + 4 * kChunkPx;            // [32 i][288 (tap, o)]
constexpr int kB2Bar = kB2W2t + 32 * kK2 * 2;
constexpr int kB2End = kB2Bar + 64;
constexpr int kB2Span = kB2SetBytes + 16 * kHaloChunk;   // the farthest MN-major read of a1 (set 1)
constexpr int kB2Smem = (kB2Span > kB2End ? kB2Span : kB2End);
static_assert(kB2X + 2 * kChunkPx + 16 * kChunkPx <= kB2Smem, "MN-major reads of x stay in shared memory");

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

__global__ void __launch_bounds__(kNetThreads, 1)
mpnet_bwd2_kernel(const uint8_t *__restrict__ weights, const uint4 *__restrict__ feats, const uint16_t *__restrict__ acts,
                  const uint16_t *__restrict__ dz2, int batch, int W, int H, float *__restrict__ grad,
                  uint32_t *__restrict__ status) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t *sDz1 = smem + kB2Dz1, *sW2t = smem + kB2W2t;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kB2Bar);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + kB2Bar + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < kB2Smem / 16; e += kNetThreads) reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const uint16_t *gw2 = reinterpret_cast<const uint16_t *>(weights + kOffW2);
  for (int e = tid; e < 32 * kK2; e += kNetThreads) {
    const int o = e / kK2, col = e % kK2, tap = col / 32, i = col % 32;
    *reinterpret_cast<uint16_t *>(sW2t + core_off(i, tap * 32 + o, kK2)) = gw2[e];
  }
  for (int set = 0; set < 2; ++set) {
    for (int h = tid; h < 392; h += kNetThreads)
      *reinterpret_cast<uint4 *>(smem + set * kB2SetBytes + kB2SetA1 + 4 * kHaloChunk + h * 16) =
          make_uint4(0x3F80u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(smem + kB2X + set * 2 * kChunkPx + kChunkPx + tid * 16) = make_uint4(0x3F80u, 0u, 0u, 0u);
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  // D: da1 cols 0-31; dW2^T of tap t cols 32 + 32 t (t = 0..8, to 319); dW1^T cols 320-351
  const uint32_t tmem = *s_tmem;
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
  uint32_t phase = 0;
  bool ok = true, first = true;
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const long long ntiles = (long long)batch * H * tiles_x;
  // asynchronous copies of tile T's halos and x into buffer set `set`
  // (zero-filled outside the image)
  auto fetch = [&](long long T, int set) {
    const int tx = (int)(T % tiles_x), y = (int)((T / tiles_x) % H), b = (int)(T / ((long long)tiles_x * H));
    const int x0 = tx * kTileW;
    const uint32_t base = smem_u32(smem) + set * kB2SetBytes;
    for (int h = tid; h < kHaloRows; h += kNetThreads) {
      const int r = h / kHaloW, c = h % kHaloW, yy = y - 1 + r, xx = x0 - 1 + c;
      const bool v = yy >= 0 && yy < H && xx >= 0 && xx < W;
      const size_t q = v ? ((size_t)b * H + yy) * W + xx : 0;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        cp_async16(base + kB2SetDz2 + g * kHaloChunk + h * 16, dz2 + q * 32 + 8 * g, v);
        cp_async16(base + kB2SetA1 + g * kHaloChunk + h * 16, acts + q * 96 + 8 * g, v);
      }
    }
    const int x = x0 + tid;
    cp_async16(smem_u32(smem) + kB2X + set * 2 * kChunkPx + tid * 16, feats + (x < W ? ((size_t)b * H + y) * W + x : 0),
               x < W);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // Per tile: da1 (18 MMAs) is committed on its own and the dW2 MMAs (72)
  // queue behind it, so the dz1 epilogue runs while the tensor core
  // accumulates dW2; dW1 (8 MMAs) follows the epilogue. The next tile's da1
  // commit covers all of them (one thread's MMAs complete in order), so its
  // wait also frees this tile's buffers for the prefetch two tiles ahead.
  long long t = blockIdx.x;
  if (t < ntiles) fetch(t, 0);
  bool pending = false;   // MMAs issued and not yet covered by a completed wait
  for (int it = 0; t < ntiles && ok; t += gridDim.x, ++it) {
    const int set = it & 1, p = tid;
    uint8_t *sA1 = smem + set * kB2SetBytes + kB2SetA1, *sDz2 = smem + set * kB2SetBytes + kB2SetDz2;
    uint8_t *sX = smem + kB2X + set * 2 * kChunkPx;
    // 1. this tile's halos and x have landed
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    // 2. da1: the transposed 3 x 3 convolution as an implicit GEMM - tap
    //    (ky, kx) reads dz2 at halo row (2 - ky) * 130 + (2 - kx) + q; then
    //    dW2^T per tap: a1 at halo row ky * 130 + kx + q against dz2 of the
    //    centre row (halo row 131 + q), MN-major over the tile's pixels
    if (tid == 0) {
      for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        for (int j = 0; j < 2; ++j)
          mma_bf16(tmem + 0, sdesc(smem_u32(sDz2) + 2 * j * kHaloChunk + ((2 - ky) * kHaloW + (2 - kx)) * 16, kHaloChunk, 128),
                   sdesc(smem_u32(sW2t) + (2 * tap + j) * 256, 128, (kK2 / 8) * 128), idesc_bf16(128, 32),
                   (tap | j) ? 1u : 0u);
      }
      mma_commit(bar);
      for (int s2 = 0; s2 < kTileW / 16; ++s2) {
        const uint32_t acc = (!first || s2 > 0) ? 1u : 0u;
        const uint32_t bdz2 = smem_u32(sDz2) + (kHaloW + 1) * 16 + s2 * 256;
        for (int tap = 0; tap < 9; ++tap) {
          const int ky = tap / 3, kx = tap % 3;
          mma_bf16(tmem + 32 + 32 * tap, sdesc(smem_u32(sA1) + (ky * kHaloW + kx) * 16 + s2 * 256, 128, kHaloChunk),
                   sdesc(bdz2, 128, kHaloChunk), idesc_bf16_mn(64, 32), acc);
        }
      }
    }
    pending = true;
    ok = bar_wait(bar, phase);   // da1 done, and every MMA of the previous tile
    phase ^= 1u;
    tc_after_sync();
    // 3. the previous tile's buffer set is free: prefetch the next tile
    if (t + gridDim.x < ntiles) fetch(t + gridDim.x, set ^ 1);
    // 4. dz1 = da1 [a1 > 0] (a1 of the centre row: halo row 131 + q)
    {
      float da[32];
      tmem_ld32(tmem + lane_base + 0, da);
      uint32_t a1w[16], w[16];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const uint4 u = *reinterpret_cast<const uint4 *>(sA1 + g * kHaloChunk + (kHaloW + 1 + p) * 16);
        a1w[4 * g] = u.x; a1w[4 * g + 1] = u.y; a1w[4 * g + 2] = u.z; a1w[4 * g + 3] = u.w;
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float lo = __uint_as_float(a1w[k] << 16), hi = __uint_as_float(a1w[k] & 0xFFFF0000u);
        w[k] = pack_bf16x2(lo > 0.f ? da[2 * k] : 0.f, hi > 0.f ? da[2 * k + 1] : 0.f);
      }
      st_chunks(sDz1, kChunkPx, p, w);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    // 5. dW1^T: x against dz1
    if (tid == 0) {
      for (int s2 = 0; s2 < kTileW / 16; ++s2)
        mma_bf16(tmem + 320, sdesc(smem_u32(sX) + s2 * 256, 128, kChunkPx),
                 sdesc(smem_u32(sDz1) + s2 * 256, 128, kChunkPx), idesc_bf16_mn(64, 32),
                 (!first || s2 > 0) ? 1u : 0u);
    }
    first = false;
    tc_before_sync();
    ok = __syncthreads_and(ok) != 0;   // uniform loop exit
  }
  // the last tile's dW MMAs (after a wait that gave up: everything still in
  // flight) under one more commit and one more bounded wait
  if (pending) {
    if (tid == 0) mma_commit(bar);
    const bool done = bar_wait(bar, phase);
    phase ^= 1u;
    ok = __syncthreads_and(ok && done) != 0;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy outlives the CTA
  if (!ok && tid == 0) atomicOr(status, kStatusTimeout);
  if (!first) {
    tc_after_sync();
    float d[32];
    const int r = m64_row(tid);
    for (int tap = 0; tap < 9; ++tap) {
      tmem_ld32(tmem + lane_base + 32 + 32 * tap, d);
      if (r >= 0 && r < 32) {
        for (int o = 0; o < 32; ++o) atomicAdd(grad + kGW2 + o * 288 + tap * 32 + r, d[o]);
      } else if (r == 32 && tap == 0) {
        for (int o = 0; o < 32; ++o) atomicAdd(grad + kGb2 + o, d[o]);
      }
    }
    tmem_ld32(tmem + lane_base + 320, d);
    if (r >= 0 && r < 8) {
      for (int o = 0; o < 32; ++o) atomicAdd(grad + kGW1 + o * 16 + r, d[o]);
    } else if (r == 8) {
      for (int o = 0; o < 32; ++o) atomicAdd(grad + kGb1 + o, d[o]);
    }
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// Adam on the FP32 master parameters (gradient layout), refreshing the BF16
// weights and FP32 biases of the blob.
__global__ void mpnet_adam_kernel(uint8_t *__restrict__ weights, float *__restrict__ master, float *__restrict__ m,
                                  float *__restrict__ v, const float *__restrict__ grad, float lr, float beta1,
                                  float beta2, float eps, float bc1, float bc2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kGTotal) return;
  const float g = grad[k];
  const float mk = beta1 * m[k] + (1.f - beta1) * g;
  const float vk = beta2 * v[k] + (1.f - beta2) * g * g;
  m[k] = mk;
  v[k] = vk;
  float w = master[k] - lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
  if (k < kGW2 && (k % 16) >= 8) w = 0.f;   // padded input channels of W1 stay zero
  master[k] = w;
  __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(weights);
  if (k < kGw4 + 32) {
    // W1, W2, W3, w4 are contiguous in both layouts (1024 + 18432 + 2048 + 64 bytes)
    wb[k] = __float2bfloat16_rn(w);
  } else {
    reinterpret_cast<float *>(weights + kOffB1)[k - kGb1] = w;   // b1 b2 b3 b4 contiguous too
  }
}
}  // namespace

cudaError_t launch_selftest_wait(uint32_t *status, long long limit, cudaStream_t s) {
  selftest_wait_kernel<<<1, 1, 0, s>>>(status, limit);
  return cudaGetLastError();
}

cudaError_t launch_mpnet_forward(const void *weights, const uint16_t *feats, int batch, int W, int H, float *out,
                                 uint16_t *acts, uint32_t *status, int num_sms, cudaStream_t s) {
  if (batch <= 0 || W <= 0 || H <= 0) return cudaSuccess;
  // units: strips x row segments; the segment length balances the units over
  // the warpgroups (a unit of S output rows takes S + 4 pipeline steps)
  FwdUnits un;
  un.tiles_x = (W + kTileW - 1) / kTileW;
  const long long strips = (long long)batch * un.tiles_x;
  const long long slots = (long long)num_sms * kGroups;
  double best = 1e300;
  un.seg_rows = H;
  for (int S = 4; S <= 96; ++S) {
    const long long segs = (H + S - 1) / S;
    const long long rounds = (strips * segs + slots - 1) / slots;
    const double cost = (double)rounds * (S + 4);   // pipeline fill and drain: 4 steps
    if (cost < best - 1e-9) { best = cost; un.seg_rows = S; }
    if (S >= H) break;
  }
  un.segs = (H + un.seg_rows - 1) / un.seg_rows;
  un.count = strips * un.segs;
  const long long ctas = (un.count + kGroups - 1) / kGroups;
  const int grid = (int)(ctas < num_sms ? ctas : num_sms);
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return cudaErrorNotSupported;
  // the input as a 4-D tensor (channel, x, y, image); box = one 130-pixel
  // halo row; out-of-range elements (image borders) read as zero
  CUtensorMap map;
  const cuuint64_t dims[4] = {8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)batch};
  const cuuint64_t strides[3] = {16, (cuuint64_t)W * 16, (cuuint64_t)W * H * 16};
  const cuuint32_t box[4] = {8, (cuuint32_t)kHaloW, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(feats), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(mpnet_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
  if (e != cudaSuccess) return e;
  mpnet_fwd_kernel<<<grid, kFwdThreads, kFwdSmem, s>>>(map, static_cast<const uint8_t *>(weights), batch, W, H, un,
                                                       out, acts, status);
  return cudaGetLastError();
}

}  // namespace dags

namespace dags {

cudaError_t launch_mpnet_train(void *weights, float *master, float *adam_m, float *adam_v, int step,
                               const uint16_t *feats, const float *target, int batch, int W, int H, float lr,
                               double *loss, const MpnetScratch &sc, uint32_t *status, int num_sms, cudaStream_t s) {
  const long long npix = (long long)batch * H * W;
  cudaError_t e = cudaMemsetAsync(sc.grad, 0, kGTotal * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.inv_n, 0, 2 * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  mpnet_count_kernel<<<num_sms, 256, 0, s>>>(target, npix, sc.inv_n, nullptr);
  mpnet_count_finish_kernel<<<1, 1, 0, s>>>(sc.inv_n);
  e = launch_mpnet_forward(weights, feats, batch, W, H, sc.y, sc.acts, status, num_sms, s);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)batch * H * ((W + kTileW - 1) / kTileW);
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  // bwd1 holds 128 TMEM columns and 43 KB of shared memory: four CTAs per SM
  // give four independent tile streams
  const int grid1 = (int)(ntiles < 4ll * num_sms ? ntiles : 4ll * num_sms);
  e = cudaFuncSetAttribute(mpnet_bwd1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kB1Smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(mpnet_bwd2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kB2Smem);
  if (e != cudaSuccess) return e;
  mpnet_bwd1_kernel<<<grid1, kNetThreads, kB1Smem, s>>>(static_cast<const uint8_t *>(weights), sc.y, target, sc.acts,
                                                       batch, W, H, sc.inv_n, sc.dz2, sc.grad, loss, status);
  mpnet_bwd2_kernel<<<grid, kNetThreads, kB2Smem, s>>>(static_cast<const uint8_t *>(weights),
                                                       reinterpret_cast<const uint4 *>(feats), sc.acts, sc.dz2, batch,
                                                       W, H, sc.grad, status);
  const float beta1 = 0.9f, beta2 = 0.999f;
  const float bc1 = 1.f - powf(beta1, (float)step), bc2 = 1.f - powf(beta2, (float)step);
  mpnet_adam_kernel<<<(kGTotal + 255) / 256, 256, 0, s>>>(static_cast<uint8_t *>(weights), master, adam_m, adam_v,
                                                          sc.grad, lr, beta1, beta2, 1e-8f, bc1, bc2);
  return cudaGetLastError();
}

}  // namespace dags
