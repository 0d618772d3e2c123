// Epipolar verification and static recovery (Sec. IV-C, Eqs. (18), (19)) on
// sm_103a:
//
//   epi_F_kernel        F = K^-T [t]x R K^-1 from the two poses, FP64, one
//                       thread
//   epi_dist_kernel     per match: the point-to-epipolar-line distance d of
//                       Eq. (18) in FP64, and the match's
//                       rank inside its Gaussian's group (one atomic per
//                       match on the Gaussian's count)
//   scan (3 kernels)    exclusive scan of the per-Gaussian counts into group
//                       offsets: 1024 counts per CTA, the CTA sums by one CTA,
//                       then the offsets added back
//   epi_scatter_kernel  d into its group's slot (offset + rank)
//   epi_median_kernel   per Gaussian with matches: the lower median of its
//                       group by rank counting (the groups hold a few values;
//                       the result does not depend on the order the atomics
//                       gave), the consistency test dbar < eps of Eq. (19),
//                       and the recovery of a dynamic-labelled consistent
//                       Gaussian: label 0, M <- min(M, m_static)
//
// Gaussian ids come from the caller: an id >= n is skipped and recorded as
// an index error in the status word (DAGS_E_BOUNDS at the next sync).
#include "common.cuh"

namespace dags {

namespace {

constexpr int kEpiBlock = 256;
constexpr int kScanItems = 4;                  // counts per thread in the block scan
constexpr int kScanTile = kEpiBlock * kScanItems;

// F = K^-T [t]x R K^-1 of the relative pose (R, t) = T_2W T_1W^-1, in FP64
// by one thread (FP64 instructions are scarce on GB300: the per-match kernel
// only reads it).
__global__ void epi_F_kernel(Raster r, const double *__restrict__ pose_1, const double *__restrict__ pose_2,
                             double *__restrict__ F) {
  pdl_wait();
  if (threadIdx.x != 0) return;
  {
    // R = R2 R1^T, t = t2 - R t1, E = [t]x R, F = K^-T E K^-1
    double R[9], t[3], E[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        R[3 * a + b] = pose_2[4 * a] * pose_1[4 * b] + pose_2[4 * a + 1] * pose_1[4 * b + 1] +
                       pose_2[4 * a + 2] * pose_1[4 * b + 2];
    for (int a = 0; a < 3; ++a)
      t[a] = pose_2[4 * a + 3] - (R[3 * a] * pose_1[3] + R[3 * a + 1] * pose_1[7] + R[3 * a + 2] * pose_1[11]);
    const double tx[9] = {0.0, -t[2], t[1], t[2], 0.0, -t[0], -t[1], t[0], 0.0};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) E[3 * a + b] = tx[3 * a] * R[b] + tx[3 * a + 1] * R[3 + b] + tx[3 * a + 2] * R[6 + b];
    // K^-1 = [[1/fx, 0, -cx/fx], [0, 1/fy, -cy/fy], [0, 0, 1]]
    const double ifx = 1.0 / (double)r.fx, ify = 1.0 / (double)r.fy;
    const double kx = -(double)r.cx * ifx, ky = -(double)r.cy * ify;
    double EK[9];   // E K^-1
    for (int a = 0; a < 3; ++a) {
      EK[3 * a + 0] = E[3 * a] * ifx;
      EK[3 * a + 1] = E[3 * a + 1] * ify;
      EK[3 * a + 2] = E[3 * a] * kx + E[3 * a + 1] * ky + E[3 * a + 2];
    }
    // K^-T (E K^-1): rows 0, 1 scale, row 2 combines
    for (int b = 0; b < 3; ++b) {
      F[b] = EK[b] * ifx;
      F[3 + b] = EK[3 + b] * ify;
      F[6 + b] = EK[b] * kx + EK[3 + b] * ky + EK[6 + b];
    }
  }
}

__global__ void __launch_bounds__(kEpiBlock)
epi_dist_kernel(const double *__restrict__ F, const float2 *__restrict__ p1, const float2 *__restrict__ p2,
                const int32_t *__restrict__ gid, int64_t m, int64_t n, float *__restrict__ dist,
                uint32_t *__restrict__ count, uint32_t *__restrict__ rank, uint32_t *status) {
  pdl_wait();
  __shared__ double s_F[9];
  if (threadIdx.x < 9) s_F[threadIdx.x] = F[threadIdx.x];
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * kEpiBlock + threadIdx.x;
  if (k >= m) return;
  const float2 a1 = p1[k], a2 = p2[k];
  const double u1 = a1.x, v1 = a1.y, u2 = a2.x, v2 = a2.y;
  const double la = s_F[0] * u1 + s_F[1] * v1 + s_F[2];
  const double lb = s_F[3] * u1 + s_F[4] * v1 + s_F[5];
  const double lc = s_F[6] * u1 + s_F[7] * v1 + s_F[8];
  const double num = fabs(u2 * la + v2 * lb + lc);
  const double den = sqrt(la * la + lb * lb);
  dist[k] = den > 0.0 ? (float)(num / den) : 0.f;
  const int32_t g = gid[k];
  if (g < 0 || (int64_t)g >= n) {
    atomicOr(status, kStatusBounds);
    rank[k] = 0xFFFFFFFFu;
    return;
  }
  rank[k] = atomicAdd(count + g, 1u);
}

// Exclusive scan of count[0, n) into off[0, n): per CTA 1024 counts (four
// per thread, then a shared-memory scan of the thread sums); block sums out.
__global__ void __launch_bounds__(kEpiBlock)
scan_tiles_kernel(const uint32_t *__restrict__ count, int64_t n, uint32_t *__restrict__ off,
                  uint32_t *__restrict__ block_sum) {
  pdl_wait();
  __shared__ uint32_t s[kEpiBlock];
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
  uint32_t v[kScanItems], acc = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < n ? count[base + j] : 0u;
    acc += v[j];
  }
  s[tid] = acc;
  __syncthreads();
  for (int o = 1; o < kEpiBlock; o <<= 1) {
    const uint32_t add = tid >= o ? s[tid - o] : 0u;
    __syncthreads();
    s[tid] += add;
    __syncthreads();
  }
  uint32_t run = s[tid] - acc;   // exclusive prefix of this thread's items
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) off[base + j] = run;
    run += v[j];
  }
  if (tid == kEpiBlock - 1) block_sum[blockIdx.x] = s[tid];
}

// One CTA: exclusive scan of the block sums in place, sequential chunks.
__global__ void __launch_bounds__(kEpiBlock)
scan_sums_kernel(uint32_t *__restrict__ block_sum, int nb) {
  pdl_wait();
  __shared__ uint32_t s[kEpiBlock];
  __shared__ uint32_t carry;
  const int tid = threadIdx.x;
  if (tid == 0) carry = 0u;
  __syncthreads();
  for (int c0 = 0; c0 < nb; c0 += kEpiBlock) {
    const uint32_t v = c0 + tid < nb ? block_sum[c0 + tid] : 0u;
    s[tid] = v;
    __syncthreads();
    for (int o = 1; o < kEpiBlock; o <<= 1) {
      const uint32_t add = tid >= o ? s[tid - o] : 0u;
      __syncthreads();
      s[tid] += add;
      __syncthreads();
    }
    if (c0 + tid < nb) block_sum[c0 + tid] = carry + s[tid] - v;
    __syncthreads();
    if (tid == kEpiBlock - 1) carry += s[tid];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kEpiBlock)
scan_add_kernel(uint32_t *__restrict__ off, int64_t n, const uint32_t *__restrict__ block_sum) {
  pdl_wait();
  const int64_t i = (int64_t)blockIdx.x * kEpiBlock + threadIdx.x;
  if (i < n) off[i] += block_sum[i / kScanTile];
}

__global__ void __launch_bounds__(kEpiBlock)
epi_scatter_kernel(const int32_t *__restrict__ gid, const uint32_t *__restrict__ rank, const float *__restrict__ dist,
                   int64_t m, const uint32_t *__restrict__ off, float *__restrict__ vals) {
  pdl_wait();
  const int64_t k = (int64_t)blockIdx.x * kEpiBlock + threadIdx.x;
  if (k >= m) return;
  const uint32_t rk = rank[k];
  if (rk == 0xFFFFFFFFu) return;
  vals[off[gid[k]] + rk] = dist[k];
}

__global__ void __launch_bounds__(kEpiBlock)
epi_median_kernel(const uint32_t *__restrict__ count, const uint32_t *__restrict__ off,
                  const float *__restrict__ vals, int64_t n, float eps, float m_static, float4 *__restrict__ gauss,
                  uint8_t *__restrict__ labels, float *__restrict__ dbar) {
  pdl_wait();
  const int64_t g = (int64_t)blockIdx.x * kEpiBlock + threadIdx.x;
  if (g >= n) return;
  const uint32_t c = count[g];
  if (c == 0) {
    if (dbar) dbar[g] = __int_as_float(0x7fc00000);
    return;
  }
  const float *v = vals + off[g];
  const uint32_t want = (c - 1) / 2;
  float med = v[0];
  for (uint32_t i = 0; i < c; ++i) {
    // rank of v[i] in the ascending order (ties broken by position)
    const float x = v[i];
    uint32_t rk = 0;
    for (uint32_t j = 0; j < c; ++j) {
      const float y = v[j];
      rk += (y < x || (y == x && j < i)) ? 1u : 0u;
    }
    if (rk == want) { med = x; break; }
  }
  if (dbar) dbar[g] = med;
  if (med < eps && labels[g] == 1) {
    labels[g] = 0;
    float4 w = gauss[4 * g + 2];
    w.w = fminf(w.w, m_static);
    gauss[4 * g + 2] = w;
  }
}

}  // namespace

int64_t epi_scan_blocks(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

cudaError_t launch_epipolar(const Raster &r, const double *pose_1, const double *pose_2, const float2 *p1,
                            const float2 *p2, const int32_t *gid, int64_t m, float4 *gauss, int64_t n,
                            uint8_t *labels, float eps, float m_static, float *dist, float *dbar, const EpiBuffers &b,
                            uint32_t *status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b.count, 0, (size_t)(n > 0 ? n : 1) * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const unsigned gm = (unsigned)((m + kEpiBlock - 1) / kEpiBlock);
  const unsigned gn = (unsigned)((n + kEpiBlock - 1) / kEpiBlock);
  const int nb = (int)epi_scan_blocks(n);
  // programmatic launches after the first: each kernel waits for its
  // predecessor's memory before its first access, and its launch overlaps
  // the predecessor's last wave
  if (m > 0) {
    epi_F_kernel<<<1, 32, 0, s>>>(r, pose_1, pose_2, b.F);
    e = launch_pdl(epi_dist_kernel, dim3(gm), dim3(kEpiBlock), 0, s, (const double *)b.F, p1, p2, gid, m, n, dist,
                   b.count, b.rank, status);
  }
  if (n > 0 && e == cudaSuccess) {
    e = launch_pdl(scan_tiles_kernel, dim3((unsigned)nb), dim3(kEpiBlock), 0, s, (const uint32_t *)b.count, n, b.off,
                   b.block_sum);
    if (e == cudaSuccess) e = launch_pdl(scan_sums_kernel, dim3(1), dim3(kEpiBlock), 0, s, b.block_sum, nb);
    if (e == cudaSuccess)
      e = launch_pdl(scan_add_kernel, dim3(gn), dim3(kEpiBlock), 0, s, b.off, n, (const uint32_t *)b.block_sum);
  }
  if (m > 0 && e == cudaSuccess)
    e = launch_pdl(epi_scatter_kernel, dim3(gm), dim3(kEpiBlock), 0, s, gid, (const uint32_t *)b.rank,
                   (const float *)dist, m, (const uint32_t *)b.off, b.vals);
  if (n > 0 && e == cudaSuccess)
    e = launch_pdl(epi_median_kernel, dim3(gn), dim3(kEpiBlock), 0, s, (const uint32_t *)b.count,
                   (const uint32_t *)b.off, (const float *)b.vals, n, eps, m_static, gauss, labels, dbar);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace dags
