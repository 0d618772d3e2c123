// Spatiotemporal motion-probability update (Sec. IV-A, Eq. (17)) on sm_103a.
//
//   mp_pixel_sum_kernel   per pixel: residual e(p) between the observed and
//                         the rendered RGB-D, stored; per-region count and sum
//                         (shared-memory partials, one FP64 atomic per region
//                         per CTA)
//   mp_pixel_var_kernel   per pixel: centred squares (e - mean_k)^2 summed per
//                         region the same way (two passes: no cancellation)
//   mp_pixel_map_kernel   per pixel: the fused MP M_p, Eqs. (2)-(7), from
//                         the region statistics; Gamma_geo of a pixel that no
//                         instance claims uses the dispersion of e over the
//                         pixel's own disk of radius r_s (its associated
//                         neighbourhood); stored for the gather
//   mp_pyramid_kernel     per pixel of pyramid level s >= 1 (only when the
//                         association uses S > 1 levels): the 2x2 box mean
//                         of level s - 1 for M_p and e, the 2x2 max for the
//                         rendered depth
//   mp_gauss_kernel       per Gaussian: projection, the association N(G),
//                         Eq. (1), the union over the levels of the disks of
//                         radius r_s around pi(G) / 2^s, over the stored M_p
//                         (or the caller's map); M_hat, Eq. (8), with weights
//                         2^-s exp(-d^2 / (2 sigma_w^2)); Var{M_p}; sigma_e,G;
//                         U, Eq. (10); CTA min/max of U -> global
//   mp_apply_kernel       per observed Gaussian: normalised U, C, alpha,
//                         Eqs. (11), (17); M^t, Eq. (9), written into the
//                         record; first radix-select level of the two medians
//   mp_select_kernel      further radix-select levels (exact lower medians of
//                         M^t and U_tilde over the observed Gaussians, bits
//                         31-21, 20-10, 9-0 of the non-negative floats);
//                         the last CTA of the last level writes tau, U_bar
//   mp_labels_kernel      labels, Eq. (12)
// The last CTA of each histogram kernel finds the bin holding the median's
// rank (one warp scans the bins).
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"

namespace dags {

namespace {

constexpr int kMpBlock = 256;
constexpr int kSelBins = 2048;

struct MpCfg {
  float kappa_c, lam, sigma_min, e_floor, sigma_g, sigma_c, lam_u, eps, alpha_min, alpha_max, rho, r_s, sigma_w,
      vis_tol, z_near, tau_floor;
  int fusion_mode, seg_refreshed, n_regions, scales;
};

constexpr int kMaxScales = DAGS_MP_MAX_SCALES;

// Workspace of the update (carved from the ctx's MP buffers).
struct MpWs {
  float *e;              // [P] residual per pixel
  double *acc;           // [256][4] region count, sum, centred sum of squares, -
  float *mhat, *sige, *U, *Mt, *Ut;  // [N]
  uint8_t *obs;          // [N]
  uint32_t *hist;        // [2][kSelBins]
  uint32_t *sel;         // select state: [0] n_obs, [1] Umin bits, [2] Umax bits, [3] done counter,
                         // [4..5] prefix (M, U), [6..7] remaining rank (M, U)
  double *stats;         // caller's output
  const float *mp_map;   // [P] external per-pixel MP replacing M_p, or null
  float *mp_pixel;       // [P] out: the fused M_p, or null
  float *mpf;            // [P] the fused M_p (workspace)
  uint32_t *status;      // the ctx's status word (index checks of a DAGS_CHECK build)
  // association pyramid, level s: M_p (or the external map), e and the
  // rendered depth as row-major Ws x Hs maps (level 0: the frame's own)
  const float *lm[kMaxScales], *le[kMaxScales], *ld[kMaxScales];
  int lw[kMaxScales], lh[kMaxScales];
};

// The region of pixel p (its instance label; checked against the table size
// in a DAGS_CHECK build, where an out-of-range label counts as background).
__device__ __forceinline__ int region_of(const uint8_t *inst, size_t p, int n_regions, uint32_t *status) {
  int k = inst[p];
  if (!DAGS_IN_BOUNDS(k < n_regions, status)) k = 0;
  (void)status;
  return k;
}

// Order-preserving map of floats to uint32 (for atomic min/max of values
// that may be slightly negative).
__device__ __forceinline__ uint32_t f2o(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ float residual(const float4 tg, const float *img, size_t P, size_t p, float kappa_c) {
  const float dr = img[3 * P + p];
  float e = tg.w > 0.f ? fabsf(tg.w - dr) : 0.f;
  e += kappa_c * (fabsf(tg.x - img[p]) + fabsf(tg.y - img[P + p]) + fabsf(tg.z - img[2 * P + p]));
  return e;
}

__global__ void __launch_bounds__(kMpBlock)
mp_pixel_sum_kernel(MpWs m, const float4 *__restrict__ targets, const float *__restrict__ image,
                    const uint8_t *__restrict__ inst, int P, MpCfg c) {
  pdl_wait();
  __shared__ float s_cnt[DAGS_MP_MAX_REGIONS], s_sum[DAGS_MP_MAX_REGIONS];
  for (int k = threadIdx.x; k < c.n_regions; k += blockDim.x) { s_cnt[k] = 0.f; s_sum[k] = 0.f; }
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  // select state and histograms start cleared (used from mp_gauss_kernel on)
  for (int k = p; k < 2 * kSelBins; k += gridDim.x * blockDim.x) m.hist[k] = 0u;
  if (p == 0) {
    m.sel[0] = 0u;            // observed count
    m.sel[1] = 0xFFFFFFFFu;   // min of U (ordered key)
    m.sel[2] = 0u;            // max of U (ordered key)
    m.sel[3] = 0u;            // CTA counter
  }
  __syncthreads();
  float e = 0.f;
  int k = -1;
  if (p < P) {
    e = residual(targets[p], image, (size_t)P, (size_t)p, c.kappa_c);
    m.e[p] = e;
    k = region_of(inst, p, c.n_regions, m.status);
  }
  // most pixels of a warp share a region: sum per region over the warp
  // first, then one shared atomic per region per warp
  unsigned pending = __ballot_sync(0xffffffffu, k >= 0);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const int key = __shfl_sync(0xffffffffu, k, leader);
    const bool mine = k == key;
    const unsigned grp = __ballot_sync(0xffffffffu, mine);
    const float sum = warp_sum(mine ? e : 0.f);
    if ((int)(threadIdx.x & 31) == leader) {
      atomicAdd(&s_cnt[key], (float)__popc(grp));
      atomicAdd(&s_sum[key], sum);
    }
    pending &= ~grp;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < c.n_regions; k += blockDim.x)
    if (s_cnt[k] > 0.f) {
      atomicAdd(&m.acc[4 * k + 0], (double)s_cnt[k]);
      atomicAdd(&m.acc[4 * k + 1], (double)s_sum[k]);
    }
}

__global__ void __launch_bounds__(kMpBlock)
mp_pixel_var_kernel(MpWs m, const uint8_t *__restrict__ inst, int P, MpCfg c) {
  pdl_wait();
  __shared__ float s_mean[DAGS_MP_MAX_REGIONS], s_sq[DAGS_MP_MAX_REGIONS];
  for (int k = threadIdx.x; k < c.n_regions; k += blockDim.x) {
    const double cnt = m.acc[4 * k + 0];
    s_mean[k] = cnt > 0.0 ? (float)(m.acc[4 * k + 1] / cnt) : 0.f;
    s_sq[k] = 0.f;
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  float sq = 0.f;
  int k = -1;
  if (p < P) {
    k = region_of(inst, p, c.n_regions, m.status);
    const float d = m.e[p] - s_mean[k];
    sq = d * d;
  }
  // per-region sums over the warp first, as in the pixel-sum pass
  unsigned pending = __ballot_sync(0xffffffffu, k >= 0);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const int key = __shfl_sync(0xffffffffu, k, leader);
    const bool mine = k == key;
    const unsigned grp = __ballot_sync(0xffffffffu, mine);
    const float sum = warp_sum(mine ? sq : 0.f);
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(&s_sq[key], sum);
    pending &= ~grp;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < c.n_regions; k += blockDim.x)
    if (s_sq[k] != 0.f) atomicAdd(&m.acc[4 * k + 2], (double)s_sq[k]);
}

// Region parameters used per pixel: mean, e_ub, Gamma_geo, use-mean flag.
__device__ __forceinline__ void region_params(const MpWs &m, const MpCfg &c, int k, float4 *out) {
  const double cnt = m.acc[4 * k + 0];
  const float mean = cnt > 0.0 ? (float)(m.acc[4 * k + 1] / cnt) : 0.f;
  const float sd = cnt > 0.0 ? sqrtf((float)(m.acc[4 * k + 2] / cnt)) : 0.f;
  const float eub = fmaxf(mean + c.lam * sd, c.e_floor);
  const float ggeo = expf(-sd / c.sigma_g);
  const float use_mean = (k >= 1 && sd < c.sigma_min) ? 1.f : 0.f;
  *out = make_float4(mean, eub, ggeo, use_mean);
}

__device__ __forceinline__ float pixel_mp(float e, const float4 reg, const float2 tab, int fusion_mode) {
  const float e_used = reg.w != 0.f ? reg.x : e;
  const float mp_geo = fminf(fmaxf(e_used / reg.y, 0.f), 1.f);
  float K = reg.z / (tab.y + reg.z);
  if (fusion_mode == 1) K = 0.f;
  else if (fusion_mode == 2) K = 1.f;
  return (1.f - K) * tab.x + K * mp_geo;
}

// Population std of e over the disk {(di, dj): di^2 + dj^2 <= r_s^2} around
// pixel (x, y), clipped to the image; two passes (mean, then centred squares).
__device__ __forceinline__ float disk_std(const float *__restrict__ e, int x, int y, int W, int H, float r_s) {
  const int R = (int)floorf(r_s);
  const float rs2 = r_s * r_s;
  const int y0 = max(y - R, 0), y1 = min(y + R, H - 1), x0 = max(x - R, 0), x1 = min(x + R, W - 1);
  float s = 0.f;
  int cnt = 0;
  for (int yy = y0; yy <= y1; ++yy)
    for (int xx = x0; xx <= x1; ++xx) {
      const int di = xx - x, dj = yy - y;
      if ((float)(di * di + dj * dj) > rs2) continue;
      s += __ldg(e + (size_t)yy * W + xx);
      ++cnt;
    }
  const float mean = s / (float)cnt;
  float sq = 0.f;
  for (int yy = y0; yy <= y1; ++yy)
    for (int xx = x0; xx <= x1; ++xx) {
      const int di = xx - x, dj = yy - y;
      if ((float)(di * di + dj * dj) > rs2) continue;
      const float d = __ldg(e + (size_t)yy * W + xx) - mean;
      sq += d * d;
    }
  return sqrtf(sq / (float)cnt);
}

// The same for a disk of at most 5 x 5 pixels (floor(r_s) = 2, the default
// radius): the box unrolled, one pass over the values less the centre's
// (sums of d and d^2, whose mean square less the squared mean is the
// population variance; the shift keeps both sums small).
__device__ __forceinline__ float disk_std_r2(const float *__restrict__ e, int x, int y, int W, int H, float rs2) {
  const float c = __ldg(e + (size_t)y * W + x);
  float s = 0.f, s2 = 0.f, cnt = 0.f;
#pragma unroll
  for (int dj = -2; dj <= 2; ++dj) {
    const int yy = y + dj;
    const bool row = yy >= 0 && yy < H;
#pragma unroll
    for (int di = -2; di <= 2; ++di) {
      const int xx = x + di;
      if (row && xx >= 0 && xx < W && (float)(di * di + dj * dj) <= rs2) {
        const float d = __ldg(e + (size_t)yy * W + xx) - c;
        s += d;
        s2 = fmaf(d, d, s2);
        cnt += 1.f;
      }
    }
  }
  const float m = s / cnt;
  return sqrtf(fmaxf(s2 / cnt - m * m, 0.f));
}

// The fused per-pixel M_p map, Eqs. (2)-(7): read by the gather and, when
// asked for, returned to the caller (who may train or evaluate a learned
// proposal against the method). Gamma_geo = exp(-sigma / sigma_g) takes the
// region's sigma_e inside an instance and, for a pixel that no instance
// claims, the dispersion over the pixel's associated neighbourhood (the
// sentence after Eq. (7)), read as its disk of radius r_s.
__global__ void __launch_bounds__(kMpBlock)
mp_pixel_map_kernel(MpWs m, const uint8_t *__restrict__ inst, const float2 *__restrict__ table, int W, int H,
                    MpCfg c) {
  pdl_wait();
  __shared__ float4 s_reg[DAGS_MP_MAX_REGIONS];
  __shared__ float2 s_tab[DAGS_MP_MAX_REGIONS];
  for (int k = threadIdx.x; k < c.n_regions; k += blockDim.x) {
    region_params(m, c, k, &s_reg[k]);
    s_tab[k] = table[k];
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < W * H) {
    const int k = region_of(inst, p, c.n_regions, m.status);
    float4 reg = s_reg[k];
    if (k == 0) {
      const float sd = floorf(c.r_s) == 2.f ? disk_std_r2(m.e, p % W, p / W, W, H, c.r_s * c.r_s)
                                            : disk_std(m.e, p % W, p / W, W, H, c.r_s);
      reg.z = expf(-sd / c.sigma_g);
    }
    const float mp = pixel_mp(m.e[p], reg, s_tab[k], c.fusion_mode);
    m.mpf[p] = mp;
    if (m.mp_pixel) m.mp_pixel[p] = mp;
  }
}

// Level s of the association pyramid from level s - 1: each pixel covers a
// 2x2 block; M_p and e take the block's mean, the rendered depth its maximum
// (the occlusion test's maximum over a level-s pixel is then the maximum over
// the full-resolution pixels it covers).
__global__ void __launch_bounds__(kMpBlock)
mp_pyramid_kernel(MpWs m, int s, float *__restrict__ om, float *__restrict__ oe, float *__restrict__ od) {
  pdl_wait();
  const int W = m.lw[s], H = m.lh[s], Wp = m.lw[s - 1];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= W * H) return;
  const int x = q % W, y = q / W;
  const size_t a = (size_t)(2 * y) * Wp + 2 * x, b = a + Wp;
  const float *__restrict__ im = m.lm[s - 1], *__restrict__ ie = m.le[s - 1], *__restrict__ id = m.ld[s - 1];
  om[q] = ((im[a] + im[a + 1]) + (im[b] + im[b + 1])) * 0.25f;
  oe[q] = ((ie[a] + ie[a + 1]) + (ie[b] + ie[b + 1])) * 0.25f;
  od[q] = fmaxf(fmaxf(id[a], id[a + 1]), fmaxf(id[b], id[b + 1]));
}

// The pixel rectangle of the disk of radius r_s around (us, vs) clipped to a
// Ws x Hs level; false when it is empty (or the centre is not finite).
__device__ __forceinline__ bool disk_rect(float us, float vs, int Ws, int Hs, float r_s, int *i0, int *i1, int *j0,
                                          int *j1) {
  if (!(us > -r_s - 1.f && us < (float)Ws + r_s && vs > -r_s - 1.f && vs < (float)Hs + r_s)) return false;
  *i0 = (int)fmaxf(ceilf(us - r_s), 0.f);
  *i1 = (int)fminf(floorf(us + r_s), (float)(Ws - 1));
  *j0 = (int)fmaxf(ceilf(vs - r_s), 0.f);
  *j1 = (int)fminf(floorf(vs + r_s), (float)(Hs - 1));
  return *i0 <= *i1 && *j0 <= *j1;
}

__global__ void __launch_bounds__(kMpBlock)
mp_gauss_kernel(MpWs m, const float4 *__restrict__ gauss, int64_t n, const double *__restrict__ pose,
                const float *__restrict__ image, Raster r, MpCfg c) {
  pdl_wait();
  __shared__ float sp[12];
  __shared__ uint32_t s_min, s_max, s_cnt;
  const float *__restrict__ mpsrc = m.mp_map ? m.mp_map : m.mpf;
  if (threadIdx.x < 12) sp[threadIdx.x] = (float)pose[threadIdx.x];
  if (threadIdx.x == 0) { s_min = 0xFFFFFFFFu; s_max = 0u; s_cnt = 0u; }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float4 g0 = __ldg(gauss + 4 * i), g2 = __ldg(gauss + 4 * i + 2);
    const float x = sp[0] * g0.x + sp[1] * g0.y + sp[2] * g0.z + sp[3];
    const float y = sp[4] * g0.x + sp[5] * g0.y + sp[6] * g0.z + sp[7];
    const float z = depth_key(g0, sp);
    bool observed = false;
    float mhat = 0.f, var = 0.f, sige = 0.f;
    const float u = r.fx * x / z + r.cx, v = r.fy * y / z + r.cy;
    if (z > c.z_near) {
      const float rs2 = c.r_s * c.r_s, inv2s2 = 1.f / (2.f * c.sigma_w * c.sigma_w);
      float sw = 0.f, swm = 0.f, sm = 0.f, se = 0.f, dmax = -INFINITY;
      int cnt = 0;
#pragma unroll
      for (int s = 0; s < kMaxScales; ++s) {
        if (s >= c.scales) break;
        const float sc = 1.f / (float)(1 << s);              // 2^-s: exact
        const float us = u * sc, vs = v * sc;
        const int Ws = m.lw[s];
        int i0, i1, j0, j1;
        if (!disk_rect(us, vs, Ws, m.lh[s], c.r_s, &i0, &i1, &j0, &j1)) continue;
        const float *__restrict__ lm = s == 0 ? mpsrc : m.lm[s];
        const float *__restrict__ le = m.le[s], *__restrict__ ld = m.ld[s];
        for (int jj = j0; jj <= j1; ++jj)
          for (int ii = i0; ii <= i1; ++ii) {
            const float dx = (float)ii - us, dy = (float)jj - vs, d2 = dx * dx + dy * dy;
            if (d2 > rs2) continue;
            const size_t p = (size_t)jj * Ws + ii;
            const float e = le[p];
            const float mp = lm[p];
            const float w = sc * expf(-d2 * inv2s2);
            sw += w; swm += w * mp; sm += mp; se += e; ++cnt;
            dmax = fmaxf(dmax, ld[p]);
          }
      }
      observed = cnt > 0 && !(c.vis_tol > 0.f && dmax > 0.f && z > dmax + c.vis_tol);
      if (observed) {
        mhat = swm / sw;
        const float mm = sm / cnt, me = se / cnt;
        float vm = 0.f, ve = 0.f;
#pragma unroll
        for (int s = 0; s < kMaxScales; ++s) {
          if (s >= c.scales) break;
          const float sc = 1.f / (float)(1 << s);
          const float us = u * sc, vs = v * sc;
          const int Ws = m.lw[s];
          int i0, i1, j0, j1;
          if (!disk_rect(us, vs, Ws, m.lh[s], c.r_s, &i0, &i1, &j0, &j1)) continue;
          const float *__restrict__ lm = s == 0 ? mpsrc : m.lm[s];
          const float *__restrict__ le = m.le[s];
          for (int jj = j0; jj <= j1; ++jj)
            for (int ii = i0; ii <= i1; ++ii) {
              const float dx = (float)ii - us, dy = (float)jj - vs;
              if (dx * dx + dy * dy > rs2) continue;
              const size_t p = (size_t)jj * Ws + ii;
              const float e = le[p];
              const float mp = lm[p];
              vm += (mp - mm) * (mp - mm);
              ve += (e - me) * (e - me);
            }
        }
        var = vm / cnt;
        sige = sqrtf(ve / cnt);
      }
    }
    float U = 0.f;
    if (observed) {
      const float M0 = g2.w;
      U = -M0 * logf(M0 + c.eps) - (1.f - M0) * logf(1.f - M0 + c.eps) + c.lam_u * var;
      atomicMin(&s_min, f2o(U));
      atomicMax(&s_max, f2o(U));
      atomicAdd(&s_cnt, 1u);
    }
    m.obs[i] = observed ? 1 : 0;
    m.mhat[i] = mhat;
    m.sige[i] = sige;
    m.U[i] = U;
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_cnt) {
    atomicMin(&m.sel[1], s_min);
    atomicMax(&m.sel[2], s_max);
    atomicAdd(&m.sel[0], s_cnt);
  }
}

// One warp finds, for rank r, the bin b with cum(b - 1) <= r < cum(b) of a
// kSelBins histogram; returns b and writes the rank within the bin.
__device__ __forceinline__ int find_bin(const uint32_t *hist, uint32_t r, uint32_t *r_in_bin) {
  const int lane = threadIdx.x & 31;
  constexpr int per = kSelBins / 32;
  uint32_t mine = 0;
  for (int b = 0; b < per; ++b) mine += __ldcg(hist + lane * per + b);
  uint32_t inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  const uint32_t before = inc - mine;
  const unsigned hit = __ballot_sync(0xffffffffu, before <= r && r < inc);
  const int owner = __ffs(hit) - 1;
  int bin = -1;
  uint32_t rr = 0;
  if (lane == owner) {
    uint32_t run = before;
    for (int b = 0; b < per; ++b) {
      const uint32_t hcount = __ldcg(hist + lane * per + b);
      if (r < run + hcount) { bin = lane * per + b; rr = r - run; break; }
      run += hcount;
    }
  }
  bin = __shfl_sync(0xffffffffu, bin, owner < 0 ? 0 : owner);
  rr = __shfl_sync(0xffffffffu, rr, owner < 0 ? 0 : owner);
  *r_in_bin = rr;
  return bin;
}

// Level-l radix select step over the observed Gaussians' (M^t, U_tilde):
// level 0 uses bits 31-21, level 1 bits 20-10, level 2 bits 9-0.
__device__ __forceinline__ void select_shift(int level, int *shift, uint32_t *mask) {
  *shift = level == 0 ? 21 : (level == 1 ? 10 : 0);
  *mask = level == 2 ? 0x3FFu : 0x7FFu;
}

__device__ bool last_cta(uint32_t *counter) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
    if (s_last) __threadfence();
  }
  __syncthreads();
  return s_last != 0;
}

// After a histogram level: the last CTA finds both medians' bins, advances
// their prefixes and remaining ranks, clears the histograms; after the last
// level it writes the statistics.
__device__ void select_finish(const MpWs &m, int level, const MpCfg &c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 2) {
    const uint32_t nobs = __ldcg(m.sel + 0);
    if (nobs > 0) {
      const uint32_t rank = level == 0 ? (nobs - 1) / 2 : __ldcg(m.sel + 6 + warp);
      uint32_t rin = 0;
      const int bin = find_bin(m.hist + warp * kSelBins, rank, &rin);
      int shift;
      uint32_t mask;
      select_shift(level, &shift, &mask);
      if (lane == 0) {
        const uint32_t prefix = (level == 0 ? 0u : __ldcg(m.sel + 4 + warp)) | ((uint32_t)bin << shift);
        m.sel[4 + warp] = prefix;
        m.sel[6 + warp] = rin;
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * kSelBins; k += blockDim.x) m.hist[k] = 0u;
  if (level == 2 && threadIdx.x == 0) {
    const uint32_t nobs = __ldcg(m.sel + 0);
    const float medM = nobs ? __uint_as_float(__ldcg(m.sel + 4)) : nanf("");
    const float medU = nobs ? __uint_as_float(__ldcg(m.sel + 5)) : 0.f;
    m.stats[0] = nobs ? fmax((double)medM, (double)c.tau_floor) : (double)c.tau_floor;
    m.stats[1] = medU;
    m.stats[2] = medM;
    m.stats[3] = nobs ? (double)o2f(__ldcg(m.sel + 1)) : 0.0;
    m.stats[4] = nobs ? (double)o2f(__ldcg(m.sel + 2)) : 0.0;
    m.stats[5] = (double)nobs;
  }
  if (threadIdx.x == 0) m.sel[3] = 0u;
}

__global__ void __launch_bounds__(kMpBlock)
mp_apply_kernel(MpWs m, float4 *__restrict__ gauss, int64_t n, MpCfg c) {
  pdl_wait();
  __shared__ uint32_t s_h[2 * kSelBins];
  for (int k = threadIdx.x; k < 2 * kSelBins; k += blockDim.x) s_h[k] = 0u;
  __syncthreads();
  const float umin = o2f(m.sel[1]), umax = o2f(m.sel[2]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!m.obs[i]) continue;
    const float ut = umax > umin ? (m.U[i] - umin) / (umax - umin) : 0.f;
    const float C = expf(-m.sige[i] / c.sigma_c);
    float a = c.alpha_min + (c.alpha_max - c.alpha_min) * (1.f - ut) * C;
    a = fminf(fmaxf(a, c.alpha_min), c.alpha_max);
    if (!c.seg_refreshed) a *= c.rho;
    float *rec = reinterpret_cast<float *>(gauss + 4 * i);
    const float M0 = rec[11];
    const float Mt = (1.f - a) * M0 + a * m.mhat[i];
    rec[11] = Mt;
    m.Mt[i] = Mt;
    m.Ut[i] = ut;
    atomicAdd(&s_h[__float_as_uint(Mt) >> 21], 1u);
    atomicAdd(&s_h[kSelBins + (__float_as_uint(ut) >> 21)], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * kSelBins; k += blockDim.x)
    if (s_h[k]) atomicAdd(&m.hist[k], s_h[k]);
  if (last_cta(m.sel + 3)) select_finish(m, 0, c);
}

__global__ void __launch_bounds__(kMpBlock)
mp_select_kernel(MpWs m, int64_t n, int level, MpCfg c) {
  pdl_wait();
  __shared__ uint32_t s_h[2 * kSelBins];
  for (int k = threadIdx.x; k < 2 * kSelBins; k += blockDim.x) s_h[k] = 0u;
  __syncthreads();
  int shift;
  uint32_t mask;
  select_shift(level, &shift, &mask);
  const int top = shift + (level == 2 ? 10 : 11);   // bits above this level are the prefix
  const uint32_t pm = m.sel[4], pu = m.sel[5];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!m.obs[i]) continue;
    const uint32_t bm = __float_as_uint(m.Mt[i]), bu = __float_as_uint(m.Ut[i]);
    if ((bm >> top) == (pm >> top)) atomicAdd(&s_h[(bm >> shift) & mask], 1u);
    if ((bu >> top) == (pu >> top)) atomicAdd(&s_h[kSelBins + ((bu >> shift) & mask)], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * kSelBins; k += blockDim.x)
    if (s_h[k]) atomicAdd(&m.hist[k], s_h[k]);
  if (last_cta(m.sel + 3)) select_finish(m, level, c);
}

__global__ void __launch_bounds__(kMpBlock)
mp_labels_kernel(MpWs m, int64_t n, uint8_t *__restrict__ labels) {
  pdl_wait();
  const double tau = m.stats[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (m.obs[i]) labels[i] = (double)m.Mt[i] > tau ? 1 : 0;
}

__global__ void mp_region_stats_kernel(MpWs m, MpCfg c) {
  pdl_wait();
  for (int k = threadIdx.x; k < c.n_regions; k += blockDim.x) {
    float4 reg;
    region_params(m, c, k, &reg);
    const double cnt = m.acc[4 * k + 0];
    double *o = m.stats + DAGS_MP_STATS_HEAD + 4 * k;
    o[0] = cnt;
    o[1] = cnt > 0.0 ? m.acc[4 * k + 1] / cnt : 0.0;
    o[2] = cnt > 0.0 ? sqrt(m.acc[4 * k + 2] / cnt) : 0.0;
    o[3] = reg.y;
  }
}

// Semantic-on-demand trigger, Eqs. (13)-(16): one thread reads the frame's
// U_bar and background residual mean from the MP statistics.
__global__ void semantic_trigger_kernel(const double *__restrict__ stats, double w_u, double w_r, double theta,
                                        double e_ref, int n_max, int seg_refreshed, int32_t *state,
                                        double *score) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double u_bar = stats[1];
  const double cnt0 = stats[DAGS_MP_STATS_HEAD + 0];
  const double e_bar = cnt0 > 0.0 ? stats[DAGS_MP_STATS_HEAD + 1] : 0.0;
  const double R = fmin(fmax(e_bar / e_ref, 0.0), 1.0);
  const double S = w_u * u_bar + w_r * R;
  const int since = seg_refreshed ? 0 : state[0] + 1;
  state[0] = since;
  state[1] = (S > theta || since + 1 >= n_max) ? 1 : 0;
  if (score) {
    score[0] = e_bar;
    score[1] = R;
    score[2] = S;
  }
}

}  // namespace

cudaError_t launch_mp_update(const MpBuffers &b, float *gauss, int64_t n, const double *pose, const Raster &r,
                             const float4 *targets, const float *image, const uint8_t *inst, const float *table,
                             int n_regions, const dags_mp_cfg &cfg, int seg_refreshed, uint8_t *labels,
                             double *stats, const float *mp_map, float *mp_pixel, uint32_t *status,
                             int num_sms, cudaStream_t s) {
  MpWs m;
  m.status = status;
  m.mp_map = mp_map;
  m.mp_pixel = mp_pixel;
  m.mpf = b.mpf;
  m.e = b.e; m.acc = b.acc; m.mhat = b.mhat; m.sige = b.sige; m.U = b.U; m.Mt = b.Mt; m.Ut = b.Ut;
  m.obs = b.obs; m.hist = b.hist; m.sel = b.sel; m.stats = stats;
  MpCfg c;
  c.kappa_c = cfg.kappa_c; c.lam = cfg.lam; c.sigma_min = cfg.sigma_min; c.e_floor = cfg.e_floor;
  c.sigma_g = cfg.sigma_g; c.sigma_c = cfg.sigma_c; c.lam_u = cfg.lam_u; c.eps = cfg.eps;
  c.alpha_min = cfg.alpha_min; c.alpha_max = cfg.alpha_max; c.rho = cfg.rho; c.r_s = cfg.r_s;
  c.sigma_w = cfg.sigma_w; c.vis_tol = cfg.vis_tol; c.z_near = cfg.z_near; c.tau_floor = cfg.tau_floor;
  c.fusion_mode = cfg.fusion_mode; c.seg_refreshed = seg_refreshed; c.n_regions = n_regions;
  c.scales = cfg.scales < 1 ? 1 : (cfg.scales > kMaxScales ? kMaxScales : cfg.scales);
  const int P = r.W * r.H;
  // the association pyramid: level 0 is the frame's own maps, levels 1.. are
  // carved from b.pyr (M_p, e, depth per level)
  float *pyr_out[kMaxScales][3] = {};
  {
    float *cur = b.pyr;
    for (int s = 0; s < kMaxScales; ++s) {
      m.lw[s] = r.W >> s;
      m.lh[s] = r.H >> s;
      if (s == 0) {
        m.lm[0] = mp_map ? mp_map : b.mpf;
        m.le[0] = b.e;
        m.ld[0] = image + 3 * (size_t)P;
        continue;
      }
      const size_t Ps = (size_t)m.lw[s] * m.lh[s];
      for (int k = 0; k < 3; ++k) pyr_out[s][k] = cur + k * Ps;
      cur += 3 * Ps;
      m.lm[s] = pyr_out[s][0];
      m.le[s] = pyr_out[s][1];
      m.ld[s] = pyr_out[s][2];
    }
  }
  // the region accumulators start at zero (the select state is cleared by
  // the first kernel)
  cudaError_t e = cudaMemsetAsync(b.acc, 0, DAGS_MP_MAX_REGIONS * 4 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const unsigned gp = (unsigned)((P + kMpBlock - 1) / kMpBlock);
  const unsigned gg = (unsigned)((n + kMpBlock - 1) / kMpBlock > 0 ? (n + kMpBlock - 1) / kMpBlock : 1);
  // the histogram passes (median selection) and the labels: two CTAs per SM
  // striding over the Gaussians, so that each CTA's clearing and flushing of
  // its 2 x 2048 shared bins is spread over several Gaussians per thread
  const unsigned gs = gg < 2u * (unsigned)num_sms ? gg : 2u * (unsigned)num_sms;
  mp_pixel_sum_kernel<<<gp, kMpBlock, 0, s>>>(m, targets, image, inst, P, c);
  if (e == cudaSuccess) e = launch_pdl(mp_pixel_var_kernel, dim3(gp), dim3(kMpBlock), 0, s, m, inst, P, c);
  if (!mp_map || mp_pixel)
    if (e == cudaSuccess)
      e = launch_pdl(mp_pixel_map_kernel, dim3(gp), dim3(kMpBlock), 0, s, m, inst,
                     reinterpret_cast<const float2 *>(table), r.W, r.H, c);
  for (int l = 1; l < c.scales; ++l) {
    const int Pl = m.lw[l] * m.lh[l];
    if (Pl > 0 && e == cudaSuccess)
      e = launch_pdl(mp_pyramid_kernel, dim3((unsigned)((Pl + kMpBlock - 1) / kMpBlock)), dim3(kMpBlock), 0, s, m, l,
                     pyr_out[l][0], pyr_out[l][1], pyr_out[l][2]);
  }
  if (e == cudaSuccess)
    e = launch_pdl(mp_gauss_kernel, dim3(gg), dim3(kMpBlock), 0, s, m, reinterpret_cast<const float4 *>(gauss), n,
                   pose, image, r, c);
  if (e == cudaSuccess)
    e = launch_pdl(mp_apply_kernel, dim3(gs), dim3(kMpBlock), 0, s, m, reinterpret_cast<float4 *>(gauss), n, c);
  if (e == cudaSuccess) e = launch_pdl(mp_select_kernel, dim3(gs), dim3(kMpBlock), 0, s, m, n, 1, c);
  if (e == cudaSuccess) e = launch_pdl(mp_select_kernel, dim3(gs), dim3(kMpBlock), 0, s, m, n, 2, c);
  if (e == cudaSuccess) e = launch_pdl(mp_labels_kernel, dim3(gs), dim3(kMpBlock), 0, s, m, n, labels);
  if (e == cudaSuccess) e = launch_pdl(mp_region_stats_kernel, dim3(1), dim3(256), 0, s, m, c);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_semantic_trigger(const double *stats, const dags_sched_cfg &cfg, int seg_refreshed,
                                    int32_t *state, double *score, cudaStream_t s) {
  semantic_trigger_kernel<<<1, 32, 0, s>>>(stats, cfg.w_u, cfg.w_r, cfg.theta, cfg.e_ref, cfg.n_max,
                                           seg_refreshed ? 1 : 0, state, score);
  return cudaGetLastError();
}

}  // namespace dags

namespace dags {

namespace {

__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return a | (b << 16);
}

// Per-pixel input of the learned MP network: rendered MP, |dC| (3), |dD|
// where the observed depth is valid, observed depth, rendered opacity, the
// MP_ins of the pixel's region (Eq. (2)); one 16-byte BF16 row per pixel.
__global__ void __launch_bounds__(kMpBlock)
mpnet_features_kernel(const float *__restrict__ image, const float4 *__restrict__ targets,
                      const uint8_t *__restrict__ inst, const float2 *__restrict__ table, int n_regions, int P,
                      uint4 *__restrict__ feats, uint32_t *status) {
  __shared__ float s_mu[DAGS_MP_MAX_REGIONS];
  for (int k = threadIdx.x; k < n_regions; k += blockDim.x) s_mu[k] = table[k].x;
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const size_t Q = (size_t)P;
  const float4 t = __ldg(targets + p);
  const float cr = __ldg(image + p), cg = __ldg(image + Q + p), cb = __ldg(image + 2 * Q + p);
  const float d = __ldg(image + 3 * Q + p), o = __ldg(image + 4 * Q + p), rmp = __ldg(image + 5 * Q + p);
  const bool valid = t.w > 0.f;
  const int k = region_of(inst, p, n_regions, status);
  feats[p] = make_uint4(bf16x2_bits(rmp, fabsf(t.x - cr)), bf16x2_bits(fabsf(t.y - cg), fabsf(t.z - cb)),
                        bf16x2_bits(valid ? fabsf(t.w - d) : 0.f, valid ? t.w : 0.f), bf16x2_bits(o, s_mu[k]));
}

}  // namespace

cudaError_t launch_mpnet_features(const float *image, const float4 *targets, const uint8_t *inst, const float *table,
                                  int n_regions, int P, uint16_t *feats, uint32_t *status, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  mpnet_features_kernel<<<(P + kMpBlock - 1) / kMpBlock, kMpBlock, 0, s>>>(
      image, targets, inst, reinterpret_cast<const float2 *>(table), n_regions, P, reinterpret_cast<uint4 *>(feats),
      status);
  return cudaGetLastError();
}

}  // namespace dags
