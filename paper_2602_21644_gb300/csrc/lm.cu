// Levenberg-Marquardt pose refinement (Sec. V-A(c)) on sm_103a.
//
// The tracking objective is the MP-weighted L1 loss of Eqs. (20)-(22) with
// the static weight w(u) held constant in the linearisation. Its L1 terms
// enter a weighted least-squares problem by iterative reweighting: channel
// residual r with coefficient c (lambda_pho w for r, g, b; lambda_depth w
// where the observed depth is valid) gets the weight W = c / max(|r|, delta).
// One iteration:
//
//   preprocess, tile scan, emit    as for the forward (splat_fwd.cu)
//   pose_tangent_kernel   per visible Gaussian, the derivative of its 2D
//                         record (centre, conic in log2 units, depth) along
//                         the six twist directions xi = (rho, phi) of the
//                         left perturbation T <- exp(xi^) T
//   render_jac_kernel     one CTA per 16x16 tile: the forward compositing
//                         with forward-mode tangents (the derivative of alpha,
//                         of the transmittance and of the composited colour
//                         and depth, 30 accumulators per pixel), then per
//                         pixel the loss and W J J^T, W r J; tile partials in
//                         FP32, the last CTA sums them in FP64 in a fixed order
//                         into (L, H, g)
//   LM step               FP64, one thread on shared-memory copies: accept the
//                         linearisation point if its loss is lower, adapt the
//                         damping, solve the damped 6x6 system by Cholesky and
//                         step the pose; inside the tracking loop it runs in
//                         the last CTA of render_jac_kernel, on its own as
//                         lm_step_kernel
//
// The kernels use programmatic dependent launch like the other splatting
// kernels: each waits for its predecessor's memory before its first access.
#include "common.cuh"
#include "tile_sort.cuh"

namespace dags {

namespace {

constexpr int kJacBatch = kTilePix;   // list entries staged in shared memory per round (one per thread)
constexpr int kJacTanBytes = kJacBatch * 9 * 16;   // their tangent records (dynamic shared memory)
constexpr int kTan4 = 9;         // float4 per Gaussian tangent record (36 floats)
constexpr int kNormal = 28;      // L, the upper triangle of H (21), g (6)

// Tangent record of a visible Gaussian: for twist direction k = 0..5 the six
// floats (du, dv, da', db', dc', dz) at offset 6k, where (a', b', c') are the
// exponent coefficients of the projected record (log2 units).
__global__ void __launch_bounds__(kPrepBlock, 6)
pose_tangent_kernel(Workspace ws, const float4 *__restrict__ gauss, int64_t n, Raster r,
                    float4 *__restrict__ tan) {
  pdl_wait();
  // the tracking loop's bucket layout: the grid's first CTA (dispatched
  // first, so that it runs beside the first wave) ranks the tiles by the
  // previous Jacobian render's counts into this iteration's render order,
  // and the visible list is still the preprocess's append cursor
  const bool ordering = ws.order_next != nullptr;
  if (ordering && blockIdx.x == 0) {
    rank_tiles(ws.prev_count, r.T, ws.order_next, ws.band);
    return;
  }
  const int64_t nb = (int64_t)gridDim.x - (ordering ? 1 : 0);
  const int64_t bid = (int64_t)blockIdx.x - (ordering ? 1 : 0);
  const uint32_t nv = ws.bucket_cap ? ws.vis_append[0] : ws.vis_n[0];
  float P[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) P[k] = ws.pose32[k];
  for (int64_t t = bid * blockDim.x + threadIdx.x; t < (int64_t)nv; t += nb * blockDim.x) {
    const uint32_t id = ws.vis_ids[t];
    if (!DAGS_IN_BOUNDS(id < (uint64_t)n, ws.counters + CNT_STATUS)) continue;
    const float4 g0 = __ldg(gauss + 4 * id), g1 = __ldg(gauss + 4 * id + 1), g2 = __ldg(gauss + 4 * id + 2);
    Proj q;
    float out[36];
    if (!project_gaussian(g0, g1, g2, P, r, q)) {
#pragma unroll
      for (int k = 0; k < 36; ++k) out[k] = 0.f;
    } else {
      const float x = q.x, y = q.y, z = q.z;
      const float iz = 1.f / z, iz2 = iz * iz;
      const bool clx = q.txz > r.limx || q.txz < -r.limx;
      const bool cly = q.tyz > r.limy || q.tyz < -r.limy;
      const float idet = 1.f / q.det;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        // camera mean: e_k (rho), phi x p (phi); K = R_cw Rq S: [phi]x K
        float dp[3] = {0.f, 0.f, 0.f}, dK[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) dK[e] = 0.f;
        if (k < 3) {
          dp[k] = 1.f;
        } else if (k == 3) {
          dp[1] = -z; dp[2] = y;
#pragma unroll
          for (int s = 0; s < 3; ++s) { dK[3 + s] = -q.K[6 + s]; dK[6 + s] = q.K[3 + s]; }
        } else if (k == 4) {
          dp[0] = z; dp[2] = -x;
#pragma unroll
          for (int s = 0; s < 3; ++s) { dK[s] = q.K[6 + s]; dK[6 + s] = -q.K[s]; }
        } else {
          dp[0] = -y; dp[1] = x;
#pragma unroll
          for (int s = 0; s < 3; ++s) { dK[s] = -q.K[3 + s]; dK[3 + s] = q.K[s]; }
        }
        // the guard clamp freezes x/z (y/z) in the Jacobian
        const float dtx = clx ? 0.f : (dp[0] * z - x * dp[2]) * iz2;
        const float dty = cly ? 0.f : (dp[1] * z - y * dp[2]) * iz2;
        const float dj00 = -r.fx * dp[2] * iz2, dj02 = -r.fx * (dtx * z - q.tx * dp[2]) * iz2;
        const float dj11 = -r.fy * dp[2] * iz2, dj12 = -r.fy * (dty * z - q.ty * dp[2]) * iz2;
        float dA = 0.f, dB = 0.f, dC = 0.f;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          const float dm0 = dj00 * q.K[s] + q.j00 * dK[s] + dj02 * q.K[6 + s] + q.j02 * dK[6 + s];
          const float dm1 = dj11 * q.K[3 + s] + q.j11 * dK[3 + s] + dj12 * q.K[6 + s] + q.j12 * dK[6 + s];
          dA += 2.f * q.m0[s] * dm0;
          dC += 2.f * q.m1[s] * dm1;
          dB += dm0 * q.m1[s] + q.m0[s] * dm1;
        }
        // conic (ca, cb, cc) = (C, -B, A) / det
        const float ddet = dA * q.C + q.A * dC - 2.f * q.B * dB;
        const float dca = (dC - q.ca * ddet) * idet;
        const float dcb = (-dB - q.cb * ddet) * idet;
        const float dcc = (dA - q.cc * ddet) * idet;
        out[6 * k + 0] = r.fx * (dp[0] * z - x * dp[2]) * iz2;
        out[6 * k + 1] = r.fy * (dp[1] * z - y * dp[2]) * iz2;
        out[6 * k + 2] = -0.5f * kLog2e * dca;
        out[6 * k + 3] = -kLog2e * dcb;
        out[6 * k + 4] = -0.5f * kLog2e * dcc;
        out[6 * k + 5] = dp[2];
      }
    }
    float4 *o = tan + (size_t)id * kTan4;
#pragma unroll
    for (int w = 0; w < kTan4; ++w) o[w] = make_float4(out[4 * w], out[4 * w + 1], out[4 * w + 2], out[4 * w + 3]);
  }
}

// Index of H[a][b] (a <= b) in the packed upper triangle.
__host__ __device__ constexpr int tri(int a, int b) { return a * 6 - a * (a - 1) / 2 + (b - a); }

// LM state (DAGS_LM_STATE doubles): T_best[12], L_best, mu, H_best[21],
// g_best[6], accepted count, iteration count, last L, last accepted flag.
enum { ST_T = 0, ST_L = 12, ST_MU = 13, ST_H = 14, ST_G = 35, ST_ACC = 41, ST_IT = 42, ST_LAST_L = 43,
       ST_LAST_A = 44 };

// One LM decision and damped step by one thread, on shared-memory copies:
// n the normal equations at p (the linearisation point), st the state; on
// return st is updated and p holds the next linearisation point.
__device__ void lm_decide_solve(const double *n, double *st, double *p, const dags_lm_cfg &c) {
  const double L = n[0];
  double mu = st[ST_MU];
  const bool accept = L < st[ST_L];
  if (accept) {
    for (int k = 0; k < 12; ++k) st[ST_T + k] = p[k];
    st[ST_L] = L;
    for (int k = 0; k < 21; ++k) st[ST_H + k] = n[1 + k];
    for (int k = 0; k < 6; ++k) st[ST_G + k] = n[22 + k];
    mu = fmax(mu * c.down, c.mu_min);
    st[ST_ACC] += 1.0;
  } else {
    mu = fmin(mu * c.up, c.mu_max);
  }
  st[ST_MU] = mu;
  st[ST_IT] += 1.0;
  st[ST_LAST_L] = L;
  st[ST_LAST_A] = accept ? 1.0 : 0.0;
  // (H + mu diag(H) + floor tr(H)/6 I) delta = -g by Cholesky
  double A[6][6], d[6];
  double tr = 0.0;
  for (int a = 0; a < 6; ++a) tr += st[ST_H + tri(a, a)];
  bool ok = tr > 0.0;
  if (ok) {
    for (int a = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b) A[a][b] = A[b][a] = st[ST_H + tri(a, b)];
    for (int a = 0; a < 6; ++a) A[a][a] += mu * A[a][a] + c.floor * (tr / 6.0);
    for (int j = 0; j < 6 && ok; ++j) {
      double sjj = A[j][j];
      for (int k = 0; k < j; ++k) sjj -= A[j][k] * A[j][k];
      if (!(sjj > 0.0)) { ok = false; break; }
      // the diagonal holds 1 / l_jj: one reciprocal square root per pivot and
      // multiplications elsewhere (dependent FP64 divisions are what costs)
      const double inv = rsqrt(sjj);
      A[j][j] = inv;
      for (int i = j + 1; i < 6; ++i) {
        double sij = A[i][j];
        for (int k = 0; k < j; ++k) sij -= A[i][k] * A[j][k];
        A[i][j] = sij * inv;
      }
    }
  }
  if (ok) {
    double y[6];
    for (int i = 0; i < 6; ++i) {
      double t = -st[ST_G + i];
      for (int k = 0; k < i; ++k) t -= A[i][k] * y[k];
      y[i] = t * A[i][i];
    }
    for (int i = 5; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < 6; ++k) t -= A[k][i] * d[k];
      d[i] = t * A[i][i];
    }
  } else {
    for (int i = 0; i < 6; ++i) d[i] = 0.0;
  }
  double T[12];
  for (int k = 0; k < 12; ++k) T[k] = st[ST_T + k];
  se3_exp_left(T, d);
  for (int k = 0; k < 12; ++k) p[k] = T[k];
}

// The LM step by a CTA of at least 48 threads (all must call it): the inputs
// are staged in shared memory by parallel loads, one thread decides and
// solves, and the results are written back in parallel.
__device__ void lm_step_cta(const double *nrm, double *state, double *pose_try, double *pose_best,
                            const dags_lm_cfg &c) {
  __shared__ double s_n[kNormal], s_st[DAGS_LM_STATE], s_p[12];
  const int t = threadIdx.x;
  if (t < kNormal) s_n[t] = nrm[t];
  if (t < DAGS_LM_STATE) s_st[t] = state[t];
  if (t < 12) s_p[t] = pose_try[t];
  __syncthreads();
  if (t == 0) lm_decide_solve(s_n, s_st, s_p, c);
  __syncthreads();
  if (t < DAGS_LM_STATE) state[t] = s_st[t];
  if (t < 12) {
    pose_try[t] = s_p[t];
    pose_best[t] = s_st[ST_T + t];
  }
}

// Three CTAs per SM (a budget of 80 registers, 30 tangent accumulators per
// pixel, some of them spilled to L1): the kernel is bound by instruction
// issue, and six warps per scheduler hide more latency than the four that
// the unspilled 118 registers allowed (146 against 160 us per launch at the
// tracking size; four CTAs per SM spill more and take 154).
__global__ void __launch_bounds__(kTilePix, 3)
render_jac_kernel(Workspace ws, Raster r, Loss l, float delta, const float4 *__restrict__ targets,
                  const float4 *__restrict__ tan, float *__restrict__ partial, double *__restrict__ normal,
                  float *__restrict__ jac, float *__restrict__ image, int32_t *__restrict__ last, LmFuse fuse) {
  pdl_wait();
  __shared__ __align__(16) uint64_t s_key[kSortSmallCap];
  __shared__ float4 s_a[kJacBatch], s_b[kJacBatch], s_c[kJacBatch];   // s_a: {u hi, v hi, u lo, v lo}
  __shared__ float2 s_e[kJacBatch];                                   // box half extents
  extern __shared__ float4 s_t[];   // kJacBatch * kTan4
  __shared__ float s_red[kTilePix / 32][kNormal];
  __shared__ int s_last;
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the tracking loop's fixed-capacity buckets: a tile whose list overflowed
  // its bucket is skipped and reported, and the render publishes the counts
  // and the visible count as the forward of the first-order loop does;
  // otherwise an overflow anywhere skips every tile
  bool ovf;
  int tile;
  if (ws.bucket_cap) {
    tile = (int)ws.tile_order[blockIdx.x];
    const uint32_t c = ws.tile_count[tile];
    ovf = c > ws.bucket_cap;
    if (tid == 0) {
      ws.prev_count[tile] = c;
      atomicMax(reinterpret_cast<unsigned long long *>(ws.counters + CNT_REQ_LO), (unsigned long long)c * r.T);
      if (ovf) atomicOr(ws.counters + CNT_STATUS, kStatusCapacity);
      if (blockIdx.x == 0) {
        ws.vis_n[0] = ws.vis_append[0];
        ws.vis_append[0] = 0u;
      }
    }
  } else {
    ovf = pairs_overflow_ws(ws);
    tile = ovf ? (int)blockIdx.x : (int)ws.tile_order[blockIdx.x];
  }
  const int tx = tile % r.tiles_x, ty = tile / r.tiles_x;
  const int bx0 = tx * kTile + (warp & 1) * 8, by0 = ty * kTile + (warp >> 1) * 4;
  const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
  const bool inside = px < r.W && py < r.H;
  uint32_t s = 0u, e = 0u;
  if (!ovf) tile_range(ws, tile, s, e);
  const float bcx = (float)bx0 + 3.5f, bcy = (float)by0 + 1.5f;
  const bool own_sort = sort_tile_bucket(ws, s, (int)(e - s), s_key);

  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f, oo = 0.f, rm = 0.f;
  float dT[6], jr[6], jg[6], jb[6], jd[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) { dT[k] = 0.f; jr[k] = 0.f; jg[k] = 0.f; jb[k] = 0.f; jd[k] = 0.f; }
  int lastk = 0;
  bool done = !inside;
  const float fpx = (float)px, fpy = (float)py;
  for (uint32_t base = s; base < e; base += kJacBatch) {
    if (__syncthreads_count(!done) == 0) break;
    const int cnt = (int)min((uint32_t)kJacBatch, e - base);
    // thread q stages entry q: its record and its tangent record
    const int q = tid;
    if (q < cnt) {
      const uint32_t k = base + q;
      uint32_t id = own_sort ? (uint32_t)s_key[k - s] : ws.sorted_ids[k];
      if (!DAGS_IN_BOUNDS(id < (uint32_t)ws.max_n, ws.counters + CNT_STATUS)) id = 0;
      const float4 *tg = tan + (size_t)id * kTan4;
      float4 *st = s_t + q * kTan4;
      const float4 r0 = ws.rec2d[(size_t)id * 3 + 0];
      const float2 lo = ws.rec_lo[id];
      s_a[q] = make_float4(r0.x, r0.y, lo.x, lo.y);
      s_e[q] = make_float2(r0.z, r0.w);
      s_b[q] = ws.rec2d[(size_t)id * 3 + 1];
      s_c[q] = ws.rec2d[(size_t)id * 3 + 2];
#pragma unroll
      for (int w = 0; w < kTan4; ++w) st[w] = tg[w];
    }
    __syncthreads();
    if (__all_sync(FULL, done)) continue;
    for (int g = 0; g < kJacBatch / 32 && g * 32 < cnt; ++g) {
      const int jj = g * 32 + lane;
      bool hit = false;
      if (jj < cnt) {
        const float4 a = s_a[jj];
        const float2 ex = s_e[jj];
        hit = fabsf(a.x - bcx) <= ex.x + 3.5f && fabsf(a.y - bcy) <= ex.y + 1.5f;
      }
      unsigned mask = __ballot_sync(FULL, hit);
      while (mask) {
        const int j = g * 32 + __ffs(mask) - 1;
        mask &= mask - 1;
        if (done) continue;
        const float4 a = s_a[j], b = s_b[j];
        const float dx = (a.x - fpx) + a.z, dy = (a.y - fpy) + a.w;
        const float p = fmaf(b.x * dx, dx, fmaf(b.y * dx, dy, fmaf(b.z * dy, dy, b.w)));
        if (p < r.log2_alpha_min) continue;
        const float ag = hw_exp2(p);
        const bool clamped = ag > r.alpha_max;
        const float alpha = clamped ? r.alpha_max : ag;
        const float tt = T * (1.f - alpha);
        if (tt < r.t_min) { done = true; continue; }
        const float w = alpha * T;
        const float4 c = s_c[j];
        const uint32_t rg = __float_as_uint(c.z), bl = __float_as_uint(c.w);
        const float cR = bf16_lo(rg), cG = bf16_hi(rg), cB = bf16_lo(bl);
        cr += cR * w; cg += cG * w; cb += cB * w;
        dd += c.x * w; oo += w; rm += c.y * w;
        // tangents: p' = da' dx^2 + db' dx dy + dc' dy^2 + dp/du du + dp/dv dv,
        // alpha' = alpha ln2 p' (0 where clamped), weight' = alpha' T + alpha T';
        // the next entry's T = T - weight, so its T' = T' - weight'
        const float gx = fmaf(2.f * b.x, dx, b.y * dy), gy = fmaf(b.y, dx, 2.f * b.z * dy);
        const float dx2 = dx * dx, dxy = dx * dy, dy2 = dy * dy;
        const float aln = clamped ? 0.f : alpha * kLn2;
        const float4 *t4 = s_t + j * kTan4;
        float tv[36];
#pragma unroll
        for (int q = 0; q < kTan4; ++q) {
          const float4 v4 = t4[q];
          tv[4 * q] = v4.x; tv[4 * q + 1] = v4.y; tv[4 * q + 2] = v4.z; tv[4 * q + 3] = v4.w;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float *t = tv + 6 * k;
          const float dp = fmaf(t[2], dx2, fmaf(t[3], dxy, fmaf(t[4], dy2, fmaf(gx, t[0], gy * t[1]))));
          const float da = aln * dp;
          const float dw = fmaf(da, T, alpha * dT[k]);
          jr[k] = fmaf(cR, dw, jr[k]);
          jg[k] = fmaf(cG, dw, jg[k]);
          jb[k] = fmaf(cB, dw, jb[k]);
          jd[k] = fmaf(c.x, dw, fmaf(w, t[5], jd[k]));
          dT[k] -= dw;
        }
        T = tt;
        lastk = (int)(base - s) + j + 1;
      }
      if (__all_sync(FULL, done)) break;
    }
  }

  float acc[kNormal];
#pragma unroll
  for (int k = 0; k < kNormal; ++k) acc[k] = 0.f;
  if (inside) {
    const size_t P = (size_t)r.W * r.H;
    const size_t pix = (size_t)py * r.W + px;
    float wgt;
    if (l.weight_mode == 0) wgt = oo > l.o_eps ? (oo - rm) / oo : 0.f;
    else wgt = oo - rm;
    const float4 tg = targets[pix];
    const bool dvalid = tg.w > 0.f;
    if (tg.x >= 0.f) {
      const float res[4] = {cr - tg.x, cg - tg.y, cb - tg.z, dd - tg.w};
      const float coef[4] = {l.lambda_pho * wgt, l.lambda_pho * wgt, l.lambda_pho * wgt,
                             dvalid ? l.lambda_depth * wgt : 0.f};
      const float l1 = fabsf(res[0]) + fabsf(res[1]) + fabsf(res[2]);
      acc[0] = wgt * (l.lambda_pho * l1 + (dvalid ? l.lambda_depth * fabsf(res[3]) : 0.f));
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        const float *J = ch == 0 ? jr : ch == 1 ? jg : ch == 2 ? jb : jd;
        const float W = coef[ch] / fmaxf(fabsf(res[ch]), delta);
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          const float wa = W * J[a];
          acc[22 + a] = fmaf(wa, res[ch], acc[22 + a]);
#pragma unroll
          for (int b2 = a; b2 < 6; ++b2) acc[1 + tri(a, b2)] = fmaf(wa, J[b2], acc[1 + tri(a, b2)]);
        }
      }
    }
    if (jac) {
      float4 *jp = reinterpret_cast<float4 *>(jac + pix * 24);
      jp[0] = make_float4(jr[0], jr[1], jr[2], jr[3]);
      jp[1] = make_float4(jr[4], jr[5], jg[0], jg[1]);
      jp[2] = make_float4(jg[2], jg[3], jg[4], jg[5]);
      jp[3] = make_float4(jb[0], jb[1], jb[2], jb[3]);
      jp[4] = make_float4(jb[4], jb[5], jd[0], jd[1]);
      jp[5] = make_float4(jd[2], jd[3], jd[4], jd[5]);
    }
    if (image) {
      float *img = image + pix;
      img[0 * P] = cr; img[1 * P] = cg; img[2 * P] = cb; img[3 * P] = dd;
      img[4 * P] = oo; img[5 * P] = rm; img[6 * P] = T; img[7 * P] = wgt;
    }
    if (last) last[pix] = lastk;
  }
  // tile partials: warp sums, then the 8 warps in a fixed order
#pragma unroll
  for (int k = 0; k < kNormal; ++k) {
    const float v = warp_sum(acc[k]);
    if (lane == 0) s_red[warp][k] = v;
  }
  __syncthreads();
  if (tid < kNormal) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kTilePix / 32; ++w) t += s_red[w][tid];
    // by tile, so that the final sum's order does not depend on the launch order
    partial[(size_t)tile * kNormal + tid] = t;
  }
  __syncthreads();
  if (tid == 0) {
    // the bucket is empty again for the next iteration's binning (its list
    // was read before the compositing)
    if (ws.bucket_cap) ws.tile_count[tile] = 0u;
    __threadfence();
    const unsigned int done_ctas = atomicAdd(ws.counters + CNT_DONE_RENDER, 1u);
    s_last = (done_ctas == gridDim.x - 1);
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  // FP64 sum of the tile partials: column c by 8 threads with a fixed stride,
  // then those 8 in order
  __shared__ double s_d[kNormal * 8];
  if (tid < kNormal * 8) {
    const int c = tid >> 3, part = tid & 7;
    // four independent accumulators per thread (dependent FP64 additions
    // are slow on GB300), combined in a fixed order
    double a4[4] = {0.0, 0.0, 0.0, 0.0};
    int j = 0;
    for (int k = part; k < (int)gridDim.x; k += 8, ++j) a4[j & 3] += (double)__ldcg(partial + (size_t)k * kNormal + c);
    s_d[tid] = (a4[0] + a4[1]) + (a4[2] + a4[3]);
  }
  __syncthreads();
  __shared__ double s_nrm[kNormal];
  // a pair-capacity overflow leaves tiles unrendered (all of them in the
  // general layout; in the bucket layout those whose list exceeded its
  // bucket, which the largest requirement of this iteration tells)
  bool any_ovf = ovf;
  if (ws.bucket_cap)
    any_ovf = __ldcg(reinterpret_cast<const unsigned long long *>(ws.counters + CNT_REQ_LO)) >
              (unsigned long long)ws.bucket_cap * (unsigned long long)r.T;
  if (tid < kNormal) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += s_d[tid * 8 + k];
    // then the loss is NaN, so the LM step rejects this point
    if (any_ovf && tid == 0) t = __longlong_as_double(0x7ff8000000000000ll);
    normal[tid] = t;
    s_nrm[tid] = t;
  }
  if (tid == 0) ws.counters[CNT_DONE_RENDER] = 0u;
  __syncthreads();
  // inside the LM loop the step runs here, in the last CTA
  if (fuse.state) {
    lm_step_cta(s_nrm, fuse.state, fuse.pose_try, fuse.pose_best, fuse.cfg);
    // the bucket layout: if the next linearisation point (as the preprocess
    // stages it in FP32) has left the bounds the candidates were culled for,
    // move the culling pose to it and empty the list; the next preprocess
    // then takes every Gaussian once and re-culls
    if (ws.bucket_cap && ws.cand_n && ws.cull_pose) {
      __shared__ float s_np[12];
      __shared__ int s_out;
      __syncthreads();
      if (tid < 12) s_np[tid] = __double2float_rn(fuse.pose_try[tid]);
      __syncthreads();
      if (tid == 0) s_out = within_cull_bounds(s_np, ws.cull_pose) ? 0 : 1;
      __syncthreads();
      if (s_out && tid < 12) ws.cull_pose[tid] = s_np[tid];
      if (tid == 0) {
        if (s_out) *ws.cand_n = 0u;
        ws.counters[CNT_RECULL] = s_out ? 1u : 0u;
      }
    }
  }
}

__global__ void lm_init_kernel(const double *__restrict__ pose, double *__restrict__ state,
                               double *__restrict__ pose_try, double mu0) {
  pdl_wait();
  const int t = threadIdx.x;
  if (t < 12) {
    state[ST_T + t] = pose[t];
    pose_try[t] = pose[t];
  }
  if (t >= 12 && t < DAGS_LM_STATE) state[t] = 0.0;
  __syncthreads();
  if (t == 0) {
    state[ST_L] = __longlong_as_double(0x7ff0000000000000ll);   // +inf: the first point is accepted
    state[ST_MU] = mu0;
  }
}

__global__ void lm_step_kernel(const double *__restrict__ normal, double *__restrict__ state,
                               double *__restrict__ pose_try, double *__restrict__ pose_best, dags_lm_cfg c) {
  pdl_wait();
  lm_step_cta(normal, state, pose_try, pose_best, c);
}

}  // namespace

cudaError_t launch_pose_tangents(const Workspace &ws, const float4 *gauss, int64_t n, const Raster &r, float4 *tan,
                                 int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t need = (n + kPrepBlock - 1) / kPrepBlock;
  const unsigned grid = (unsigned)(need < (int64_t)num_sms * 8 ? need : (int64_t)num_sms * 8);
  // (plus the ranking CTA of the tracking loop)
  return launch_pdl(pose_tangent_kernel, dim3(grid + (ws.order_next ? 1u : 0u)), dim3(kPrepBlock), 0, s, ws, gauss,
                    n, r, tan);
}

// The Jacobian render's dynamic shared memory (the batch's tangent records)
// exceeds the default 48 KB: raised once per device, at the ctx's first LM
// call (before any stream capture).
cudaError_t lm_kernel_setup() {
  return cudaFuncSetAttribute(render_jac_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kJacTanBytes);
}

cudaError_t launch_render_jac(const Workspace &ws, const Raster &r, const Loss &l, float delta,
                              const float4 *targets, const float4 *tan, float *partial, double *normal, float *jac,
                              float *image, int32_t *last, const LmFuse &fuse, cudaStream_t s) {
  return launch_pdl(render_jac_kernel, dim3((unsigned)r.T), dim3(kTilePix), kJacTanBytes, s, ws, r, l, delta, targets, tan,
                    partial, normal, jac, image, last, fuse);
}

cudaError_t launch_lm_init(const double *pose, double *state, double *pose_try, double mu0, cudaStream_t s) {
  return launch_pdl(lm_init_kernel, dim3(1), dim3(64), 0, s, pose, state, pose_try, mu0);
}

cudaError_t launch_lm_step(const double *normal, double *state, double *pose_try, double *pose_best,
                           const dags_lm_cfg &c, cudaStream_t s) {
  return launch_pdl(lm_step_kernel, dim3(1), dim3(64), 0, s, normal, state, pose_try, pose_best, c);
}

}  // namespace dags
