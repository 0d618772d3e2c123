// Backward half of the MP-aware splatting path (sm_103a).
//
//   render_bwd_kernel      one CTA per 16x16 tile: walks the tile's sorted
//                          list back to front from the furthest recorded
//                          contributor, re-deriving each pixel's
//                          transmittance from its final value (T_k =
//                          T_{k+1} / (1 - alpha_k)) with running suffix sums,
//                          so no per-pair state is stored; the per-Gaussian
//                          2D gradients of the 32 pixels of a warp are summed
//                          with shuffles and added with one atomic per
//                          Gaussian per warp.
//   preprocess_bwd_kernel  per Gaussian over all views: chains the 2D
//                          gradients through conic, EWA covariance, Jacobian,
//                          camera transform, scale and rotation to the record's
//                          parameters, and to the pose twist (mean and
//                          covariance paths); per-view pose partials are summed
//                          per CTA and then, by the last CTA, in a fixed order
//                          in FP64.
#include "common.cuh"
#include "tile_sort.cuh"

namespace dags {

namespace {

constexpr int kMaxViewsSmem = 64;
// the reduce-scatter's component k is 2D-gradient word k
static_assert(G2_U == 0 && G2_Z == 5 && G2_BL == 9 && kGradWords >= 10, "2D-gradient word order");

// FULL: every parameter's 2D gradients (else the pose path's six words);
// MASKS: visit only the entries the forward recorded as taken by the warp
// (ws.warp_masks); COUNT: count evaluations and contributions (ws.evals).
template <bool FULL, bool MASKS, bool COUNT>
__global__ void __launch_bounds__(kTilePix, 5)
render_bwd_kernel(Workspace ws, Raster r, Loss l, const float4 *__restrict__ targets,
                  const float *__restrict__ image, const int32_t *__restrict__ last,
                  const float *__restrict__ upstream) {
  pdl_wait();
  pdl_trigger();
  __shared__ float4 s_a[kTilePix], s_b[kTilePix], s_c[kTilePix];   // s_a: {u hi, v hi, u lo, v lo}
  __shared__ float2 s_e[kTilePix];                                  // box half extents
  __shared__ float *s_dst[kTilePix];                                // the entry's 2D-gradient words
  __shared__ int s_max;
  const unsigned FULLM = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (ws.bucket_cap) {
    // fixed-bucket layout: an overflowed tile is skipped (its count is
    // cleared for the next preprocess all the same)
    const int t = (int)ws.tile_order[blockIdx.x];
    if (ws.tile_count[t] > ws.bucket_cap) {
      __syncthreads();
      if (tid == 0) ws.tile_count[t] = 0u;
      return;
    }
  } else {
    const uint64_t tot = (uint64_t)ws.counters[CNT_REQ_LO] | ((uint64_t)ws.counters[CNT_REQ_HI] << 32);
    if (tot > (uint64_t)ws.max_pairs) return;
  }
  // the 2D-gradient word whose warp sum this lane receives from the
  // reduce-scatter below (words G2_U .. G2_Z, and with FULL up to G2_BL), and
  // whether it is the lowest lane holding that word (the one that adds it)
  const int comp = FULL ? rs_component<10>(lane) : rs_component<6>(lane);
  const bool writer = __ffs(__match_any_sync(0xffffffffu, (unsigned)comp)) - 1 == lane;
  const int tile = (int)ws.tile_order[blockIdx.x];   // longest lists first
  const int v = tile / r.T, tv = tile - v * r.T;
  const int tx = tv % r.tiles_x, ty = tv / r.tiles_x;
  const int bx0 = tx * kTile + (warp & 1) * 8, by0 = ty * kTile + (warp >> 1) * 4;
  const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
  const bool inside = px < r.W && py < r.H;
  uint32_t s, e_unused;
  tile_range(ws, tile, s, e_unused);
  // the forward's record of the entries this warp's pixels took (groups of
  // 32 entries; later groups fall back to the box test)
  const uint32_t *const wmask = MASKS ? ws.warp_masks + (size_t)tile * kMaskGroups * 8 + warp : nullptr;
  const size_t vbase = (size_t)v * ws.max_n;
  const size_t P = (size_t)r.W * r.H;
  const float bcx = (float)bx0 + 3.5f, bcy = (float)by0 + 1.5f;

  float T = 1.f;
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f, g5 = 0.f;  // upstream per channel
  int lastp = 0;
  if (inside && upstream) {
    // the caller's gradients of its own function of the six composited
    // channels take the place of the loss's
    const size_t pix = (size_t)py * r.W + px;
    const float *up = upstream + (size_t)v * 6 * P + pix;
    g0 = up[0]; g1 = up[P]; g2 = up[2 * P]; g3 = up[3 * P]; g4 = up[4 * P]; g5 = up[5 * P];
    T = image[(size_t)v * DAGS_IMG_CHANNELS * P + 6 * P + pix];
    lastp = last[(size_t)v * P + pix];
  } else if (inside) {
    // a pixel whose target has negative red is outside the loss (no gradient)
    const size_t pix = (size_t)py * r.W + px;
    const float *img = image + (size_t)v * DAGS_IMG_CHANNELS * P + pix;
    const float cr = img[0], cg = img[P], cb = img[2 * P], dd = img[3 * P];
    const float oo = img[4 * P], rm = img[5 * P];
    T = img[6 * P];
    const float w = img[7 * P];
    const float4 tg = targets[(size_t)v * P + pix];
    lastp = tg.x >= 0.f ? last[(size_t)v * P + pix] : 0;
    const float rc0 = cr - tg.x, rc1 = cg - tg.y, rc2 = cb - tg.z, rd = dd - tg.w;
    const bool dvalid = tg.w > 0.f;
    auto sgn = [](float x) { return (float)((x > 0.f) - (x < 0.f)); };
    g0 = l.lambda_pho * w * sgn(rc0);
    g1 = l.lambda_pho * w * sgn(rc1);
    g2 = l.lambda_pho * w * sgn(rc2);
    g3 = dvalid ? l.lambda_depth * w * sgn(rd) : 0.f;
    if (l.weight_grad) {
      const float lw = l.lambda_pho * (fabsf(rc0) + fabsf(rc1) + fabsf(rc2)) +
                       (dvalid ? l.lambda_depth * fabsf(rd) : 0.f);
      if (l.weight_mode == 0) {
        if (oo > l.o_eps) { g4 = lw * rm / (oo * oo); g5 = -lw / oo; }
      } else {
        g4 = lw;
        g5 = -lw;
      }
    }
  }
  if (tid == 0) s_max = 0;
  __syncthreads();
  const int wmax = (int)__reduce_max_sync(FULLM, (unsigned)lastp);
  if (lane == 0) atomicMax(&s_max, wmax);
  __syncthreads();
  const int kmax = s_max;

  // Sg = sum over channels of g_ch * S_ch, S_ch the channel's composited sum
  // behind the current Gaussian: dL/dalpha needs only this contraction
  float Sg = 0.f;
  unsigned n_eval = 0, n_contrib = 0;
  const float fpx = (float)px, fpy = (float)py;
  // batches of kTilePix entries aligned as the forward's (the recorded
  // masks address entries by their 32-entry group in the tile's list); the
  // first batch walked is the one holding the last contributor
  for (int end = kmax, beg; end > 0; end = beg) {
    beg = ((end - 1) / kTilePix) * kTilePix;
    __syncthreads();
    if (beg + tid < end && DAGS_IN_BOUNDS((uint64_t)s + beg + tid < (uint64_t)ws.max_pairs, ws.counters + CNT_STATUS)) {
      uint32_t id = ws.sorted_ids[s + beg + tid];
      if (!DAGS_IN_BOUNDS(id < (uint32_t)ws.max_n, ws.counters + CNT_STATUS)) id = 0;
      const size_t slot = vbase + id;
      s_dst[tid] = ws.grad2d + slot * kGradWords;
      const float4 r0 = ws.rec2d[slot * 3 + 0];
      const float2 lo = ws.rec_lo[slot];
      s_a[tid] = make_float4(r0.x, r0.y, lo.x, lo.y);
      s_e[tid] = make_float2(r0.z, r0.w);
      s_b[tid] = ws.rec2d[slot * 3 + 1];
      s_c[tid] = ws.rec2d[slot * 3 + 2];
    }
    __syncthreads();
    const int cnt = end - beg;
    if (wmax <= beg) continue;               // no pixel of this warp reaches this batch
    const int top = min(cnt, wmax - beg);    // entries [beg, beg + top) may matter to this warp
    for (int g = (top - 1) >> 5; g >= 0; --g) {
      const int gk = (beg >> 5) + g;
      unsigned mask;
      const bool recorded = MASKS && gk < kMaskGroups;
      if (recorded) {
        mask = __ldg(wmask + gk * 8);
      } else {
        const int jj = g * 32 + lane;
        bool hit = false;
        if (jj < cnt) {
          const float4 a = s_a[jj];
          const float2 ex = s_e[jj];
          hit = fabsf(a.x - bcx) <= ex.x + 3.5f && fabsf(a.y - bcy) <= ex.y + 1.5f;
        }
        mask = __ballot_sync(FULLM, hit);
      }
      const int lim = top - g * 32;
      if (lim < 32) mask &= (1u << lim) - 1u;
      while (mask) {
        const int bit = 31 - __clz(mask);
        mask &= ~(1u << bit);
        const int j = g * 32 + bit;
        const int k = beg + j;
        // evaluated by every lane, without branches: a lane past its last
        // contributor or below alpha_min keeps T and Sg and carries zero
        // gradients, so each contributing lane's values are those of the
        // branching form, operation for operation
        const float4 a = s_a[j], b = s_b[j];
        const float dx = (a.x - fpx) + a.z, dy = (a.y - fpy) + a.w;
        const float bxdx = b.x * dx, bydx = b.y * dx, bzdy = b.z * dy;
        const float p = fmaf(bxdx, dx, fmaf(bydx, dy, fmaf(bzdy, dy, b.w)));
        const bool contrib = k < lastp && p >= r.log2_alpha_min;
        if (COUNT) { n_eval += k < lastp ? 1u : 0u; n_contrib += contrib ? 1u : 0u; }
        const float ag = hw_exp2(p);
        const float alpha = fminf(r.alpha_max, ag);
        const float inv = hw_rcp(1.f - alpha);
        T = contrib ? T * inv : T;           // transmittance in front of this Gaussian
        // the weight, zero for a lane that does not take the entry (its
        // depth gradient and suffix update then vanish without a select)
        const float wk = contrib ? alpha * T : 0.f;
        const float4 c = s_c[j];
        const uint32_t rgb = __float_as_uint(c.z), blb = __float_as_uint(c.w);
        const float fr = bf16_lo(rgb), fg = bf16_hi(rgb), fb = bf16_lo(blb);
        // dL/dalpha = sum_ch g_ch (c_ch T - S_ch / (1 - alpha))
        const float gcv = fmaf(g0, fr, fmaf(g1, fg, fmaf(g2, fb, fmaf(g3, c.x, fmaf(g5, c.y, g4)))));
        const float dal = fmaf(gcv, T, -Sg * inv);
        const float gz = g3 * wk;
        float gr = 0.f, gg = 0.f, gbl = 0.f, go = 0.f;
        if (FULL) {
          gr = g0 * wk;
          gg = g1 * wk;
          gbl = g2 * wk;
        }
        // below the clamp, d alpha / d(natural exponent) = alpha; the
        // exponent in log2 units is p, so d/dx of the natural exponent is
        // ln2 * dp/dx (at the clamp alpha does not move with the exponent)
        const bool slope = contrib && ag <= r.alpha_max;
        const float dpw = slope ? dal * alpha : 0.f;
        const float hl = dpw * kLn2;
        // d p / d(u, v) = (2 a' dx + b' dy, b' dx + 2 c' dy) from the
        // exponent's products; d(natural exponent) / d(conic) = -(dx^2 / 2,
        // dx dy, dy^2 / 2)
        const float gu = hl * fmaf(2.f, bxdx, b.y * dy);
        const float gv = hl * fmaf(2.f, bzdy, bydx);
        const float tx = dpw * dx, ty = dpw * dy;
        const float ga = -0.5f * (tx * dx);
        const float gb = -(tx * dy);
        const float gc = -0.5f * (ty * dy);
        if (FULL) go = slope ? dal * hw_exp2(p - b.w) : 0.f;
        Sg = fmaf(gcv, wk, Sg);
        // a recorded entry has a contributing lane: the forward took it for
        // the same pixels by the same arithmetic
        if (recorded || __any_sync(FULLM, contrib)) {
          // reduce-scatter over the warp: every lane then holds the warp sum
          // of word `comp`, and one lane per word adds it with one atomic
          float *dst = s_dst[j];
          float sum;
          if constexpr (FULL) {
            const float v10[10] = {gu, gv, ga, gb, gc, gz, go, gr, gg, gbl};
            sum = warp_reduce_scatter<10>(v10, lane);
          } else {
            const float v6[6] = {gu, gv, ga, gb, gc, gz};
            sum = warp_reduce_scatter<6>(v6, lane);
          }
          if (writer) atomicAdd(dst + comp, sum);
        }
      }
    }
  }
  if (COUNT) add_eval_counts(ws, 1, n_eval, n_contrib);
  // the fixed-bucket layout's counts start at zero for the next preprocess
  // (the adjoint is the last reader of the tile's range)
  if (ws.bucket_cap && tid == 0) ws.tile_count[tile] = 0u;
}

// Chains the 2D gradients of the Gaussian projected as q in view slot `slot`
// (pose Pm) to the pose twist (pg, added) and, FULL, to the record's
// parameters (acc, added).
template <bool FULL>
__device__ __forceinline__ void chain_proj(const Workspace &ws, const Raster &r, const Proj &q, const float *Pm,
                                           size_t slot, float *pg, float *acc) {
  const float *gd = ws.grad2d + slot * kGradWords;
  const float4 ga4 = *reinterpret_cast<const float4 *>(gd);
  const float4 gb4 = *reinterpret_cast<const float4 *>(gd + 4);
  const float gu = ga4.x, gv = ga4.y, gA = ga4.z, gB = ga4.w, gC = gb4.x, gzz = gb4.y;
  // conic -> 2D covariance: dS = -Q Gq Q with Gq the symmetric-matrix form of
  // the conic gradient (the off-diagonal appears twice in the quadratic form)
  const float qa = q.ca, qb = q.cb, qc = q.cc;
  const float h = 0.5f * gB;
  const float t00 = qa * gA + qb * h, t01 = qa * h + qb * gC;
  const float t10 = qb * gA + qc * h, t11 = qb * h + qc * gC;
  const float d00 = -(t00 * qa + t01 * qb);
  const float d01 = -(t00 * qb + t01 * qc);
  const float d11 = -(t10 * qb + t11 * qc);
  // Sigma' = M2 M2^T + d I with M2 = J K: dM2 = 2 dS M2
  float dm0[3], dm1[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    dm0[s] = 2.f * (d00 * q.m0[s] + d01 * q.m1[s]);
    dm1[s] = 2.f * (d01 * q.m0[s] + d11 * q.m1[s]);
  }
  const float dj00 = dm0[0] * q.K[0] + dm0[1] * q.K[1] + dm0[2] * q.K[2];
  const float dj02 = dm0[0] * q.K[6] + dm0[1] * q.K[7] + dm0[2] * q.K[8];
  const float dj11 = dm1[0] * q.K[3] + dm1[1] * q.K[4] + dm1[2] * q.K[5];
  const float dj12 = dm1[0] * q.K[6] + dm1[1] * q.K[7] + dm1[2] * q.K[8];
  float dK[9];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    dK[s] = q.j00 * dm0[s];
    dK[3 + s] = q.j11 * dm1[s];
    dK[6 + s] = q.j02 * dm0[s] + q.j12 * dm1[s];
  }
  // camera-space mean
  const float z = q.z, iz = 1.f / z, iz2 = iz * iz;
  float dpx = gu * r.fx * iz;
  float dpy = gv * r.fy * iz;
  float dpz = -gu * r.fx * q.x * iz2 - gv * r.fy * q.y * iz2 + gzz;
  dpz += -dj00 * r.fx * iz2 - dj11 * r.fy * iz2;
  const bool clx = q.txz > r.limx || q.txz < -r.limx;
  const bool cly = q.tyz > r.limy || q.tyz < -r.limy;
  if (!clx) { dpx += -dj02 * r.fx * iz2; dpz += dj02 * 2.f * r.fx * q.x * iz2 * iz; }
  else { dpz += dj02 * r.fx * q.tx * iz2; }
  if (!cly) { dpy += -dj12 * r.fy * iz2; dpz += dj12 * 2.f * r.fy * q.y * iz2 * iz; }
  else { dpz += dj12 * r.fy * q.ty * iz2; }
  // pose twist (left perturbation): rho += dp, phi += p x dp + the covariance
  // term from K' = (I + [phi]x) K: B = K dK^T
  pg[0] += dpx; pg[1] += dpy; pg[2] += dpz;
  pg[3] += q.y * dpz - z * dpy;
  pg[4] += z * dpx - q.x * dpz;
  pg[5] += q.x * dpy - q.y * dpx;
  float Bm[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      Bm[3 * a + b] = q.K[3 * a] * dK[3 * b] + q.K[3 * a + 1] * dK[3 * b + 1] + q.K[3 * a + 2] * dK[3 * b + 2];
  pg[3] += Bm[5] - Bm[7];
  pg[4] += Bm[6] - Bm[2];
  pg[5] += Bm[1] - Bm[3];
  if (FULL) {
    const float4 gc4 = *reinterpret_cast<const float4 *>(gd + 8);
    const float go = gb4.z;
    acc[0] += Pm[0] * dpx + Pm[4] * dpy + Pm[8] * dpz;
    acc[1] += Pm[1] * dpx + Pm[5] * dpy + Pm[9] * dpz;
    acc[2] += Pm[2] * dpx + Pm[6] * dpy + Pm[10] * dpz;
    acc[3] += go * q.o * (1.f - q.o);
    // K = R M, M = Rq diag(S): dM = R^T dK
    float dRq[9];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      float dS = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float dM = Pm[a] * dK[s] + Pm[4 + a] * dK[3 + s] + Pm[8 + a] * dK[6 + s];
        dS += q.Rq[3 * a + s] * dM;
        dRq[3 * a + s] = dM * q.S[s];
      }
      acc[8 + s] += dS * q.S[s];
    }
    const float w = q.nq[0], x = q.nq[1], y = q.nq[2], zq = q.nq[3];
    const float dn0 = -2.f * zq * dRq[1] + 2.f * y * dRq[2] + 2.f * zq * dRq[3] - 2.f * x * dRq[5] -
                      2.f * y * dRq[6] + 2.f * x * dRq[7];
    const float dn1 = 2.f * y * dRq[1] + 2.f * zq * dRq[2] + 2.f * y * dRq[3] - 4.f * x * dRq[4] -
                      2.f * w * dRq[5] + 2.f * zq * dRq[6] + 2.f * w * dRq[7] - 4.f * x * dRq[8];
    const float dn2 = -4.f * y * dRq[0] + 2.f * x * dRq[1] + 2.f * w * dRq[2] + 2.f * x * dRq[3] +
                      2.f * zq * dRq[5] - 2.f * w * dRq[6] + 2.f * zq * dRq[7] - 4.f * y * dRq[8];
    const float dn3 = -4.f * zq * dRq[0] - 2.f * w * dRq[1] + 2.f * x * dRq[2] + 2.f * w * dRq[3] -
                      4.f * zq * dRq[4] + 2.f * y * dRq[5] + 2.f * x * dRq[6] + 2.f * y * dRq[7];
    const float ndn = w * dn0 + x * dn1 + y * dn2 + zq * dn3;
    const float iq = 1.f / q.qlen;
    acc[4] += (dn0 - w * ndn) * iq;
    acc[5] += (dn1 - x * ndn) * iq;
    acc[6] += (dn2 - y * ndn) * iq;
    acc[7] += (dn3 - zq * ndn) * iq;
    acc[12] += gb4.w;   // colour: slots G2_R, G2_G, G2_BL
    acc[13] += gc4.x;
    acc[14] += gc4.y;
  }
}

// Whether the Gaussian of view slot `slot` has a non-empty tile range, and if
// so its projection.
__device__ __forceinline__ bool visible_proj(const Workspace &ws, const Raster &r, const float4 &g0,
                                             const float4 &g1, const float4 &g2, const float *Pm, size_t slot,
                                             Proj &q) {
  const uint2 rc = ws.rect[slot];
  return (rc.x >> 16) > (rc.x & 0xFFFF) && project_gaussian(g0, g1, g2, Pm, r, q);
}

// chain_proj of Gaussian (g0, g1, g2) when it is visible.
template <bool FULL>
__device__ __forceinline__ void chain_one(const Workspace &ws, const Raster &r, const float4 &g0, const float4 &g1,
                                          const float4 &g2, const float *Pm, size_t slot, float *pg, float *acc) {
  Proj q;
  if (visible_proj(ws, r, g0, g1, g2, Pm, slot, q)) chain_proj<FULL>(ws, r, q, Pm, slot, pg, acc);
}

// Compensated (double-FP32) addition: (h, l) += (bh, bl) through two-sum,
// the high words' rounding error carried into the low word.
__device__ __forceinline__ void cadd(float &h, float &l, float bh, float bl) {
  float sh, se;
  two_sum(h, bh, sh, se);
  h = sh;
  l = __fadd_rn(__fadd_rn(l, bl), se);
}

// Sums pg[6] over the CTA in compensated FP32 (a fixed shuffle tree, then
// the warps in order) and stores the (high, low) partial of (view v, CTA b).
__device__ __forceinline__ void store_pose_partial(const Workspace &ws, float *pg, int v, int b, int nb,
                                                   float2 (*s_red)[6]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float h = pg[c], l = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      cadd(h, l, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, l, o));
    if (lane == 0) s_red[wid][c] = make_float2(h, l);
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float h = 0.f, l = 0.f;
    for (int w = 0; w < kBwdPrepBlock / 32; ++w) cadd(h, l, s_red[w][threadIdx.x].x, s_red[w][threadIdx.x].y);
    ws.pose_partial[((size_t)v * nb + b) * 6 + threadIdx.x] = make_float2(h, l);
  }
  __syncthreads();
}

// FULL: one thread per Gaussian, all views, parameter gradients written.
// !FULL (pose only): a fixed grid strides over the Gaussians of each view.
// The last CTA sums the pose partials in a fixed order in FP64 (one warp per
// twist component) and, if ps.poses is set, applies the pose step.
template <bool FULL>
__global__ void __launch_bounds__(kBwdPrepBlock)
preprocess_bwd_kernel(Workspace ws, const float4 *__restrict__ gauss, int64_t n, int views, Raster r,
                      float *__restrict__ grad_gauss, double *__restrict__ grad_pose, PoseStep ps) {
  // pose only, tracking loop: the grid's first CTA (dispatched first, so
  // that it runs beside the chain CTAs from the start) ranks the tiles by
  // this iteration's counts for the next iteration's render order; the
  // chain CTAs are numbered from the second
  const bool ordering = !FULL && ws.order_next != nullptr;
  if (ordering && blockIdx.x == 0) {
    pdl_wait();
    pdl_trigger();
    rank_tiles(ws.prev_count, r.T, ws.order_next, ws.band);
    return;
  }
  __shared__ float sp[kMaxViewsSmem * 12];
  __shared__ float2 s_red[kBwdPrepBlock / 32][6];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nb = gridDim.x - (ordering ? 1 : 0);
  const int bid = blockIdx.x - (ordering ? 1 : 0);
  // pose only, one view: the visible list, the records, their tile ranges
  // and the FP32 pose were written two or more launches before this one, so
  // each thread projects its first visible Gaussian before waiting for the
  // adjoint, whose 2D gradients it reads after the wait
  Proj q0;
  bool pre = false, pre_vis = false;
  // the pose step's bias corrections depend only on the Adam step count,
  // written by the previous iteration's step (three launches back): every
  // CTA forms them before its wait, and the last one uses its own
  __shared__ double s_presc[2];
  const bool presc = !FULL && views == 1 && ps.poses != nullptr;
  if (presc && (tid == 6 || tid == 7)) {
    const double k = __ldcg(ps.state + 12) + 1.0;
    s_presc[tid - 6] = tid == 6 ? adam_bias1(ps.cfg, k) : adam_bias2(ps.cfg, k);
  }
  int64_t pre_k = 0;
  size_t pre_slot = 0;
  if (!FULL && views == 1) {
    for (int k = tid; k < 12; k += blockDim.x) sp[k] = __ldcg(ws.pose32 + k);
    __syncthreads();
    pre = true;
    pre_k = (int64_t)bid * blockDim.x + tid;
    if (pre_k < (int64_t)__ldcg(ws.vis_n)) {
      const int64_t i = __ldcg(ws.vis_ids + pre_k);
      if (DAGS_IN_BOUNDS(i >= 0 && i < n, ws.counters + CNT_STATUS)) {
        pre_slot = (size_t)i;
        const float4 g0 = __ldg(gauss + 4 * i + 0), g1 = __ldg(gauss + 4 * i + 1), g2 = __ldg(gauss + 4 * i + 2);
        pre_vis = visible_proj(ws, r, g0, g1, g2, sp, pre_slot, q0);
      }
    }
  }
  pdl_wait();
  pdl_trigger();
  if (!pre) {
    for (int k = threadIdx.x; k < views * 12; k += blockDim.x) sp[k] = ws.pose32[k];
    __syncthreads();
  }
  if (FULL) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0, g2 = g0;
    if (i < n) {
      g0 = __ldg(gauss + 4 * i + 0);
      g1 = __ldg(gauss + 4 * i + 1);
      g2 = __ldg(gauss + 4 * i + 2);
    }
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.f;
    for (int v = 0; v < views; ++v) {
      float pg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (i < n) chain_one<true>(ws, r, g0, g1, g2, sp + v * 12, (size_t)v * ws.max_n + i, pg, acc);
      if (grad_pose) store_pose_partial(ws, pg, v, blockIdx.x, nb, s_red);
    }
    if (i < n) {
      float4 *out = reinterpret_cast<float4 *>(grad_gauss + 16 * i);
      out[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      out[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
      out[2] = make_float4(acc[8], acc[9], acc[10], 0.f);
      out[3] = make_float4(acc[12], acc[13], acc[14], 0.f);
    }
  } else {
    // pose only: the visible Gaussians of each view (the others have no
    // 2D gradient)
    for (int v = 0; v < views; ++v) {
      float pg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const int64_t nv = ws.vis_n[v];
      const uint32_t *vis = ws.vis_ids + (size_t)v * ws.max_n;
      for (int64_t k = (int64_t)bid * blockDim.x + tid; k < nv; k += (int64_t)nb * blockDim.x) {
        if (pre && k == pre_k) {
          if (pre_vis) chain_proj<false>(ws, r, q0, sp, pre_slot, pg, nullptr);
          continue;
        }
        int64_t i = vis[k];
        if (!DAGS_IN_BOUNDS(i >= 0 && i < n, ws.counters + CNT_STATUS)) continue;
        const float4 g0 = __ldg(gauss + 4 * i + 0), g1 = __ldg(gauss + 4 * i + 1), g2 = __ldg(gauss + 4 * i + 2);
        chain_one<false>(ws, r, g0, g1, g2, sp + v * 12, (size_t)v * ws.max_n + i, pg, nullptr);
      }
      store_pose_partial(ws, pg, v, bid, nb, s_red);
    }
  }
  if (!grad_pose) return;
  // last CTA: barrier, then one thread's fence and counter increment
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned t = atomicAdd(ws.counters + CNT_DONE_BWDPREP, 1u);
    s_last = (t == (unsigned)nb - 1u);
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  // the CTA partials of each view, summed by every thread of the last CTA:
  // thread t takes CTAs t, t + 128, ... (all loads of a round issued before
  // they are added), each component in compensated FP32 in a fixed order,
  // then a fixed shuffle tree and the warps in order; the result is the
  // FP64 sum of the high and low words
  for (int v = 0; v < views; ++v) {
    const float2 *src = ws.pose_partial + (size_t)v * nb * 6;
    float h[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, l[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int b0 = tid; b0 < nb; b0 += kBwdPrepBlock * 4) {
      float2 t[4][6];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + kBwdPrepBlock * u;
#pragma unroll
        for (int c = 0; c < 6; ++c) t[u][c] = b < nb ? __ldcg(src + (size_t)b * 6 + c) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 6; ++c) cadd(h[c], l[c], t[u][c].x, t[u][c].y);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        cadd(h[c], l[c], __shfl_xor_sync(0xffffffffu, h[c], o), __shfl_xor_sync(0xffffffffu, l[c], o));
      if (lane == 0) s_red[wid][c] = make_float2(h[c], l[c]);
    }
    __syncthreads();
    if (tid < 6) {
      float hh = 0.f, ll = 0.f;
      for (int w = 0; w < kBwdPrepBlock / 32; ++w) cadd(hh, ll, s_red[w][tid].x, s_red[w][tid].y);
      grad_pose[v * 6 + tid] = (double)hh + (double)ll;
    }
    __syncthreads();
  }
  if (tid == 0) ws.counters[CNT_DONE_BWDPREP] = 0u;
  if (ps.poses) {
    __shared__ double s_xi[6], s_sc[3];
    for (int v = 0; v < views; ++v)
      pose_adam_exp_cta(ps.poses + 12 * v, grad_pose + 6 * v, ps.state + 13 * v, ps.cfg, s_xi, s_sc,
                        presc ? s_presc : nullptr);
    // the tracking loop: if the new pose (as the preprocess stages it in
    // FP32) has left the bounds the candidates were culled for, move the
    // culling pose to it and empty the list; the next preprocess then takes
    // every Gaussian once and re-culls
    if (ordering && ws.cand_n && ws.cull_pose) {
      __shared__ float s_np[12];
      __shared__ int s_out;
      __syncthreads();
      if (tid < 12) s_np[tid] = __double2float_rn(ps.poses[tid]);
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

}  // namespace

cudaError_t launch_render_bwd(const Workspace &ws, int views, int64_t n, const Raster &r, const Loss &l,
                              const float4 *targets, const float *image, const int32_t *last, bool full,
                              cudaStream_t s, const float *upstream) {
  (void)n;
  const dim3 grid((unsigned)(views * r.T));
  const bool masks = ws.warp_masks != nullptr, count = ws.count_evals != 0;
#define DAGS_BWD(F, M, C) \
  launch_pdl(render_bwd_kernel<F, M, C>, grid, dim3(kTilePix), 0, s, ws, r, l, targets, image, last, upstream)
  if (full) return count ? DAGS_BWD(true, false, true) : DAGS_BWD(true, false, false);
  if (masks) return count ? DAGS_BWD(false, true, true) : DAGS_BWD(false, true, false);
  return count ? DAGS_BWD(false, false, true) : DAGS_BWD(false, false, false);
#undef DAGS_BWD
}

cudaError_t launch_preprocess_bwd(const Workspace &ws, const float4 *gauss, int64_t n, int views,
                                  const Raster &r, float *grad_gauss, double *grad_pose, const PoseStep &ps,
                                  cudaStream_t s) {
  if (views > kMaxViewsSmem) return cudaErrorInvalidValue;
  const unsigned gx = (unsigned)((n + kBwdPrepBlock - 1) / kBwdPrepBlock);
  unsigned grid = gx > 0 ? gx : 1u;
  if (grad_gauss) {
    return launch_pdl(preprocess_bwd_kernel<true>, dim3(grid), dim3(kBwdPrepBlock), 0, s, ws, gauss, n, views, r,
                      grad_gauss, grad_pose, ps);
  } else {
    // pose only: a fixed grid of 4 CTAs per SM (one wave) strides over the
    // visible Gaussians (at most one per thread at the tracking size); the
    // tracking loop adds one CTA that ranks the tiles for the next
    // iteration's render order
    const unsigned cap = (unsigned)(4 * (ws.band > 0 ? ws.band : 1));
    if (grid > cap) grid = cap;
    if (ws.order_next) grid += 1;
    return launch_pdl(preprocess_bwd_kernel<false>, dim3(grid), dim3(kBwdPrepBlock), 0, s, ws, gauss, n, views, r,
                      grad_gauss, grad_pose, ps);
  }
  return cudaGetLastError();
}

}  // namespace dags
