// Fused forward and pose-only adjoint of one tracking iteration (sm_103a).
//
//   render_track_kernel   one CTA per 16x16 tile (launched longest list
//                         first), one warp per 8x4 pixel block. The CTA sorts
//                         its bucket as the forward render does, composites
//                         front to back (Eq. (20)), forms the static weight
//                         and the MP-weighted L1 loss of Eqs. (21), (22) and
//                         the loss's upstream gradients per pixel, writes the
//                         image, and then walks the same list back to front
//                         for the adjoint, with every pixel's forward state
//                         (final transmittance, last contributor, upstream
//                         gradients) still in registers. While compositing,
//                         each warp records which list entries at least one
//                         of its pixels took (one bit per entry); the adjoint
//                         visits only those. A list that fits one staging
//                         batch is not staged again for the adjoint. The
//                         per-Gaussian 2D gradients of the pose path (centre,
//                         conic, depth) are summed over each warp with a
//                         reduce-scatter and added with one atomic per word;
//                         the last CTA sums the loss in FP64.
#include "common.cuh"
#include "tile_sort.cuh"

namespace dags {

namespace {

constexpr int kMaskGroups = 32;   // entries with a recorded contribution mask: 32 groups of 32 (1024)

__global__ void __launch_bounds__(kTilePix, 5)
render_track_kernel(Workspace ws, Raster r, Loss l, const float4 *__restrict__ targets, float *__restrict__ image,
                    int32_t *__restrict__ last, double *__restrict__ loss) {
  pdl_wait();
  __shared__ uint64_t s_key[kSortSmallCap];
  __shared__ float4 s_a[kTilePix], s_b[kTilePix], s_c[kTilePix];   // s_a: {u hi, v hi, u lo, v lo}
  __shared__ float2 s_e[kTilePix];                                  // box half extents
  __shared__ uint32_t s_id[kTilePix];
  __shared__ uint32_t s_cm[kTilePix / 32][kMaskGroups];             // per warp: entries it took
  __shared__ double s_red[kTilePix / 32];
  __shared__ int s_max, s_last;
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool ovf = pairs_overflow_ws(ws);
  const int tile = ovf ? (int)blockIdx.x : (int)ws.tile_order[blockIdx.x];
  const int tx = tile % r.tiles_x, ty = tile / r.tiles_x;
  const int bx0 = tx * kTile + (warp & 1) * 8, by0 = ty * kTile + (warp >> 1) * 4;
  const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
  const bool inside = px < r.W && py < r.H;
  uint32_t s = 0u, e = 0u;
  if (!ovf) tile_range(ws, tile, s, e);
  const float bcx = (float)bx0 + 3.5f, bcy = (float)by0 + 1.5f;
  const float fpx = (float)px, fpy = (float)py;
  // the pose-only adjoint's reduce-scatter leaves word `comp` of the six
  // 2D-gradient words in this lane; the lowest lane holding it adds it
  const int comp = rs_component<6>(lane);
  const bool writer = __ffs(__match_any_sync(FULL, (unsigned)comp)) - 1 == lane;

  // the order stays in shared memory for lists that fit (both passes read it
  // there); longer lists are merged through sorted_ids
  const bool own_sort = sort_tile_bucket(ws, s, (int)(e - s), s_key, false);
  for (int k = tid; k < (kTilePix / 32) * kMaskGroups; k += kTilePix) (&s_cm[0][0])[k] = 0u;

  // stages list entries [base, base + cnt) of the tile (called by the CTA)
  auto stage = [&](uint32_t base, int cnt) {
    if (tid < cnt) {
      const uint32_t k = base + tid;
      uint32_t id = own_sort ? (uint32_t)s_key[k - s] : ws.sorted_ids[k];
      if (!DAGS_IN_BOUNDS(id < (uint32_t)ws.max_n && k < (uint64_t)ws.max_pairs, ws.counters + CNT_STATUS)) id = 0;
      const float4 r0 = ws.rec2d[(size_t)id * 3 + 0];
      const float2 lo = ws.rec_lo[id];
      s_id[tid] = id;
      s_a[tid] = make_float4(r0.x, r0.y, lo.x, lo.y);
      s_e[tid] = make_float2(r0.z, r0.w);
      s_b[tid] = ws.rec2d[(size_t)id * 3 + 1];
      s_c[tid] = ws.rec2d[(size_t)id * 3 + 2];
    }
  };

  // ---- forward: front-to-back compositing ----
  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f, oo = 0.f, rm = 0.f;
  int lastk = 0;
  unsigned n_eval = 0, n_contrib = 0;
  bool done = !inside;
  uint32_t staged = 0xFFFFFFFFu;       // base (list offset) of the batch in shared memory
  for (uint32_t base = s; base < e; base += kTilePix) {
    if (__syncthreads_count(!done) == 0) break;
    const int cnt = (int)min((uint32_t)kTilePix, e - base);
    stage(base, cnt);
    staged = base - s;
    __syncthreads();
    if (__all_sync(FULL, done)) continue;
    for (int g = 0; g < 8 && g * 32 < cnt; ++g) {
      const int jj = g * 32 + lane;
      bool hit = false;
      if (jj < cnt) {
        const float4 a = s_a[jj];
        const float2 ex = s_e[jj];
        hit = fabsf(a.x - bcx) <= ex.x + 3.5f && fabsf(a.y - bcy) <= ex.y + 1.5f;
      }
      unsigned mask = __ballot_sync(FULL, hit);
      unsigned took = 0u;
      while (mask) {
        const int bit = __ffs(mask) - 1;
        const int j = g * 32 + bit;
        mask &= mask - 1;
        bool contrib = false;
        if (!done) {
          const float4 a = s_a[j], b = s_b[j];
          const float dx = (a.x - fpx) + a.z, dy = (a.y - fpy) + a.w;
          const float p = fmaf(b.x * dx, dx, fmaf(b.y * dx, dy, fmaf(b.z * dy, dy, b.w)));
          ++n_eval;
          if (p >= r.log2_alpha_min) {
            const float alpha = fminf(r.alpha_max, hw_exp2(p));
            const float tt = T * (1.f - alpha);
            if (tt < r.t_min) {
              done = true;
            } else {
              contrib = true;
              ++n_contrib;
              const float w = alpha * T;
              const float4 c = s_c[j];
              const uint32_t rg = __float_as_uint(c.z), bl = __float_as_uint(c.w);
              cr += bf16_lo(rg) * w; cg += bf16_hi(rg) * w; cb += bf16_lo(bl) * w;
              dd += c.x * w; oo += w; rm += c.y * w;
              T = tt;
              lastk = (int)(base - s) + j + 1;
            }
          }
        }
        if (__any_sync(FULL, contrib)) took |= 1u << bit;
      }
      const int gk = (int)((base - s) >> 5) + g;
      if (lane == 0 && gk < kMaskGroups) s_cm[warp][gk] = took;
      if (__all_sync(FULL, done)) break;
    }
  }

  // ---- epilogue: image, loss, the loss's upstream gradients ----
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f, g5 = 0.f;
  int lastp = 0;
  float lpx = 0.f;
  if (inside) {
    const size_t P = (size_t)r.W * r.H;
    const size_t pix = (size_t)py * r.W + px;
    const float wgt = l.weight_mode == 0 ? (oo > l.o_eps ? (oo - rm) / oo : 0.f) : oo - rm;
    const float4 tg = targets[pix];
    const float rc0 = cr - tg.x, rc1 = cg - tg.y, rc2 = cb - tg.z, rd = dd - tg.w;
    const bool dvalid = tg.w > 0.f;
    const float l1 = fabsf(rc0) + fabsf(rc1) + fabsf(rc2);
    const float ld = dvalid ? fabsf(rd) : 0.f;
    // a target with negative red is a pixel outside the loss
    if (tg.x >= 0.f) {
      lpx = wgt * (l.lambda_pho * l1 + l.lambda_depth * ld);
      lastp = lastk;
      auto sgn = [](float x) { return (float)((x > 0.f) - (x < 0.f)); };
      g0 = l.lambda_pho * wgt * sgn(rc0);
      g1 = l.lambda_pho * wgt * sgn(rc1);
      g2 = l.lambda_pho * wgt * sgn(rc2);
      g3 = dvalid ? l.lambda_depth * wgt * sgn(rd) : 0.f;
      if (l.weight_grad) {
        const float lw = l.lambda_pho * l1 + l.lambda_depth * ld;
        if (l.weight_mode == 0) {
          if (oo > l.o_eps) { g4 = lw * rm / (oo * oo); g5 = -lw / oo; }
        } else {
          g4 = lw;
          g5 = -lw;
        }
      }
    }
    float *img = image + pix;
    img[0 * P] = cr; img[1 * P] = cg; img[2 * P] = cb; img[3 * P] = dd;
    img[4 * P] = oo; img[5 * P] = rm; img[6 * P] = T; img[7 * P] = wgt;
    last[pix] = lastk;
  }
  // the tile's loss in FP64, then the frame's by the last CTA (below)
  {
    const double lsum = warp_sum_d((double)lpx);
    if (lane == 0) s_red[warp] = lsum;
  }
  if (tid == 0) s_max = 0;
  __syncthreads();
  const int wmax = (int)__reduce_max_sync(FULL, (unsigned)lastp);
  if (lane == 0) atomicMax(&s_max, wmax);
  __syncthreads();
  const int kmax = s_max;

  // ---- adjoint: back to front from each pixel's last contributor ----
  float Sg = 0.f;
  unsigned b_eval = 0, b_contrib = 0;
  for (int end = kmax; end > 0;) {
    const int beg = ((end - 1) / kTilePix) * kTilePix;   // batches aligned as in the forward
    const int cnt = min(kTilePix, (int)(e - s) - beg);
    if ((uint32_t)beg != staged) {
      __syncthreads();
      stage(s + (uint32_t)beg, cnt);
      staged = (uint32_t)beg;
      __syncthreads();
    }
    if (wmax > beg) {
      const int top = min(end, wmax) - beg;             // entries [beg, beg + top) may matter to this warp
      for (int g = (top - 1) >> 5; g >= 0; --g) {
        const int gk = (beg >> 5) + g;
        unsigned mask;
        if (gk < kMaskGroups) {
          mask = s_cm[warp][gk];
        } else {
          const int jj = g * 32 + lane;
          bool hit = false;
          if (jj < cnt) {
            const float4 a = s_a[jj];
            const float2 ex = s_e[jj];
            hit = fabsf(a.x - bcx) <= ex.x + 3.5f && fabsf(a.y - bcy) <= ex.y + 1.5f;
          }
          mask = __ballot_sync(FULL, hit);
        }
        const int lim = top - g * 32;
        if (lim < 32) mask &= (1u << lim) - 1u;
        while (mask) {
          const int bit = 31 - __clz(mask);
          mask &= ~(1u << bit);
          const int j = g * 32 + bit;
          const int k = beg + j;
          bool contrib = false;
          float gu = 0.f, gv = 0.f, ga = 0.f, gb = 0.f, gc = 0.f, gz = 0.f;
          if (k < lastp) {
            const float4 a = s_a[j], b = s_b[j];
            const float dx = (a.x - fpx) + a.z, dy = (a.y - fpy) + a.w;
            const float p = fmaf(b.x * dx, dx, fmaf(b.y * dx, dy, fmaf(b.z * dy, dy, b.w)));
            ++b_eval;
            if (p >= r.log2_alpha_min) {
              contrib = true;
              ++b_contrib;
              const float ag = hw_exp2(p);
              const float alpha = fminf(r.alpha_max, ag);
              const float inv = hw_rcp(1.f - alpha);
              T *= inv;                       // transmittance in front of this Gaussian
              const float wk = alpha * T;
              const float4 c = s_c[j];
              const uint32_t rgb = __float_as_uint(c.z), blb = __float_as_uint(c.w);
              const float fr = bf16_lo(rgb), fg = bf16_hi(rgb), fb = bf16_lo(blb);
              // dL/dalpha = sum_ch g_ch (c_ch T - S_ch / (1 - alpha)), with
              // Sg the contracted suffix sum
              const float gcv = fmaf(g0, fr, fmaf(g1, fg, fmaf(g2, fb, fmaf(g3, c.x, fmaf(g5, c.y, g4)))));
              const float dal = fmaf(gcv, T, -Sg * inv);
              gz = g3 * wk;
              if (ag <= r.alpha_max) {
                const float dpw = dal * alpha;
                const float hl = dpw * kLn2;
                gu = hl * (2.f * b.x * dx + b.y * dy);
                gv = hl * (b.y * dx + 2.f * b.z * dy);
                ga = -0.5f * dpw * dx * dx;
                gb = -dpw * dx * dy;
                gc = -0.5f * dpw * dy * dy;
              }
              Sg = fmaf(gcv, wk, Sg);
            }
          }
          if (__any_sync(FULL, contrib)) {
            const float v6[6] = {gu, gv, ga, gb, gc, gz};
            const float sum = warp_reduce_scatter<6>(v6, lane);
            if (writer) atomicAdd(ws.grad2d + (size_t)s_id[j] * kGradWords + comp, sum);
          }
        }
      }
    }
    end = beg;
  }
  add_eval_counts(ws, 0, n_eval, n_contrib);
  add_eval_counts(ws, 1, b_eval, b_contrib);
  // the fixed-bucket layout's counts start at zero for the next preprocess
  if (ws.bucket_cap && tid == 0) ws.tile_count[tile] = 0u;

  if (!loss) return;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kTilePix / 32; ++w) t += s_red[w];
    ws.loss_partial[tile] = t;
    __threadfence();
    const unsigned done_ctas = atomicAdd(ws.counters + CNT_DONE_RENDER, 1u);
    s_last = (done_ctas == gridDim.x - 1);
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  // deterministic FP64 sum of the per-tile partials: fixed strided
  // assignment, then a fixed tree
  __shared__ double s_d[kTilePix];
  double acc = 0.0;
  for (int k = tid; k < r.T; k += kTilePix) acc += __ldcg(ws.loss_partial + k);
  s_d[tid] = acc;
  __syncthreads();
  for (int o = kTilePix / 2; o > 0; o >>= 1) {
    if (tid < o) s_d[tid] += s_d[tid + o];
    __syncthreads();
  }
  if (tid == 0) {
    *loss = ovf ? 0.0 : s_d[0];
    ws.counters[CNT_DONE_RENDER] = 0u;
  }
}

}  // namespace

cudaError_t launch_render_track(const Workspace &ws, const Raster &r, const Loss &l, const float4 *targets,
                                float *image, int32_t *last, double *loss, cudaStream_t s) {
  return launch_pdl(render_track_kernel, dim3((unsigned)r.T), dim3(kTilePix), 0, s, ws, r, l, targets, image, last,
                    loss);
}

}  // namespace dags
