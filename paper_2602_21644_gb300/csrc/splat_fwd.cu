// Forward half of the MP-aware splatting path (sm_103a).
//
//   preprocess_kernel   per (view, Gaussian): camera transform, EWA 2D
//                       covariance, conic, opacity, the bounding box of the
//                       alpha >= alpha_min ellipse; each warp then walks the
//                       candidate tiles of its 32 Gaussians together, keeps
//                       the tiles the ellipse reaches and counts them per tile
//                       with one atomic per distinct tile per warp; the last
//                       CTA scans the counts into tile offsets.
//   emit_kernel         the same warp-cooperative walk, writing (depth bits
//                       << 32 | id) keys into per-tile buckets (order inside a
//                       bucket is arbitrary).
//   render_fwd_kernel   one CTA per 16x16 tile (launched longest list first),
//                       one warp per 8x4 pixel block: the CTA first sorts its
//                       tile's bucket (bitonic in shared memory; long buckets
//                       in 1024-key chunks merged through global memory) and
//                       writes the depth-ordered ids for the backward; the
//                       list is then staged through shared memory
//                       in batches of 256; each warp keeps (by ballot) only the
//                       entries whose ellipse box meets its block, tests alpha
//                       in the exponent before exponentiating, and leaves when
//                       all its pixels are saturated (the CTA when all warps
//                       are); front-to-back compositing of colour, depth,
//                       opacity and MP, and the static weight and MP-weighted
//                       L1 loss of Eqs. (20)-(22) in the epilogue; the last
//                       CTA sums the loss in FP64.
#include "common.cuh"
#include "tile_sort.cuh"

namespace dags {

namespace {

constexpr int kMaxViewsSmem = 64;  // poses staged in shared memory per CTA

__device__ __forceinline__ int clampi(float x, int lo, int hi) {
  // x may be huge or non-finite; clamp in float before converting
  float c = fminf(fmaxf(x, (float)lo), (float)hi);
  return c != c ? lo : (int)c;
}

// Exclusive scan of `total` uint32 per-tile counts by one CTA, through a
// shared-memory stage of kScanChunk counts (coalesced loads, then each thread
// scans a contiguous slice and the slice sums are scanned across the CTA).
// Also clears the counts and cursors for the next call, and writes order[]:
// the launch order of the renders. Tiles are ranked by descending list
// length (bins of 8 entries; empty tiles last), and each band of `band`
// consecutive ranks (one CTA per SM in a dispatch round) is reversed every
// other band, so that the SM that receives a band's longest tile receives the
// next band's shortest one. Returns the sum.
constexpr int kScanChunk = 4096;

__device__ uint64_t block_scan_tiles(uint32_t *count, uint32_t *start, uint32_t *cursor, int total,
                                     uint32_t *order, int band) {
  __shared__ uint32_t s_c[kScanChunk];
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long s_carry;
  __shared__ uint32_t s_bin[kLenBins];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int k = tid; k < kLenBins; k += blockDim.x) s_bin[k] = 0u;
  if (tid == 0) s_carry = 0ull;
  __syncthreads();
  // pass 1: length bins
  for (int c0 = 0; c0 < total; c0 += kScanChunk) {
    const int n = min(kScanChunk, total - c0);
    for (int k0 = 0; k0 < n; k0 += blockDim.x) {
      const int k = k0 + tid;
      int bin = 1024 + lane;   // no element: a key of its own
      if (k < n) {
        const uint32_t c = __ldcg(count + c0 + k);
        s_c[k] = c;
        bin = length_bin(c);
      }
      const unsigned grp = __match_any_sync(0xffffffffu, bin);
      if (bin < kLenBins && lane == __ffs(grp) - 1) atomicAdd(&s_bin[bin], (uint32_t)__popc(grp));
    }
    __syncthreads();
  }
  if (wid == 0) {
    // exclusive prefix over the bins (ascending bin = descending length):
    // lane l takes the bins [9 l, 9 l + 9)
    uint32_t loc[9], sum = 0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const int bb = 9 * lane + j;
      loc[j] = bb < kLenBins ? s_bin[bb] : 0u;
      sum += loc[j];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    uint32_t run = inc - sum;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const int bb = 9 * lane + j;
      if (bb < kLenBins) s_bin[bb] = run;
      run += loc[j];
    }
  }
  __syncthreads();
  // pass 2: offsets, order, clearing
  for (int c0 = 0; c0 < total; c0 += kScanChunk) {
    const int n = min(kScanChunk, total - c0);
    if (total > kScanChunk) {
      for (int k = tid; k < n; k += blockDim.x) s_c[k] = __ldcg(count + c0 + k);
      __syncthreads();
    }
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = min(n, tid * per), e = min(n, b + per);
    unsigned long long mine = 0;
    for (int k = b; k < e; ++k) mine += s_c[k];
    unsigned long long inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      unsigned long long t = lane < nw ? warp_tot[lane] : 0ull;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    unsigned long long run = s_carry + (wid > 0 ? warp_tot[wid - 1] : 0ull) + inc - mine;
    for (int j = 0; j < per; ++j) {
      const int k = b + j;
      int bin = 1024 + lane;   // no element: a key of its own
      if (k < e) {
        const uint32_t c = s_c[k];
        start[c0 + k] = (uint32_t)(run > 0xFFFFFFFFull ? 0xFFFFFFFFull : run);
        run += c;
        bin = length_bin(c);
      }
      // rank in the length order: one shared atomic per distinct bin per warp
      const unsigned grp = __match_any_sync(0xffffffffu, bin);
      const int leader = __ffs(grp) - 1;
      uint32_t pos = 0;
      if (bin < kLenBins && lane == leader) pos = atomicAdd(&s_bin[bin], (uint32_t)__popc(grp));
      pos = __shfl_sync(0xffffffffu, pos, leader) + (uint32_t)__popc(grp & ((1u << lane) - 1u));
      if (k < e) order[snake_slot(pos, (uint32_t)total, (uint32_t)band)] = (uint32_t)(c0 + k);
    }
    for (int k = tid; k < n; k += blockDim.x) {
      count[c0 + k] = 0u;
      cursor[c0 + k] = 0u;
    }
    __syncthreads();
    if (tid == 0) s_carry += warp_tot[nw - 1];
    __syncthreads();
  }
  return s_carry;
}

// The 32 lanes of a warp walk the candidate tiles of their 32 Gaussians
// together: lane l takes candidate c = base + l of the warp's concatenated
// candidate lists, finds its owner by binary search over the warp's
// inclusive prefix of candidate counts, and tests whether the owner's
// ellipse reaches that tile. MODE kWalkCount: the kept pairs are counted per
// tile (one atomic per distinct tile per warp); kWalkEmit: each kept pair
// gets a slot in its tile's bucket (after the offsets scan) the same way and
// its key is written; kWalkDirect: each kept pair's slot comes from the
// tile's count itself and its key goes to the tile's fixed-capacity bucket
// (slots beyond the capacity are counted, not written).
enum { kWalkCount = 0, kWalkEmit = 1, kWalkDirect = 2 };
template <int MODE>
__device__ __forceinline__ void walk_tiles(const Workspace &ws, const Raster &r, int v, uint32_t id, uint2 rect,
                                           float4 r0, float4 r1, float zkey) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int x0 = rect.x & 0xFFFF, x1 = rect.x >> 16, y0 = rect.y & 0xFFFF, y1 = rect.y >> 16;
  const int cw = x1 - x0;
  const int m = (x1 > x0 && y1 > y0) ? cw * (y1 - y0) : 0;
  int incl = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(FULL, incl, 31);
  const float thr = r1.w - r.log2_alpha_min;
  const int vbase = v * r.T;
  for (int base = 0; base < total; base += 32) {
    const int c = base + lane;
    int owner = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int cand = owner + step;
      if (__shfl_sync(FULL, incl, cand - 1) <= c) owner = cand;
    }
    owner = min(owner, 31);
    const int o_incl = __shfl_sync(FULL, incl, owner);
    const int o_m = __shfl_sync(FULL, m, owner);
    const int o_x0 = __shfl_sync(FULL, x0, owner), o_y0 = __shfl_sync(FULL, y0, owner);
    const int o_cw = __shfl_sync(FULL, cw, owner);
    const float u = __shfl_sync(FULL, r0.x, owner), vv = __shfl_sync(FULL, r0.y, owner);
    const float A2 = -__shfl_sync(FULL, r1.x, owner), B2 = -__shfl_sync(FULL, r1.y, owner);
    const float C2 = -__shfl_sync(FULL, r1.z, owner), th = __shfl_sync(FULL, thr, owner);
    const uint32_t o_id = __shfl_sync(FULL, id, owner);
    const float o_z = __shfl_sync(FULL, zkey, owner);
    bool keep = false;
    uint32_t key = 0xFFFFFFFFu;
    if (c < total) {
      const int k = c - (o_incl - o_m);
      const int tx = o_x0 + k % o_cw, ty = o_y0 + k / o_cw;
      const float px0 = (float)(tx * kTile), py0 = (float)(ty * kTile);
      const float px1 = (float)min(tx * kTile + kTile - 1, r.W - 1);
      const float py1 = (float)min(ty * kTile + kTile - 1, r.H - 1);
      keep = ellipse_reaches_rect(u, vv, A2, B2, C2, th, px0, px1, py0, py1);
      if (keep) key = (uint32_t)(vbase + ty * r.tiles_x + tx);
    }
    const unsigned grp = __match_any_sync(FULL, key);
    const int leader = __ffs(grp) - 1;
    if (MODE == kWalkCount) {
      if (keep && lane == leader) atomicAdd(ws.tile_count + key, (uint32_t)__popc(grp));
    } else if (MODE == kWalkDirect) {
      uint32_t basepos = 0;
      if (keep && lane == leader) basepos = atomicAdd(ws.tile_count + key, (uint32_t)__popc(grp));
      basepos = __shfl_sync(FULL, basepos, leader);
      if (keep) {
        const uint32_t slot = basepos + (uint32_t)__popc(grp & ((1u << lane) - 1u));
        if (slot < ws.bucket_cap)
          ws.keys[(size_t)key * ws.bucket_cap + slot] = ((uint64_t)__float_as_uint(o_z) << 32) | (uint64_t)o_id;
      }
    } else {
      // the bucket bounds are loaded before the cursor atomic so that the
      // two round trips overlap
      uint32_t t0 = 0, t1 = 0;
      if (keep) { t0 = ws.tile_start[key]; t1 = ws.tile_start[key + 1]; }
      uint32_t basepos = 0;
      if (keep && lane == leader) basepos = atomicAdd(ws.tile_cursor + key, (uint32_t)__popc(grp));
      basepos = __shfl_sync(FULL, basepos, leader);
      if (keep) {
        const uint32_t dst = t0 + basepos + (uint32_t)__popc(grp & ((1u << lane) - 1u));
        if (dst < t1) ws.keys[dst] = ((uint64_t)__float_as_uint(o_z) << 32) | (uint64_t)o_id;
      }
    }
  }
}

// Projection of Gaussian i (valid: i < n, else an empty lane) into view v:
// the projected record, its FP32 remainders, the candidate tiles and the
// zeroed 2D gradient of a visible Gaussian, its visible-list entry and the
// warp-cooperative walk over its tiles (counting, or emitting into the
// fixed-capacity buckets). Called by whole warps (ballot, walk).
struct Rec {
  float4 g0, g1, g2, g3;
};

__device__ __forceinline__ Rec load_rec(const float4 *__restrict__ gauss, int64_t i, bool valid) {
  Rec a;
  a.g0 = a.g1 = a.g2 = a.g3 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    a.g0 = __ldg(gauss + 4 * i + 0);
    a.g1 = __ldg(gauss + 4 * i + 1);
    a.g2 = __ldg(gauss + 4 * i + 2);
    a.g3 = __ldg(gauss + 4 * i + 3);
  }
  return a;
}

template <bool DIRECT>
__device__ __forceinline__ void preprocess_one(const Workspace &ws, const Rec &rec, int64_t i, bool valid, int v,
                                               const float *sp, const float *spl, const Raster &r, int zero_words) {
  const float4 &g0 = rec.g0, &g1 = rec.g1, &g2 = rec.g2, &g3 = rec.g3;
  uint2 my_rect = make_uint2(0u, 0u);
  float4 my_r0 = make_float4(0.f, 0.f, 0.f, 0.f), my_r1 = my_r0;
  float my_z = 0.f;
  if (valid) {
    const float *P = sp + v * 12;
    const size_t slot = (size_t)v * ws.max_n + i;

    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0, o2 = o0;
    float2 ulo = make_float2(0.f, 0.f);
    uint2 rect = make_uint2(0u, 0u);
    Proj q;
    if (project_gaussian(g0, g1, g2, P, r, q)) {
      // the centre from the FP64 pose in double-FP32 arithmetic (a few
      // 2^-44 relative), split into FP32 hi + lo
      {
        const float *Ph = sp + v * 12, *Pl = spl + v * 12;
        float xh, xl, yh, yl, zh, zl;
        df_row(Ph, Pl, Ph[3], Pl[3], g0.x, g0.y, g0.z, xh, xl);
        df_row(Ph + 4, Pl + 4, Ph[7], Pl[7], g0.x, g0.y, g0.z, yh, yl);
        df_row(Ph + 8, Pl + 8, Ph[11], Pl[11], g0.x, g0.y, g0.z, zh, zl);
        df_project(xh, xl, zh, zl, r.fx, r.cx, q.u, ulo.x);
        df_project(yh, yl, zh, zl, r.fy, r.cy, q.v, ulo.y);
      }
      const float lo = log2f(q.o);
      const float thr = lo - r.log2_alpha_min;             // ellipse: Q(d) <= thr
      const float cnat = 2.f * kLn2 * thr;                 // 2 ln(o / alpha_min)
      const float ex = sqrtf(cnat * q.A), ey = sqrtf(cnat * q.C);
      const float inv_tile = 1.f / (float)kTile;
      const int x0 = clampi(floorf((q.u - ex) * inv_tile), 0, r.tiles_x);
      const int y0 = clampi(floorf((q.v - ey) * inv_tile), 0, r.tiles_y);
      const int x1 = clampi(floorf((q.u + ex) * inv_tile) + 1.f, 0, r.tiles_x);
      const int y1 = clampi(floorf((q.v + ey) * inv_tile) + 1.f, 0, r.tiles_y);
      if (thr > 0.f && x1 > x0 && y1 > y0 && isfinite(q.u) && isfinite(q.v)) {
        o0 = make_float4(q.u, q.v, ex, ey);
        o1 = make_float4(-0.5f * kLog2e * q.ca, -kLog2e * q.cb, -0.5f * kLog2e * q.cc, lo);
        o2 = make_float4(q.z, g2.w, g3.x, g3.y);
        rect = make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16));
      }
    }
    // invisible Gaussians only need their empty rect: nothing reads their
    // projected record or 2D gradient
    if ((rect.x >> 16) > (rect.x & 0xFFFF)) {
      ws.rec2d[slot * 3 + 0] = o0;
      ws.rec2d[slot * 3 + 1] = o1;
      ws.rec2d[slot * 3 + 2] = o2;
      ws.rec_lo[slot] = ulo;
      float4 *gz = reinterpret_cast<float4 *>(ws.grad2d + slot * kGradWords);
      for (int w = 0; w < zero_words / 4; ++w) gz[w] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    ws.rect[slot] = rect;
    my_rect = rect;
    my_r0 = o0;
    my_r1 = o1;
    my_z = o2.x;
  }
  // Visible Gaussians (non-empty candidate range) are appended to the view's
  // list, one atomic per warp.
  {
    const bool visible = (my_rect.x >> 16) > (my_rect.x & 0xFFFF);
    const unsigned ball = __ballot_sync(0xffffffffu, visible);
    const int lane = threadIdx.x & 31;
    uint32_t basev = 0;
    if (ball && lane == __ffs(ball) - 1) basev = atomicAdd(ws.vis_append + v, (uint32_t)__popc(ball));
    basev = __shfl_sync(0xffffffffu, basev, ball ? __ffs(ball) - 1 : 0);
    if (visible)
      ws.vis_ids[(size_t)v * ws.max_n + basev + __popc(ball & ((1u << lane) - 1u))] = (uint32_t)i;
  }
  // Warp-cooperative walk over the candidate tiles of the warp's Gaussians.
  const uint32_t id = (uint32_t)(valid ? i : 0);
  if (DIRECT) walk_tiles<kWalkDirect>(ws, r, v, id, my_rect, my_r0, my_r1, my_z);
  else walk_tiles<kWalkCount>(ws, r, v, id, my_rect, my_r0, my_r1, 0.f);
}

// FP32 copies (high words and remainders) of the FP64 poses in shared memory.
__device__ __forceinline__ void stage_poses(const double *__restrict__ poses, int views, float *sp, float *spl) {
  for (int k = threadIdx.x; k < views * 12; k += blockDim.x) {
    const double pk = poses[k];
    const float hi = __double2float_rn(pk);
    sp[k] = hi;
    spl[k] = __double2float_rn(pk - (double)hi);
  }
}

__global__ void __launch_bounds__(kPrepBlock)
preprocess_kernel(Workspace ws, const float4 *__restrict__ gauss, int64_t n,
                  const double *__restrict__ poses, int views, Raster r, int zero_words) {
  pdl_wait();
  __shared__ float sp[kMaxViewsSmem * 12];
  __shared__ float spl[kMaxViewsSmem * 12];   // FP32 remainders of the FP64 poses
  const int v = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  stage_poses(poses, views, sp, spl);
  __syncthreads();
  if (blockIdx.x == 0 && blockIdx.y == 0)
    for (int k = threadIdx.x; k < views * 12; k += blockDim.x) ws.pose32[k] = sp[k];
  pdl_trigger();
  preprocess_one<false>(ws, load_rec(gauss, i, i < n), i, i < n, v, sp, spl, r, zero_words);
}

// Per-frame culling of the tracking loop: the Gaussians that can be visible
// under any pose whose rotation differs from the frame's starting pose by at
// most kCullRot rad and whose camera-space translation differs by at most
// kCullTrans m. Every camera-space point then moves by at most kCullRot |p|
// + kCullTrans; a Gaussian at least kCullNear in front of the camera moves on
// the image by less than `margin` px (set by the host from the focal length
// and the guard-clamped field of view, with a factor 2 to spare) and its
// alpha-ellipse box grows by less than 4%, so a candidate is one whose box,
// widened by 25% plus the margin, reaches the tile grid. Every Gaussian
// nearer than kCullNear that can come in front of the near plane is a
// candidate. A Gaussian below alpha_min opacity is never visible.

// Whether Gaussian (g0, g1, g2) is a candidate under the culling bounds of
// pose sp (FP32 3x4): its alpha-ellipse box, widened by kCullGrow and the
// image-motion margin, reaches the tile grid, or it is nearer than kCullNear
// and can come in front of the near plane; never below alpha_min opacity.
// (The tracking preprocess calls it only when it re-culls.)
__device__ __forceinline__ bool cull_keep(const float4 g0, const float4 g1, const float4 g2, const float *sp,
                                       const Raster &r, float margin) {
  const float x = sp[0] * g0.x + sp[1] * g0.y + sp[2] * g0.z + sp[3];
  const float y = sp[4] * g0.x + sp[5] * g0.y + sp[6] * g0.z + sp[7];
  const float z = sp[8] * g0.x + sp[9] * g0.y + sp[10] * g0.z + sp[11];
  const float m = kCullRot * sqrtf(x * x + y * y + z * z) + kCullTrans;
  const float o = 1.f / (1.f + expf(-g0.w));
  if (!(o > r.alpha_min)) return false;
  if (z < kCullNear) return z > r.z_near - m;
  Proj q;
  if (!project_gaussian(g0, g1, g2, sp, r, q)) return false;
  const float cnat = 2.f * (logf(q.o) - logf(r.alpha_min));
  const float ex = kCullGrow * sqrtf(fmaxf(cnat, 0.f) * q.A) + margin;
  const float ey = kCullGrow * sqrtf(fmaxf(cnat, 0.f) * q.C) + margin;
  const float X1 = (float)(r.tiles_x * kTile), Y1 = (float)(r.tiles_y * kTile);
  return q.u + ex >= 0.f && q.u - ex <= X1 && q.v + ey >= 0.f && q.v - ey <= Y1;
}

// Appends the warp's candidates to the list (every lane of the warp calls it).
__device__ __forceinline__ void cull_append(const Workspace &ws, bool cand, uint32_t i) {
  const unsigned ball = __ballot_sync(0xffffffffu, cand);
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  if (ball && lane == __ffs(ball) - 1) base = atomicAdd(ws.cand_n, (uint32_t)__popc(ball));
  base = __shfl_sync(0xffffffffu, base, ball ? __ffs(ball) - 1 : 0);
  if (cand) ws.cand_ids[base + __popc(ball & ((1u << lane) - 1u))] = i;
}

__global__ void __launch_bounds__(kPrepBlock)
cull_kernel(Workspace ws, const float4 *__restrict__ gauss, int64_t n, const double *__restrict__ pose, Raster r,
            float margin) {
  pdl_wait();
  __shared__ float sp[12];
  if (threadIdx.x < 12) sp[threadIdx.x] = (float)pose[threadIdx.x];
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x < 12) ws.cull_pose[threadIdx.x] = sp[threadIdx.x];
  // the frame's own cull: no re-cull is pending
  if (blockIdx.x == 0 && threadIdx.x == 0) ws.counters[CNT_RECULL] = 0u;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool cand = false;
  if (i < n) {
    const float4 g0 = __ldg(gauss + 4 * i), g1 = __ldg(gauss + 4 * i + 1), g2 = __ldg(gauss + 4 * i + 2);
    cand = cull_keep(g0, g1, g2, sp, r, margin);
  }
  cull_append(ws, cand, (uint32_t)i);
}

// The tracking loop's preprocess (one view, fixed-capacity buckets) over
// the frame's candidates, or over all Gaussians when the pose has left the
// culling bounds; a fixed grid strides over the list. With prefetch (the
// candidate list was written two or more launches earlier), each thread
// loads its first candidate's id and record before waiting for the
// predecessor (which writes the pose), so that those round trips overlap the
// predecessor's tail.
__global__ void __launch_bounds__(kPrepBlock, 6)
preprocess_cull_kernel(Workspace ws, const float4 *__restrict__ gauss, int64_t n, const double *__restrict__ pose,
                       Raster r, int zero_words, int prefetch, float margin) {
  __shared__ float sp[12], spl[12];
  __shared__ int s_valid, s_recull;
  const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t pre_count = 0, pre_i = 0;
  Rec pre;
  if (prefetch) {
    pre_count = (int64_t)__ldcg(ws.cand_n);
    if (first < pre_count) pre_i = (int64_t)__ldcg(ws.cand_ids + first);
    pre = load_rec(gauss, pre_i, first < pre_count && pre_i < n);
  }
  // (no early trigger: the forward's longest-first CTAs are placed once
  // this grid has left the SMs)
  pdl_wait();
  stage_poses(pose, 1, sp, spl);
  __syncthreads();
  if (threadIdx.x == 0) {
    s_valid = within_cull_bounds(sp, ws.cull_pose) ? 1 : 0;
    // the previous iteration's pose step left the bounds: it moved the
    // culling pose to this pose and emptied the list, which this launch
    // refills while it takes every Gaussian
    s_recull = __ldcg(ws.counters + CNT_RECULL) != 0u ? 1 : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x < 12) ws.pose32[threadIdx.x] = sp[threadIdx.x];
  // the forward takes the largest bucket's requirement with atomicMax
  if (blockIdx.x == 0 && threadIdx.x == 0)
    *reinterpret_cast<unsigned long long *>(ws.counters + CNT_REQ_LO) = 0ull;
  __syncthreads();
  const bool recull = s_recull != 0;
  const bool use_cand = s_valid != 0 && !recull;
  const int64_t count = use_cand ? (int64_t)*ws.cand_n : n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
    const int64_t k = base + threadIdx.x;
    const bool valid = k < count;
    if (prefetch && use_cand && k == first) {
      preprocess_one<true>(ws, pre, pre_i, valid && pre_i < n, 0, sp, spl, r, zero_words);
      continue;
    }
    const int64_t i = !valid ? 0 : (use_cand ? (int64_t)ws.cand_ids[k] : k);
    const Rec rec = load_rec(gauss, i, valid && i < n);
    if (recull) cull_append(ws, valid && i < n && cull_keep(rec.g0, rec.g1, rec.g2, sp, r, margin), (uint32_t)i);
    preprocess_one<true>(ws, rec, i, valid && i < n, 0, sp, spl, r, zero_words);
  }
}

__global__ void order_identity_kernel(uint32_t *order, int tiles) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < tiles; k += gridDim.x * blockDim.x) order[k] = (uint32_t)k;
}

// One CTA turns the per-tile counts into offsets and the launch order, and
// publishes the visible-list lengths and the pair total.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads)
tile_scan_kernel(Workspace ws, int views, Raster r) {
  pdl_wait();
  const uint64_t total = block_scan_tiles(ws.tile_count, ws.tile_start, ws.tile_cursor, views * r.T, ws.tile_order,
                                          ws.band > 0 ? ws.band : 1);
  for (int k = threadIdx.x; k < views; k += blockDim.x) {
    ws.vis_n[k] = ws.vis_append[k];
    ws.vis_append[k] = 0u;
  }
  if (threadIdx.x == 0) {
    ws.tile_start[views * r.T] = (uint32_t)(total > 0xFFFFFFFFull ? 0xFFFFFFFFull : total);
    ws.counters[CNT_REQ_LO] = (uint32_t)total;
    ws.counters[CNT_REQ_HI] = (uint32_t)(total >> 32);
    if (total > (uint64_t)ws.max_pairs) atomicOr(ws.counters + CNT_STATUS, kStatusCapacity);
  }
}

__device__ __forceinline__ bool pairs_overflow(const Workspace &ws, int entries) {
  uint64_t tot = (uint64_t)ws.counters[CNT_REQ_LO] | ((uint64_t)ws.counters[CNT_REQ_HI] << 32);
  (void)entries;
  return tot > (uint64_t)ws.max_pairs;
}

__global__ void __launch_bounds__(kPrepBlock)
emit_kernel(Workspace ws, int64_t n, Raster r) {
  pdl_wait();
  const int v = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // the pair total, the list length and this thread's list entry are loaded
  // together (the entry speculatively: i < n <= max_n is always in the
  // buffer; a stale value is clamped to a valid slot and discarded below)
  const uint32_t req_lo = ws.counters[CNT_REQ_LO], req_hi = ws.counters[CNT_REQ_HI];
  const int64_t nv = ws.vis_n[v];
  uint32_t id = i < n ? ws.vis_ids[(size_t)v * ws.max_n + i] : 0u;
  if ((((uint64_t)req_hi << 32) | req_lo) > (uint64_t)ws.max_pairs) return;
  if ((int64_t)blockIdx.x * blockDim.x >= nv) return;   // whole CTA past the visible list
  uint2 rect = make_uint2(0u, 0u);
  float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
  float z = 0.f;
  if (i < nv) {
    const size_t slot = (size_t)v * ws.max_n + min(id, (uint32_t)(n - 1));
    rect = ws.rect[slot];
    r0 = ws.rec2d[slot * 3 + 0];
    r1 = ws.rec2d[slot * 3 + 1];
    z = ws.rec2d[slot * 3 + 2].x;
  } else {
    id = 0;
  }
  walk_tiles<kWalkEmit>(ws, r, v, id, rect, r0, r1, z);
}

// MASKS: record per warp the list entries its pixels took (ws.warp_masks,
// the tracking loop); COUNT: count evaluations and contributions (ws.evals).
template <bool MASKS, bool COUNT>
__global__ void __launch_bounds__(kTilePix, 5)
render_fwd_kernel(Workspace ws, int views, Raster r, Loss l, const float4 *__restrict__ targets,
                  float *__restrict__ image, int32_t *__restrict__ last, double *__restrict__ loss) {
  // (no early trigger: the adjoint's CTAs are placed on the SMs as they
  // empty, which keeps its longest-first launch order spread over the SMs)
  pdl_wait();
  __shared__ __align__(16) uint64_t s_key[kSortSmallCap];
  __shared__ float4 s_a[kTilePix], s_b[kTilePix], s_c[kTilePix];   // s_a: {u hi, v hi, u lo, v lo}
  __shared__ float2 s_e[kTilePix];                                  // box half extents
  __shared__ float2 s_red[kTilePix / 32];
  __shared__ int s_last;
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // blocks are launched in order of descending list length. In the
  // fixed-bucket layout a tile whose list overflowed its bucket is skipped
  // (and reported); the forward publishes the visible count, the largest
  // bucket's requirement and the counts the next iteration's order is
  // ranked from. Otherwise an overflow anywhere skips every tile.
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
    ovf = pairs_overflow(ws, views * r.T);
    tile = ovf ? (int)blockIdx.x : (int)ws.tile_order[blockIdx.x];
  }
  const int v = tile / r.T, tv = tile - v * r.T;
  const int tx = tv % r.tiles_x, ty = tv / r.tiles_x;
  // warp w covers the 8x4 pixel block (w % 2, w / 2) of the tile
  const int bx0 = tx * kTile + (warp & 1) * 8, by0 = ty * kTile + (warp >> 1) * 4;
  const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
  const bool inside = px < r.W && py < r.H;
  uint32_t s = 0u, e = 0u;
  if (!ovf) tile_range(ws, tile, s, e);
  uint32_t *const wmask = MASKS ? ws.warp_masks + (size_t)tile * kMaskGroups * 8 + warp : nullptr;
  const size_t vbase = (size_t)v * ws.max_n;
  const float bcx = (float)bx0 + 3.5f, bcy = (float)by0 + 1.5f;

  // depth-sort the tile's bucket and publish the order for the backward: in
  // shared memory up to kSortSmallCap keys, else out of core (chunks sorted in
  // shared memory, then merged pairwise through global memory)
  const bool own_sort = sort_tile_bucket(ws, s, (int)(e - s), s_key);

  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f, oo = 0.f, rm = 0.f;
  int lastk = 0;
  unsigned n_eval = 0, n_contrib = 0;
  bool done = !inside;
  const float fpx = (float)px, fpy = (float)py;
  for (uint32_t base = s; base < e; base += kTilePix) {
    if (__syncthreads_count(!done) == 0) break;
    const uint32_t k = base + tid;
    const uint32_t id = k < e ? (own_sort ? (uint32_t)s_key[k - s] : ws.sorted_ids[k]) : 0u;
    if (k < e && DAGS_IN_BOUNDS(id < (uint32_t)ws.max_n && k < (uint64_t)ws.max_pairs, ws.counters + CNT_STATUS)) {
      const size_t slot = vbase + id;
      const float4 r0 = ws.rec2d[slot * 3 + 0];
      const float2 lo = ws.rec_lo[slot];
      s_a[tid] = make_float4(r0.x, r0.y, lo.x, lo.y);
      s_e[tid] = make_float2(r0.z, r0.w);
      s_b[tid] = ws.rec2d[slot * 3 + 1];
      s_c[tid] = ws.rec2d[slot * 3 + 2];
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kTilePix, e - base);
    if (__all_sync(FULL, done)) continue;
    for (int g = 0; g < 8 && g * 32 < cnt; ++g) {
      // entries whose ellipse box meets this warp's pixel block
      const int jj = g * 32 + lane;
      bool hit = false;
      if (jj < cnt) {
        const float4 a = s_a[jj];
        const float2 ex = s_e[jj];
        hit = fabsf(a.x - bcx) <= ex.x + 3.5f && fabsf(a.y - bcy) <= ex.y + 1.5f;
      }
      unsigned mask = __ballot_sync(FULL, hit);
      unsigned took = 0u;   // entries at least one pixel of the warp took
      while (mask) {
        const int bit = __ffs(mask) - 1;
        const int j = g * 32 + bit;
        mask &= mask - 1;
        // evaluated by every lane, without branches: a lane that is done,
        // or whose alpha is below alpha_min, or that would stop here adds
        // a zero weight and keeps T (x + 0 * c == x), so each pixel's sums
        // are those of the branching form, operation for operation
        // (explicitly rounded operations: every kernel variant computes the
        // same bits)
        const float4 a = s_a[j], b = s_b[j];
        const float dx = __fadd_rn(__fsub_rn(a.x, fpx), a.z), dy = __fadd_rn(__fsub_rn(a.y, fpy), a.w);
        const float p = __fmaf_rn(__fmul_rn(b.x, dx), dx,
                                  __fmaf_rn(__fmul_rn(b.y, dx), dy, __fmaf_rn(__fmul_rn(b.z, dy), dy, b.w)));
        const bool live = !done && p >= r.log2_alpha_min;   // else alpha < alpha_min
        const float alpha = fminf(r.alpha_max, hw_exp2(p));
        const float tt = __fmul_rn(T, __fsub_rn(1.f, alpha));
        const bool stop = live && tt < r.t_min;
        const bool contrib = live && !stop;
        if (COUNT) { n_eval += done ? 0u : 1u; n_contrib += contrib ? 1u : 0u; }
        done = done || stop;
        const float w = contrib ? __fmul_rn(alpha, T) : 0.f;
        const float4 c = s_c[j];
        const uint32_t rg = __float_as_uint(c.z), bl = __float_as_uint(c.w);
        cr = __fmaf_rn(bf16_lo(rg), w, cr); cg = __fmaf_rn(bf16_hi(rg), w, cg); cb = __fmaf_rn(bf16_lo(bl), w, cb);
        dd = __fmaf_rn(c.x, w, dd); oo = __fadd_rn(oo, w); rm = __fmaf_rn(c.y, w, rm);
        T = contrib ? tt : T;
        lastk = contrib ? (int)(base - s) + j + 1 : lastk;
        if (MASKS && __any_sync(FULL, contrib)) took |= 1u << bit;
      }
      if (MASKS) {
        const int gk = (int)((base - s) >> 5) + g;
        if (lane == 0 && gk < kMaskGroups) wmask[gk * 8] = took;
      }
      if (__all_sync(FULL, done)) break;
    }
  }

  if (COUNT) add_eval_counts(ws, 0, n_eval, n_contrib);
  float lpx = 0.f;
  if (inside) {
    const size_t P = (size_t)r.W * r.H;
    const size_t pix = (size_t)py * r.W + px;
    float wgt = 0.f;
    if (targets) {
      if (l.weight_mode == 0) wgt = oo > l.o_eps ? (oo - rm) / oo : 0.f;
      else wgt = oo - rm;
      const float4 tg = targets[(size_t)v * P + pix];
      const float l1 = fabsf(cr - tg.x) + fabsf(cg - tg.y) + fabsf(cb - tg.z);
      const float ld = tg.w > 0.f ? fabsf(dd - tg.w) : 0.f;
      lpx = tg.x >= 0.f ? __fmul_rn(wgt, __fmaf_rn(l.lambda_pho, l1, __fmul_rn(l.lambda_depth, ld))) : 0.f;
    }
    float *img = image + (size_t)v * DAGS_IMG_CHANNELS * P + pix;
    img[0 * P] = cr; img[1 * P] = cg; img[2 * P] = cb; img[3 * P] = dd;
    img[4 * P] = oo; img[5 * P] = rm; img[6 * P] = T; img[7 * P] = wgt;
    last[(size_t)v * P + pix] = lastk;
  }
  if (!loss) return;
  // the tile's 256 pixel losses are summed exactly enough for FP64 without
  // the FP64 pipe: compensated FP32 (two-sum, a high and a low word) over a
  // fixed shuffle tree, then over the 8 warps in order; the tile's partial is
  // the FP64 sum of the two words
  float lh = lpx, ll = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, lh, o), ol = __shfl_xor_sync(0xffffffffu, ll, o);
    float sh, se;
    two_sum(lh, oh, sh, se);
    lh = sh;
    ll = __fadd_rn(__fadd_rn(ll, ol), se);
  }
  if ((tid & 31) == 0) s_red[tid >> 5] = make_float2(lh, ll);
  __syncthreads();
  if (tid == 0) {
    float th = 0.f, tl = 0.f;
    for (int w = 0; w < kTilePix / 32; ++w) {
      float sh, se;
      two_sum(th, s_red[w].x, sh, se);
      th = sh;
      tl = __fadd_rn(__fadd_rn(tl, s_red[w].y), se);
    }
    ws.loss_partial[tile] = (double)th + (double)tl;
    __threadfence();
    unsigned int done_ctas = atomicAdd(ws.counters + CNT_DONE_RENDER, 1u);
    s_last = (done_ctas == gridDim.x - 1);
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  // Deterministic FP64 sum of the per-tile partials: fixed strided
  // assignment, then a fixed tree.
  __shared__ double s_d[kTilePix];
  const int np = views * r.T;
  double acc = 0.0;
  for (int k = tid; k < np; k += kTilePix) acc += __ldcg(ws.loss_partial + k);
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

cudaError_t launch_preprocess(const Workspace &ws, const float4 *gauss, int64_t n, const double *poses,
                              int views, const Raster &r, int zero_grad_words, cudaStream_t s) {
  if (views > kMaxViewsSmem) return cudaErrorInvalidValue;
  const unsigned gx = (unsigned)((n + kPrepBlock - 1) / kPrepBlock);
  dim3 grid(gx > 0 ? gx : 1u, (unsigned)views);
  cudaError_t e = launch_pdl(preprocess_kernel, grid, dim3(kPrepBlock), 0, s, ws, gauss, n, poses, views, r,
                             zero_grad_words);
  if (e == cudaSuccess) e = launch_pdl(tile_scan_kernel, dim3(1), dim3(kScanThreads), 0, s, ws, views, r);
  return e;
}

// The candidates' image motion bound: (rot (1 + L)^2 + trans / near) f, L
// the guard-clamped half field of view, times 2.
static float cull_margin(const Raster &r) {
  const float L = fmaxf(r.limx, r.limy), f = fmaxf(r.fx, r.fy);
  return 2.f * f * (kCullRot * (1.f + L) * (1.f + L) + kCullTrans / kCullNear);
}

cudaError_t launch_preprocess_direct(const Workspace &ws, const float4 *gauss, int64_t n, const double *pose,
                                     const Raster &r, int zero_grad_words, bool prefetch, cudaStream_t s) {
  if (ws.bucket_cap == 0 || !ws.cand_ids) return cudaErrorInvalidValue;
  // the frame's culled list: a fixed grid of one wave (6 CTAs per SM, the
  // register budget with the prefetched record) strides over it
  const unsigned gx = (unsigned)((n + kPrepBlock - 1) / kPrepBlock);
  const unsigned g = gx < (unsigned)(6 * ws.band) ? (gx > 0 ? gx : 1u) : (unsigned)(6 * ws.band);
  return launch_pdl(preprocess_cull_kernel, dim3(g), dim3(kPrepBlock), 0, s, ws, gauss, n, pose, r,
                    zero_grad_words, prefetch ? 1 : 0, cull_margin(r));
}

cudaError_t launch_order_identity(uint32_t *order, int tiles, cudaStream_t s) {
  if (tiles <= 0) return cudaSuccess;
  order_identity_kernel<<<(tiles + 255) / 256, 256, 0, s>>>(order, tiles);
  return cudaGetLastError();
}

cudaError_t launch_cull(const Workspace &ws, const float4 *gauss, int64_t n, const double *pose, const Raster &r,
                        cudaStream_t s) {
  const float margin = cull_margin(r);
  cudaError_t e = cudaMemsetAsync(ws.cand_n, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess || n == 0) return e;
  return launch_pdl(cull_kernel, dim3((unsigned)((n + kPrepBlock - 1) / kPrepBlock)), dim3(kPrepBlock), 0, s, ws,
                    gauss, n, pose, r, margin);
}

cudaError_t launch_emit(const Workspace &ws, int64_t n, int views, const Raster &r, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  dim3 grid((unsigned)((n + kPrepBlock - 1) / kPrepBlock), (unsigned)views);
  return launch_pdl(emit_kernel, grid, dim3(kPrepBlock), 0, s, ws, n, r);
}

cudaError_t launch_render_fwd(const Workspace &ws, int views, int64_t n, const Raster &r, const Loss &l,
                              const float4 *targets, float *image, int32_t *last, double *loss,
                              cudaStream_t s) {
  (void)n;
  const dim3 grid((unsigned)(views * r.T));
  const bool masks = ws.warp_masks != nullptr;
  if (ws.count_evals) {
    if (masks) return launch_pdl(render_fwd_kernel<true, true>, grid, dim3(kTilePix), 0, s, ws, views, r, l, targets,
                                 image, last, loss);
    return launch_pdl(render_fwd_kernel<false, true>, grid, dim3(kTilePix), 0, s, ws, views, r, l, targets, image,
                      last, loss);
  }
  if (masks) return launch_pdl(render_fwd_kernel<true, false>, grid, dim3(kTilePix), 0, s, ws, views, r, l, targets,
                               image, last, loss);
  return launch_pdl(render_fwd_kernel<false, false>, grid, dim3(kTilePix), 0, s, ws, views, r, l, targets, image,
                    last, loss);
}

}  // namespace dags
