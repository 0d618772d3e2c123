// Per-tile depth sort shared by the render kernels (sm_103a): one CTA of
// kTilePix threads sorts its tile's bucket of (depth bits << 32 | id) keys.
#pragma once

#include "common.cuh"

namespace dags {

// Render launch order: tiles ranked by descending list length in bins of 8
// entries (empty tiles last), each band of `band` consecutive ranks (one CTA
// per SM in a dispatch round) reversed every other band, so that the SM that
// receives a band's longest tile receives the next band's shortest one.
constexpr int kLenBins = 257;   // 256 length bins (descending) + empty tiles

__device__ __forceinline__ int length_bin(uint32_t c) { return c ? 255 - (int)min(c >> 3, 255u) : 256; }

// Slot of rank `pos` in the band-reversed ("snake") order of `total` ranks.
__device__ __forceinline__ uint32_t snake_slot(uint32_t pos, uint32_t total, uint32_t band) {
  const uint32_t b = pos / band, q = pos - b * band, base = b * band;
  const uint32_t width = min(band, total - base);
  return base + ((b & 1u) ? width - 1u - q : q);
}

// Ranks tiles by descending count (bins of 8 entries, empty tiles last),
// band-reversed as block_scan_tiles orders them; one whole CTA. Up to
// kRankStage tiles, the bins are formed once into shared memory by loads
// issued four at a time, so that the two passes wait on L2 once rather
// than once per round.
constexpr int kRankStage = 4096;

__device__ inline void rank_tiles(const uint32_t *count, int total, uint32_t *order, int band) {
  __shared__ uint32_t s_bin[kLenBins];
  __shared__ uint16_t s_tb[kRankStage];
  const int tid = threadIdx.x, lane = tid & 31;
  const bool staged = total <= kRankStage;
  for (int k = tid; k < kLenBins; k += blockDim.x) s_bin[k] = 0u;
  if (staged) {
#pragma unroll 4
    for (int k = tid; k < total; k += blockDim.x) s_tb[k] = (uint16_t)length_bin(__ldcg(count + k));
  }
  __syncthreads();
  auto bin_of = [&](int k) { return staged ? (int)s_tb[k] : length_bin(__ldcg(count + k)); };
  for (int k0 = 0; k0 < total; k0 += blockDim.x) {
    const int k = k0 + tid;
    int bin = 1024 + lane;   // no element: a key of its own
    if (k < total) bin = bin_of(k);
    const unsigned grp = __match_any_sync(0xffffffffu, bin);
    if (bin < kLenBins && lane == __ffs(grp) - 1) atomicAdd(&s_bin[bin], (uint32_t)__popc(grp));
  }
  __syncthreads();
  if (tid < 32) {
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
  const uint32_t bnd = band > 0 ? (uint32_t)band : 1u;
  for (int k0 = 0; k0 < total; k0 += blockDim.x) {
    const int k = k0 + tid;
    int bin = 1024 + lane;
    if (k < total) bin = bin_of(k);
    const unsigned grp = __match_any_sync(0xffffffffu, bin);
    const int leader = __ffs(grp) - 1;
    uint32_t pos = 0;
    if (bin < kLenBins && lane == leader) pos = atomicAdd(&s_bin[bin], (uint32_t)__popc(grp));
    pos = __shfl_sync(0xffffffffu, pos, leader) + (uint32_t)__popc(grp & ((1u << lane) - 1u));
    if (k < total) order[snake_slot(pos, (uint32_t)total, bnd)] = (uint32_t)k;
  }
}


// Ascending bitonic sort of s[0, len2) (len2 a power of two) by the CTA.
__device__ __forceinline__ void bitonic_smem(uint64_t *s, int len2) {
  for (int k = 2; k <= len2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (len2 >> 1); t += blockDim.x) {
        const int i = 2 * t - (t & (j - 1));
        const int p = i + j;
        const uint64_t a = s[i], b = s[p];
        const bool up = (i & k) == 0;
        if ((a > b) == up) { s[i] = b; s[p] = a; }
      }
      __syncthreads();
    }
  }
}

// Ascending sort of s[0, n) (s 16-byte aligned, n <= kTilePix, unique keys)
// by rank: thread i counts the keys below key i with broadcast reads of the
// whole list, then every key is stored at its rank. The same order as the
// bitonic network; n steps of one thread instead of log2(n)^2 / 2 barrier
// stages of the CTA, which pays for lists of up to one key per thread.
__device__ __forceinline__ void rank_sort_smem(uint64_t *s, int n) {
  const int tid = threadIdx.x;
  const bool has = tid < n;
  const uint64_t key = has ? s[tid] : 0ull;
  int rank = 0;
  if (has) {
    int j = 0;
    for (; j + 1 < n; j += 2) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(s + j);
      rank += (v.x < key) + (v.y < key);
    }
    if (j < n) rank += s[j] < key;
  }
  __syncthreads();
  if (has) s[rank] = key;
  __syncthreads();
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Merge sorted runs a[0, la) and b[0, lb) into out[0, la + lb) with the CTA
// (merge path: each thread finds its split by binary search, then merges its
// slice sequentially). Keys are unique within a tile.
__device__ inline void merge_runs(const uint64_t *a, int la, const uint64_t *b, int lb, uint64_t *out) {
  const int m = la + lb;
  const int per = (m + blockDim.x - 1) / blockDim.x;
  const int k0 = min(m, (int)threadIdx.x * per);
  const int k1 = min(m, k0 + per);
  if (k0 < k1) {
    int lo = max(0, k0 - lb), hi = min(k0, la);
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (a[mid] < b[k0 - mid - 1]) lo = mid + 1;
      else hi = mid;
    }
    int ia = lo, ib = k0 - lo;
    for (int k = k0; k < k1; ++k) {
      const bool take_a = ib >= lb || (ia < la && a[ia] < b[ib]);
      out[k] = take_a ? a[ia++] : b[ib++];
    }
  }
}

// True when the last preprocess needed more (tile, Gaussian) pairs than the
// workspace holds: the buckets are then incomplete and nothing is rendered.
__device__ __forceinline__ bool pairs_overflow_ws(const Workspace &ws) {
  const uint64_t tot = (uint64_t)ws.counters[CNT_REQ_LO] | ((uint64_t)ws.counters[CNT_REQ_HI] << 32);
  return tot > (uint64_t)ws.max_pairs;
}

// Depth-sorts the tile bucket keys[s, s + len) and publishes the ordered ids
// in sorted_ids[s, s + len): in shared memory (s_key, kSortSmallCap keys) when
// the bucket fits, then the sorted keys stay in s_key and the function
// returns true; otherwise out of core (chunks sorted in shared memory, then
// merged pairwise through global memory) and it returns false. With
// publish_small = false a bucket sorted in shared memory is not copied to
// sorted_ids (for a caller that reads its order from s_key only). Called by
// all threads of the CTA.
__device__ __forceinline__ bool sort_tile_bucket(const Workspace &ws, uint32_t s, int len, uint64_t *s_key,
                                                 bool publish_small = true) {
  const int tid = threadIdx.x;
  const bool own_sort = len <= kSortSmallCap;
  if (own_sort && len > 0 && len <= kTilePix) {
    // (s_key is 16-byte aligned: the rank count reads two keys at a time)
    for (int k = tid; k < len; k += kTilePix) s_key[k] = ws.keys[s + k];
    __syncthreads();
    rank_sort_smem(s_key, len);
    if (publish_small)
      for (int k = tid; k < len; k += kTilePix) ws.sorted_ids[s + k] = (uint32_t)s_key[k];
  } else if (own_sort && len > 0) {
    const int len2 = next_pow2(len);
    for (int k = tid; k < len2; k += kTilePix) s_key[k] = k < len ? ws.keys[s + k] : ~0ull;
    __syncthreads();
    bitonic_smem(s_key, len2);
    if (publish_small)
      for (int k = tid; k < len; k += kTilePix) ws.sorted_ids[s + k] = (uint32_t)s_key[k];
  } else if (len > 0) {
    uint64_t *src = ws.keys + s, *dst = ws.keys_tmp + s;
    for (int c0 = 0; c0 < len; c0 += kSortSmallCap) {
      const int cl = min(kSortSmallCap, len - c0);
      const int cl2 = next_pow2(cl);
      for (int k = tid; k < cl2; k += kTilePix) s_key[k] = k < cl ? src[c0 + k] : ~0ull;
      __syncthreads();
      bitonic_smem(s_key, cl2);
      for (int k = tid; k < cl; k += kTilePix) src[c0 + k] = s_key[k];
      __syncthreads();
    }
    for (int width = kSortSmallCap; width < len; width <<= 1) {
      for (int lo = 0; lo < len; lo += 2 * width) {
        const int la = min(width, len - lo);
        const int lb = max(0, min(width, len - lo - width));
        merge_runs(src + lo, la, src + lo + la, lb, dst + lo);
      }
      __syncthreads();
      uint64_t *t = src; src = dst; dst = t;
    }
    for (int k = tid; k < len; k += kTilePix) ws.sorted_ids[s + k] = (uint32_t)src[k];
    __syncthreads();
  }
  return own_sort;
}

}  // namespace dags
