// Two-level ingestion for universes too large for a shared-memory
// sub-histogram: the "hierarchical partitioning" the paper names for large U
// (Sec. "Limitations"), built so that every count still lands in a
// shared-memory counter instead of an L2 atomic (random L2 atomics top out at
// ~0.2 T/s on this GPU, shared-memory atomics at ~3.5 T/s).
//
// A key k splits into a bucket b = k >> L and a low part k & (2^L - 1).
//   pass 1 (partition_kernel)  per 8192-key tile: rank every key within its
//          bucket (shared-memory counters per warp), scan to bucket starts,
//          write the tile's low parts grouped by bucket (uint16), the tile's
//          bucket starts (toff[t][0..B]) and add the bucket totals up.
//   plan   (plan_kernel)       split every non-empty bucket into parts of
//          about item_keys keys (contiguous tile ranges) -> work items.
//   pass 2 (bucket_kernel)     per item: gather the bucket's segments of the
//          item's tiles, count the low parts in a shared-memory histogram of
//          2^L bins (Eq. (1) on the sub-universe, with the warp CRN) and add
//          it into H[b * 2^L ...].
// H is zeroed before pass 2.  Counting is exact: pass 1 only moves keys.
// Only equality and shifts touch keys; key < U is checked against the bound.
#include <algorithm>

#include "hist_device.cuh"
#include "internal.h"

namespace dialsort {

namespace {

constexpr uint32_t kP1Threads = 512;
constexpr uint32_t kP1Warps = kP1Threads / 32;
constexpr uint32_t kP1Tile = 8192;                        // keys per tile
constexpr uint32_t kP1Keys = kP1Tile / kP1Threads;        // 16 consecutive keys per thread

struct Item {
  uint32_t bucket, t0, t1, pad;
};


// shared-memory words before the staging buffer: counters, totals, scan scratch; a multiple of 4
__host__ __device__ __forceinline__ uint32_t p1_stage_words(uint32_t B) {
  return (kP1Warps * B + B + 16 + 3) & ~3u;
}

// ------------------------------------------------------------------ pass 1
// Thread tid owns keys [16 tid, 16 tid + 16) of the tile, so runs of keys with
// the same bucket (long under skew, sorted input or repeated keys) are merged
// by the thread itself: one shared-memory add per run, not per key.  Counts go
// to per-warp counters (red), a scan turns them into bases, and a second
// atomic on the same counters hands each run its positions.
__global__ void __launch_bounds__(kP1Threads, 2) partition_kernel(const uint32_t* __restrict__ keys, uint64_t n,
                                                                   uint32_t U, uint32_t L, uint32_t B,
                                                                   uint64_t num_tiles, uint16_t* __restrict__ low,
                                                                   uint16_t* __restrict__ toff,
                                                                   uint32_t* __restrict__ btot, uint32_t* err,
                                                                   uint32_t crn_mode) {
  (void)crn_mode;
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* cnt = sm;                          // [kP1Warps][B]: counts, then bases / cursors
  uint32_t* bacc = cnt + kP1Warps * B;         // [B]: this CTA's bucket totals over its tiles
  uint32_t* red = bacc + B;                    // block scan scratch (16 words)
  // [kP1Tile] low parts of one tile, read as uint4: starts on a 16-byte boundary
  uint16_t* stage = reinterpret_cast<uint16_t*>(sm + p1_stage_words(B));
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t lowmask = (1u << L) - 1u;
  bool bad = false;

  for (uint32_t b = tid; b < B; b += kP1Threads) bacc[b] = 0;

  for (uint64_t t = blockIdx.x; t < num_tiles; t += gridDim.x) {
    for (uint32_t i = tid; i < kP1Warps * B; i += kP1Threads) cnt[i] = 0;
    __syncthreads();
    const uint64_t base = t * kP1Tile;
    const uint32_t len = (uint32_t)((n - base) < kP1Tile ? (n - base) : kP1Tile);
    const uint32_t first = kP1Keys * tid;
    const uint4* src = reinterpret_cast<const uint4*>(keys + base + first);

    // this thread's consecutive keys; bit i of vm: key i is real and < U
    uint32_t kv[kP1Keys];
    uint32_t vm = 0;
#pragma unroll
    for (uint32_t i = 0; i < kP1Keys / 4; ++i) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (first + 4 * i + 3 < len) {
        v = __ldg(src + i);
      } else if (first + 4 * i < len) {
        v.x = keys[base + first + 4 * i];
        if (first + 4 * i + 1 < len) v.y = keys[base + first + 4 * i + 1];
        if (first + 4 * i + 2 < len) v.z = keys[base + first + 4 * i + 2];
      }
      kv[4 * i] = v.x;
      kv[4 * i + 1] = v.y;
      kv[4 * i + 2] = v.z;
      kv[4 * i + 3] = v.w;
    }
#pragma unroll
    for (uint32_t i = 0; i < kP1Keys; ++i) {
      const bool real = first + i < len;
      const bool ok = kv[i] < U;
      bad |= real && !ok;
      vm |= (real && ok) ? (1u << i) : 0u;
    }
    // Runs of one bucket pay off only when they are common (skew, sorted
    // input, repeated keys); the warp decides together how it ingests the tile.
    uint32_t same = 0;  // bit i: key i continues the bucket of key i - 1
#pragma unroll
    for (uint32_t i = 1; i < kP1Keys; ++i) same |= ((kv[i] >> L) == (kv[i - 1] >> L)) ? (1u << i) : 0u;
    same &= vm & (vm << 1);
    const bool runs = __popc(__ballot_sync(0xffffffffu, same != 0)) >= 16;
    uint32_t* wcnt = cnt + warp * B;
    if (runs) {
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i) {
        if (((vm >> i) & 1u) && !((same >> i) & 1u))  // a run starts here; its length counts the ones after it
          atomicAdd(wcnt + (kv[i] >> L), (uint32_t)__ffs(~(same >> (i + 1))));
      }
    } else {
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i)
        if ((vm >> i) & 1u) atomicAdd(wcnt + (kv[i] >> L), 1u);
    }
    __syncthreads();

    // bucket-major, warp-minor exclusive scan of the counts -> bases (in place)
    const uint32_t E = kP1Warps * B;
    const uint32_t per = (E + kP1Threads - 1) / kP1Threads;
    const uint32_t e0 = min(tid * per, E), e1 = min(e0 + per, E);
    uint32_t local = 0;
    for (uint32_t e = e0; e < e1; ++e) local += cnt[(e % kP1Warps) * B + e / kP1Warps];
    uint32_t x = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w0 = lane < kP1Warps ? red[lane] : 0u;
      uint32_t s = w0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
        if (lane >= (uint32_t)d) s += y;
      }
      if (lane < kP1Warps) red[lane] = s - w0;
      if (lane == kP1Warps - 1) red[kP1Warps] = s;  // valid keys of the tile
    }
    __syncthreads();
    uint32_t acc = red[warp] + (x - local);
    for (uint32_t e = e0; e < e1; ++e) {
      uint32_t* c = &cnt[(e % kP1Warps) * B + e / kP1Warps];
      const uint32_t v = *c;
      *c = acc;
      acc += v;
    }
    __syncthreads();
    // the tile's bucket starts (warp 0's base), and this CTA's bucket totals
    const uint32_t tile_valid = red[kP1Warps];
    uint16_t* trow = toff + t * (uint64_t)(B + 1);
    for (uint32_t b = tid; b <= B; b += kP1Threads) {
      const uint32_t start = b < B ? cnt[b] : tile_valid;
      trow[b] = (uint16_t)start;
      if (b < B) bacc[b] += (b + 1 < B ? cnt[b + 1] : tile_valid) - start;
    }
    __syncthreads();  // the bases are read above before the cursors move below
    // each run takes its positions with one atomic on its (warp, bucket) cursor
    if (runs) {
      uint32_t pos = 0;
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i) {
        if ((vm >> i) & 1u) {
          if (!((same >> i) & 1u)) {
            pos = atomicAdd(wcnt + (kv[i] >> L), (uint32_t)__ffs(~(same >> (i + 1))));
          } else {
            ++pos;
          }
          stage[pos] = (uint16_t)(kv[i] & lowmask);
        }
      }
    } else {
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i)
        if ((vm >> i) & 1u) stage[atomicAdd(wcnt + (kv[i] >> L), 1u)] = (uint16_t)(kv[i] & lowmask);
    }
    __syncthreads();
    // write the grouped low parts: tile t owns low[t * 8192 ...]
    const uint32_t vecs = (tile_valid + 7) / 8;
    uint4* dst = reinterpret_cast<uint4*>(low + t * kP1Tile);
    const uint4* st4 = reinterpret_cast<const uint4*>(stage);
    for (uint32_t v = tid; v < vecs; v += kP1Threads) dst[v] = st4[v];
    __syncthreads();
  }
  if (bad) raise_error(err, ERRBIT_KEY_RANGE);
  for (uint32_t b = tid; b < B; b += kP1Threads)
    if (bacc[b]) red_add_global(btot + b, bacc[b]);
}

// ------------------------------------------------------------------ plan
// Number of parts of every bucket (ceil(total / item_keys)) and where its
// items start in the item list.
__global__ void __launch_bounds__(1024) plan_kernel(const uint32_t* __restrict__ btot, uint32_t B,
                                                    uint64_t item_keys, uint32_t* __restrict__ pbase,
                                                    uint32_t* nitems) {
  __shared__ uint32_t red[33];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  // each thread owns a contiguous run of buckets (B <= 2047 -> at most 2)
  const uint32_t per = (B + 1023) / 1024;
  const uint32_t b0 = min(tid * per, B), b1 = min(b0 + per, B);
  uint32_t local = 0;
  for (uint32_t b = b0; b < b1; ++b) local += (uint32_t)((btot[b] + item_keys - 1) / item_keys);
  uint32_t x = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w0 = red[lane];
    uint32_t s = w0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= (uint32_t)d) s += y;
    }
    red[lane] = s - w0;
    if (lane == 31) {
      *nitems = s;
      pbase[B] = s;  // the total: pbase[b + 1] - pbase[b] is bucket b's part count
    }
  }
  __syncthreads();
  uint32_t at = red[warp] + (x - local);
  for (uint32_t b = b0; b < b1; ++b) {
    pbase[b] = at;
    at += (uint32_t)((btot[b] + item_keys - 1) / item_keys);
  }
}

// One CTA per bucket: cut the bucket into parts of about item_keys keys along
// the tiles, by a scan of the bucket's per-tile counts (a tile is never
// split; parts differ from item_keys by less than a tile).
__global__ void __launch_bounds__(1024) split_kernel(const uint16_t* __restrict__ toff, uint32_t B,
                                                     uint64_t num_tiles, uint64_t item_keys,
                                                     const uint32_t* __restrict__ pbase, Item* __restrict__ items,
                                                     uint64_t max_items) {
  __shared__ uint32_t red[33];
  const uint32_t b = blockIdx.x, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t base = pbase[b], end = pbase[b + 1];
  if (end <= base || end > max_items) return;  // no parts (or a plan that does not fit: write nothing)
  const uint32_t parts = end - base;
  uint64_t running = 0;
  for (uint64_t c = 0; c < num_tiles; c += 1024) {
    const uint64_t t = c + tid;
    uint32_t cnt = 0;
    if (t < num_tiles) {
      const uint16_t* row = toff + t * (uint64_t)(B + 1);
      cnt = (uint32_t)row[b + 1] - (uint32_t)row[b];
    }
    uint32_t x = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w0 = red[lane];
      uint32_t s = w0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
        if (lane >= (uint32_t)d) s += y;
      }
      red[lane] = s - w0;
      if (lane == 31) red[32] = s;
    }
    __syncthreads();
    const uint64_t lo = running + red[warp] + (x - cnt), hi = lo + cnt;
    if (hi > lo) {
      // parts whose first key falls in this tile start here
      for (uint64_t p = (lo + item_keys - 1) / item_keys; p * item_keys < hi && p < parts; ++p)
        items[base + p] = Item{b, (uint32_t)t, 0u, 0u};
    }
    running += red[32];
    __syncthreads();
  }
  __syncthreads();
  for (uint32_t p = tid; p < parts; p += 1024)
    items[base + p].t1 = (p + 1 < parts) ? items[base + p + 1].t0 : (uint32_t)num_tiles;
}

// ------------------------------------------------------------------ pass 2
// The CTA takes the item's tiles 512 at a time (one per thread): each thread
// reads its tile's segment bounds for this bucket, and a CTA scan turns
// segment lengths in 8-key blocks into one flat block range.  Every warp takes
// an equal slice of that range (lane l: blocks l, l + 32, ...), finds its
// first tile by binary search over the scan and then walks forward, so a few
// very long segments (a hot bucket) keep every warp busy just like many short
// ones.  Each lane keeps kP2Unroll block loads in flight before ingesting.
constexpr uint32_t kP2Threads = 512;
constexpr uint32_t kP2Unroll = 4;

struct BucketSmem {
  uint32_t excl[kP2Threads + 1];   // exclusive block counts of the chunk's tiles
  uint32_t seg0[kP2Threads];       // segment start (tile-relative), per tile
  uint32_t seg1[kP2Threads];       // segment end
  uint32_t red[kP2Threads / 32 + 1];
};

template <int MODE>
__global__ void __launch_bounds__(kP2Threads, 2) bucket_kernel(const uint16_t* __restrict__ low,
                                                               const uint16_t* __restrict__ toff, uint32_t B,
                                                               uint32_t L, uint32_t U, uint32_t* __restrict__ H,
                                                               const Item* __restrict__ items,
                                                               const uint32_t* nitems, uint32_t crn_mode,
                                                               uint32_t words_per_copy, uint32_t* err) {
  extern __shared__ __align__(16) uint32_t sh[];
  __shared__ BucketSmem bs;
  if (blockIdx.x >= *nitems) return;
  const Item it = items[blockIdx.x];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t b_lo = (uint64_t)it.bucket << L;
  const uint32_t Ub = (uint32_t)(((uint64_t)U - b_lo) < (1ull << L) ? ((uint64_t)U - b_lo) : (1ull << L));
  zero_smem(sh, words_per_copy);
  const Sink<MODE> s{sh, H + b_lo, Ub, 0u};
  bool bad = false;
  uint32_t score = 0;
  const uint4* low4 = reinterpret_cast<const uint4*>(low);

  for (uint64_t c = it.t0; c < it.t1; c += kP2Threads) {
    // this thread's tile: segment bounds and length in 8-key blocks
    const uint64_t t = c + tid;
    uint32_t a0 = 0, a1 = 0, nb = 0;
    if (t < it.t1) {
      const uint16_t* row = toff + t * (uint64_t)(B + 1);
      a0 = row[it.bucket];
      a1 = row[it.bucket + 1];
      nb = a1 > a0 ? (a1 + 7) / 8 - a0 / 8 : 0u;
    }
    uint32_t x = nb;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) bs.red[warp] = x;
    __syncthreads();  // also orders the smem histogram's zeroing before the first add
    if (warp == 0) {
      const uint32_t w0 = lane < kP2Threads / 32 ? bs.red[lane] : 0u;
      uint32_t sum = w0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, sum, d);
        if (lane >= (uint32_t)d) sum += y;
      }
      if (lane < kP2Threads / 32) bs.red[lane] = sum - w0;
      if (lane == kP2Threads / 32 - 1) bs.excl[kP2Threads] = sum;
    }
    __syncthreads();
    bs.excl[tid] = bs.red[warp] + (x - nb);
    bs.seg0[tid] = a0;
    bs.seg1[tid] = a1;
    __syncthreads();
    const uint32_t total = bs.excl[kP2Threads];
    const uint32_t ntiles = (it.t1 - c) < kP2Threads ? (uint32_t)(it.t1 - c) : kP2Threads;
    // warp w takes the flat block range [wb0, wb1); lane l starts at block wb0 + l
    const uint32_t per_warp = ((total + kP2Threads / 32 - 1) / (kP2Threads / 32) + 31) & ~31u;
    const uint32_t wb0 = min(warp * per_warp, total), wb1 = min(wb0 + per_warp, total);
    uint32_t tile_i = 0;  // chunk tile holding this lane's next block (found once, then walked)
    {
      const uint32_t j = wb0 + lane;
      uint32_t lo = 0, hi = ntiles - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (bs.excl[mid] <= j)
          lo = mid;
        else
          hi = mid - 1;
      }
      tile_i = lo;
    }
    for (uint32_t j0 = wb0; j0 < wb1; j0 += 32 * kP2Unroll) {
      uint4 q[kP2Unroll];
      uint32_t vm[kP2Unroll];
#pragma unroll
      for (uint32_t u = 0; u < kP2Unroll; ++u) {
        const uint32_t j = j0 + u * 32 + lane;
        vm[u] = 0;
        q[u] = make_uint4(0u, 0u, 0u, 0u);
        if (j < wb1) {
          while (tile_i + 1 < ntiles && bs.excl[tile_i + 1] <= j) ++tile_i;
          const uint32_t s0 = bs.seg0[tile_i], s1 = bs.seg1[tile_i];
          const uint32_t blk_in_tile = s0 / 8 + (j - bs.excl[tile_i]);  // 8-key block within the tile
          const uint32_t p0 = blk_in_tile * 8;                            // its first key, tile-relative
          const uint32_t from = s0 > p0 ? s0 - p0 : 0u;
          const uint32_t to = s1 - p0 < 8 ? s1 - p0 : 8u;
          vm[u] = ((1u << to) - 1u) & ~((1u << from) - 1u);
          q[u] = ld_stream_v4(low4 + ((c + tile_i) * (kP1Tile / 8) + blk_in_tile));
        }
      }
#pragma unroll
      for (uint32_t u = 0; u < kP2Unroll; ++u) {
        const uint32_t k[8] = {q[u].x & 0xffffu, q[u].x >> 16, q[u].y & 0xffffu, q[u].y >> 16,
                               q[u].z & 0xffffu, q[u].z >> 16, q[u].w & 0xffffu, q[u].w >> 16};
        ingest_masked<8, MODE>(k, vm[u], s, Ub, bad, crn_mode, score);
      }
    }
    __syncthreads();  // the chunk's tables are rewritten next round
  }
  if (bad) raise_error(err, ERRBIT_KEY_RANGE);
  __syncthreads();
  flush_smem<MODE>(sh, 1, words_per_copy, Ub, H + b_lo, false);
}

}  // namespace

TwoLevelLayout two_level_layout(uint64_t n, uint32_t U) {
  TwoLevelLayout T;
  uint32_t lg = 0;
  while (lg < 32 && (1ull << lg) < U) ++lg;
  T.L = std::min<uint32_t>(16, std::max<uint32_t>(8, lg > 7 ? lg - 7 : 8));
  T.B = (uint32_t)(((uint64_t)U + (1ull << T.L) - 1) >> T.L);
  T.num_tiles = (n + kP1Tile - 1) / kP1Tile;
  const uint64_t bins = 1ull << T.L;
  // about two items per resident pass-2 CTA (2 per SM on 152 SMs), but at least 8 keys per bin
  T.item_keys = std::max<uint64_t>(std::max<uint64_t>(8 * bins, 65536), n / 608 + 1);
  T.max_items = (n + T.item_keys - 1) / T.item_keys + T.B + 1;
  size_t o = 0;
  T.off_low = o;
  o = align_up(o + 2 * T.num_tiles * kP1Tile, 256);
  T.off_toff = o;
  o = align_up(o + 2 * T.num_tiles * (T.B + 1), 256);
  T.off_btot = o;
  o = align_up(o + 4 * (size_t)T.B, 256);
  T.off_items = o;
  o = align_up(o + sizeof(Item) * T.max_items, 256);
  T.off_nitems = o;
  o = align_up(o + 4, 256);
  T.off_pbase = o;
  o = align_up(o + 4 * ((size_t)T.B + 1), 256);
  T.total = o;
  T.p2_smem32 = bins * 4 <= 64u * 1024u;
  T.words_per_copy = (uint32_t)(T.p2_smem32 ? align_up(bins, 4) : align_up(bins / 2, 4));
  return T;
}

bool two_level_shape_fits(uint64_t n, uint32_t U, uint32_t key_bytes) {
  if (key_bytes != 4 || n < (1u << 20)) return false;
  const TwoLevelLayout T = two_level_layout(n, U);
  return T.B >= 2 && T.B <= 2047;
}

bool two_level_fits(uint64_t n, uint32_t U, uint32_t key_bytes, const void* keys) {
  return (reinterpret_cast<uintptr_t>(keys) & 15u) == 0 && two_level_shape_fits(n, U, key_bytes);
}

cudaError_t launch_two_level(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H, void* ws,
                             const TwoLevelLayout& T, uint32_t crn_mode, const DeviceInfo& dev, uint32_t* err,
                             cudaStream_t stream, bool accumulate) {
  char* base = static_cast<char*>(ws);
  uint16_t* low = reinterpret_cast<uint16_t*>(base + T.off_low);
  uint16_t* toff = reinterpret_cast<uint16_t*>(base + T.off_toff);
  uint32_t* btot = reinterpret_cast<uint32_t*>(base + T.off_btot);
  Item* items = reinterpret_cast<Item*>(base + T.off_items);
  uint32_t* nitems = reinterpret_cast<uint32_t*>(base + T.off_nitems);

  cudaError_t e = cudaMemsetAsync(btot, 0, 4 * (size_t)T.B, stream);
  if (e != cudaSuccess) return e;
  const size_t p1_smem = 4 * (size_t)p1_stage_words(T.B) + 2 * kP1Tile;
  e = cudaFuncSetAttribute(partition_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p1_smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, partition_kernel, kP1Threads, p1_smem);
  if (e != cudaSuccess) return e;
  const uint64_t grid1 = std::min<uint64_t>(T.num_tiles, (uint64_t)dev.sms * std::max(per_sm, 1));
  partition_kernel<<<(unsigned)grid1, kP1Threads, p1_smem, stream>>>(keys, n, U, T.L, T.B, T.num_tiles, low, toff,
                                                                    btot, err, crn_mode);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  uint32_t* pbase = reinterpret_cast<uint32_t*>(base + T.off_pbase);
  plan_kernel<<<1, 1024, 0, stream>>>(btot, T.B, T.item_keys, pbase, nitems);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  split_kernel<<<T.B, 1024, 0, stream>>>(toff, T.B, T.num_tiles, T.item_keys, pbase, items, T.max_items);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (!accumulate) e = cudaMemsetAsync(H, 0, (size_t)U * 4, stream);
  if (e != cudaSuccess) return e;
  const size_t p2_smem = (size_t)T.words_per_copy * 4;
  const uint32_t p2_threads = kP2Threads;
  const void* fn = T.p2_smem32 ? reinterpret_cast<const void*>(&bucket_kernel<MODE_SMEM32>)
                               : reinterpret_cast<const void*>(&bucket_kernel<MODE_SMEM16>);
  if (p2_smem > 48u * 1024u) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p2_smem);
    if (e != cudaSuccess) return e;
  }
  const uint16_t* lowc = low;
  const uint16_t* toffc = toff;
  uint32_t B = T.B, L = T.L, UU = U, crn = crn_mode, wpc = T.words_per_copy;
  const Item* itc = items;
  const uint32_t* nic = nitems;
  void* args[] = {&lowc, &toffc, &B, &L, &UU, &H, &itc, &nic, &crn, &wpc, &err};
  return cudaLaunchKernel(fn, dim3((unsigned)T.max_items), dim3(p2_threads), args, p2_smem, stream);
}

}  // namespace dialsort
