// Two-level ingestion for universes too large for a shared-memory
// sub-histogram: the "hierarchical partitioning" the paper names for large U
// (Sec. "Limitations"), built so that every count still lands in a
// shared-memory counter instead of an L2 atomic (random L2 atomics top out at
// ~0.2 T/s on this GPU, shared-memory atomics at ~3.5 T/s).
//
// A key k splits into a bucket b = k >> L and a low part k & (2^L - 1).
//   pass 1 (partition_kernel)  per 8192-key tile: rank every key within its
//          bucket (one shared-memory atomic per key, or per run of a bucket),
//          scan to bucket starts, write the tile's low parts grouped by bucket
//          (uint16), the tile's bucket starts (toff[t][0..B]) and add the
//          bucket totals up.
//   plan   (plan_kernel, split_kernel)  split every non-empty bucket into
//          parts of about item_keys keys (contiguous tile ranges) -> items.
//   pass 2 (bucket_kernel)     per item: gather the bucket's segments of the
//          item's tiles, count the low parts in a shared-memory histogram of
//          2^L bins (Eq. (1) on the sub-universe; eight equal low parts in a
//          chunk merge into one add, the CRN lane's local accumulation) and
//          add it into H[b * 2^L ...].
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


// Pass-1 counters: one per (bucket, warp), bucket-major with a stride of
// kP1Warps + 1 words, so one bucket's warp counters are contiguous for the
// scan while one warp's buckets spread over all banks for the atomics.  With
// many buckets (B >= kCtaCounters) one counter per bucket for the whole CTA
// instead: 16 columns of counters would crowd out CTAs, and the zeroing and
// scan would grow with them.
constexpr uint32_t kCntStride = kP1Warps + 1;
constexpr uint32_t kCtaCounters = 256;
__host__ __device__ __forceinline__ uint32_t p1_cols(uint32_t B) { return B >= kCtaCounters ? 1u : kP1Warps; }
__host__ __device__ __forceinline__ uint32_t p1_stride(uint32_t B) { return B >= kCtaCounters ? 1u : kCntStride; }

// Pass-1 shared memory, in 32-bit words: the tile's keys (filled by a bulk
// copy), the staged low parts, the counters, the bucket totals, scan scratch
// and the copy's mbarrier.
__host__ __device__ __forceinline__ uint32_t p1_words(uint32_t B) {
  return kP1Tile + kP1Tile / 2 + B * p1_stride(B) + B + 32 + 2;
}

// Polls of a bulk copy's mbarrier before it is given up (each poll waits a while in hardware).
constexpr uint32_t kCopyPolls = 1u << 16;

// ------------------------------------------------------------------ pass 1
// Warp w owns keys [512 w, 512 w + 512) of the tile; lane l takes the four
// 16-byte pieces l, l + 32, l + 64, l + 96 of them (4 consecutive keys each),
// so every shared-memory read of the keys is conflict-free.  Each key takes its
// rank with one shared-memory atomic on its (bucket, warp) counter and keeps
// it in a register; a scan turns the counters into bases, and base + rank is
// the key's slot in the tile's bucket-grouped order.  Runs of one bucket
// within a thread (skew, sorted input, repeated keys) take one atomic per
// run; the warp decides together whether to look for runs.
//
// Data movement is by bulk (1-D TMA) copies: one thread starts the copy of
// the CTA's next 32 KB tile into shared memory as soon as the current tile's
// keys have been read for the last time, so the load overlaps the scan and
// the write-out; the grouped low parts leave by a bulk store.  Keys never
// stay in registers across a barrier, which leaves room for 3 CTAs per SM.
__global__ void __launch_bounds__(kP1Threads, 3) partition_kernel(const uint32_t* __restrict__ keys, uint64_t n,
                                                                   uint32_t U, uint32_t L, uint32_t B,
                                                                   uint64_t num_tiles, uint16_t* __restrict__ low,
                                                                   uint16_t* __restrict__ toff,
                                                                   uint16_t* __restrict__ tcnt,
                                                                   uint32_t* __restrict__ btot, uint32_t* err) {
  extern __shared__ __align__(128) uint32_t sm[];
  uint32_t* kbuf = sm;                                           // [8192] keys of the tile
  uint16_t* stage = reinterpret_cast<uint16_t*>(sm + kP1Tile);   // [8192] grouped low parts
  const uint32_t cols = p1_cols(B), cstride = p1_stride(B);      // counters per bucket, and their stride
  uint32_t* cnt = sm + kP1Tile + kP1Tile / 2;                    // [B][cstride]: counts, then bases
  uint32_t* bacc = cnt + B * cstride;                            // [B]: this CTA's bucket totals
  uint32_t* red = bacc + B;                                      // [32] scan scratch; red[31]: stop flag
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + 32);         // the key copy's mbarrier
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t lowmask = (1u << L) - 1u;
  const uint32_t ncnt = B * cstride;
  const uint32_t col = cols == 1u ? 0u : warp;  // this thread's counter column
  const uint64_t full_tiles = n / kP1Tile;  // tiles loaded by a bulk copy; the ragged last one by plain loads
  bool bad = false;
  uint32_t parity = 0;

  for (uint32_t b = tid; b < B; b += kP1Threads) bacc[b] = 0;
  if (tid == 0) {
    red[31] = 0;
    mbar_init(bar, 1);
    if (blockIdx.x < full_tiles)
      bulk_load(kbuf, keys + (uint64_t)blockIdx.x * kP1Tile, kP1Tile * 4u, bar);
  }
  __syncthreads();

  for (uint64_t t = blockIdx.x; t < num_tiles; t += gridDim.x) {
    if (tid == 0) bulk_wait_read();  // the previous tile's bulk store has read the stage
    for (uint32_t i = tid; i < ncnt; i += kP1Threads) cnt[i] = 0;
    const uint64_t base = t * kP1Tile;
    const uint32_t len = (uint32_t)((n - base) < kP1Tile ? (n - base) : kP1Tile);
    if (t < full_tiles) {
      if (!mbar_wait(bar, parity, kCopyPolls)) red[31] = 1;  // the copy never landed: stop (reported below)
      parity ^= 1u;
    } else {
      for (uint32_t i = tid; i < len; i += kP1Threads) kbuf[i] = keys[base + i];
    }
    __syncthreads();
    if (red[31] != 0) break;  // every thread sees the same flag after the barrier
    // key i of this lane: tile position first + 128 (i / 4) + (i % 4)
    const uint32_t first = kP1Keys * 32u * warp + 4u * lane;
    const bool full = first + 384u + 4u <= len;  // the lane's last piece is whole

    uint32_t kv[kP1Keys];
    const uint4* mine = reinterpret_cast<const uint4*>(kbuf + first);
#pragma unroll
    for (uint32_t i = 0; i < kP1Keys / 4; ++i) {
      const uint4 v = mine[32u * i];
      kv[4 * i] = v.x;
      kv[4 * i + 1] = v.y;
      kv[4 * i + 2] = v.z;
      kv[4 * i + 3] = v.w;
    }
    // bit i of vm: key i is real and < U (all 16 in the common case).  Each key is tested against the
    // universe bound on its own; no two keys are compared with each other.
    bool all_below = true;
#pragma unroll
    for (uint32_t i = 0; i < kP1Keys; ++i) all_below = all_below && kv[i] < U;
    uint32_t vm = 0xffffu;
    if (!full || !all_below) {
      vm = 0;
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i) {
        const bool real = first + 128u * (i / 4) + (i % 4) < len;
        const bool ok = kv[i] < U;
        bad |= real && !ok;
        vm |= (real && ok) ? (1u << i) : 0u;
      }
    }
    // bit i of same: key i continues the bucket of key i - 1
    uint32_t same = 0;
#pragma unroll
    for (uint32_t i = 1; i < kP1Keys; ++i) same |= ((kv[i] >> L) == (kv[i - 1] >> L)) ? (1u << i) : 0u;
    same &= vm & (vm << 1);
    const bool runs = __popc(__ballot_sync(0xffffffffu, same != 0)) >= 16;
    // the whole warp in one bucket (sorted or repeated keys): one atomic for its 512 keys, and ranks laid
    // out so that every stage store below writes 32 consecutive slots
    const uint32_t b0 = __shfl_sync(0xffffffffu, kv[0] >> L, 0);  // in every lane: no short circuit
    const bool one_bucket = __all_sync(0xffffffffu, vm == 0xffffu && same == 0xfffeu && (kv[0] >> L) == b0);

    // ranks, two 16-bit ranks per register (a counter stays below 8192)
    uint32_t rk[kP1Keys / 2];
#pragma unroll
    for (uint32_t i = 0; i < kP1Keys / 2; ++i) rk[i] = 0;
    if (one_bucket) {
      uint32_t r0 = 0;
      if (lane == 0) r0 = atomicAdd(cnt + b0 * cstride + col, kP1Keys * 32u);
      r0 = __shfl_sync(0xffffffffu, r0, 0) + lane;
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i) rk[i / 2] |= (r0 + 32u * i) << (16 * (i & 1));
    } else if (runs) {
      uint32_t r = 0;
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i) {
        if ((vm >> i) & 1u) {
          if (!((same >> i) & 1u))  // a run starts here; its length counts the ones after it
            r = atomicAdd(cnt + (kv[i] >> L) * cstride + col, (uint32_t)__ffs(~(same >> (i + 1))));
          else
            ++r;
        }
        rk[i / 2] |= r << (16 * (i & 1));
      }
    } else if (vm == 0xffffu) {
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i)
        rk[i / 2] |= atomicAdd(cnt + (kv[i] >> L) * cstride + col, 1u) << (16 * (i & 1));
    } else {
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i) {
        const uint32_t r = ((vm >> i) & 1u) ? atomicAdd(cnt + (kv[i] >> L) * cstride + col, 1u) : 0u;
        rk[i / 2] |= r << (16 * (i & 1));
      }
    }
    __syncthreads();

    // bucket-major, warp-minor exclusive scan of the counts -> bases (in place)
    const uint32_t E = cols * B;
    const uint32_t per = (E + kP1Threads - 1) / kP1Threads;
    const uint32_t e0 = min(tid * per, E), e1 = min(e0 + per, E);
    uint32_t local = 0;
    for (uint32_t e = e0; e < e1; ++e) local += cnt[(e / cols) * cstride + e % cols];
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
      uint32_t sum = w0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, sum, d);
        if (lane >= (uint32_t)d) sum += y;
      }
      if (lane < kP1Warps) red[lane] = sum - w0;
      if (lane == kP1Warps - 1) red[kP1Warps] = sum;  // valid keys of the tile
    }
    __syncthreads();
    uint32_t acc = red[warp] + (x - local);
    for (uint32_t e = e0; e < e1; ++e) {
      uint32_t* c = &cnt[(e / cols) * cstride + e % cols];
      const uint32_t v = *c;
      *c = acc;
      acc += v;
    }
    __syncthreads();
    // the tile's bucket starts (warp 0's base), and this CTA's bucket totals
    const uint32_t tile_valid = red[kP1Warps];
    uint16_t* trow = toff + t * (uint64_t)(B + 1);
    for (uint32_t b = tid; b <= B; b += kP1Threads) {
      const uint32_t start = b < B ? cnt[b * cstride] : tile_valid;
      trow[b] = (uint16_t)start;
      if (b < B) {
        const uint32_t c = (b + 1 < B ? cnt[(b + 1) * cstride] : tile_valid) - start;
        bacc[b] += c;
        tcnt[(uint64_t)b * num_tiles + t] = (uint16_t)c;  // bucket-major copy for the split
      }
    }
    // every key to its slot: base of its (bucket, warp) + its rank (keys read again from shared memory)
#pragma unroll
    for (uint32_t i = 0; i < kP1Keys / 4; ++i) {
      const uint4 v = mine[32u * i];
      kv[4 * i] = v.x;
      kv[4 * i + 1] = v.y;
      kv[4 * i + 2] = v.z;
      kv[4 * i + 3] = v.w;
    }
    if (vm == 0xffffu) {
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i) {
        const uint32_t r = (rk[i / 2] >> (16 * (i & 1))) & 0xffffu;
        stage[cnt[(kv[i] >> L) * cstride + col] + r] = (uint16_t)(kv[i] & lowmask);
      }
    } else {
#pragma unroll
      for (uint32_t i = 0; i < kP1Keys; ++i) {
        if ((vm >> i) & 1u) {
          const uint32_t r = (rk[i / 2] >> (16 * (i & 1))) & 0xffffu;
          stage[cnt[(kv[i] >> L) * cstride + col] + r] = (uint16_t)(kv[i] & lowmask);
        }
      }
    }
    fence_proxy_async_smem();  // the stage writes, before the bulk store reads them
    __syncthreads();           // every key has been read: the next tile may land in kbuf
    if (tid == 0) {
      const uint64_t next = t + gridDim.x;
      if (next < full_tiles) bulk_load(kbuf, keys + next * kP1Tile, kP1Tile * 4u, bar);
      // the grouped low parts of tile t: low[t * 8192 ...], rounded up to whole 16-byte pieces
      const uint32_t bytes = ((tile_valid + 7u) / 8u) * 16u;
      if (bytes) bulk_store(low + t * kP1Tile, stage, bytes);
    }
  }
  if (tid == 0) {
    bulk_wait_all();
    if (red[31] != 0) {
      raise_error(err, ERRBIT_TIMEOUT);
      mbar_wait(bar, parity ^ 1u, kCopyPolls);  // give the late copy a last chance to land before exit
    }
  }
  if (bad) raise_error(err, ERRBIT_KEY_RANGE);
  __syncthreads();
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
// the tiles, by a scan of the bucket's per-tile counts (pass 1 keeps them
// bucket-major for this read; a tile is never split; parts differ from
// item_keys by less than a tile).
__global__ void __launch_bounds__(1024) split_kernel(const uint16_t* __restrict__ tcnt, uint32_t B,
                                                     uint64_t num_tiles, uint64_t item_keys,
                                                     const uint32_t* __restrict__ pbase, Item* __restrict__ items,
                                                     uint64_t max_items) {
  __shared__ uint32_t red[33];
  const uint32_t b = blockIdx.x, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t base = pbase[b], end = pbase[b + 1];
  if (end <= base || end > max_items) return;  // no parts (or a plan that does not fit: write nothing)
  const uint32_t parts = end - base;
  // thread tid: tiles [t0, t1) of the bucket's count row, read in one pass
  const uint64_t per = (num_tiles + 1023) / 1024;
  const uint64_t t0 = min((uint64_t)tid * per, num_tiles), t1 = min(t0 + per, num_tiles);
  const uint16_t* row = tcnt + (uint64_t)b * num_tiles;
  uint32_t local = 0;
  for (uint64_t t = t0; t < t1; ++t) local += row[t];
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
    uint32_t sum = w0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, sum, d);
      if (lane >= (uint32_t)d) sum += y;
    }
    red[lane] = sum - w0;
  }
  __syncthreads();
  // parts whose first key falls in tile t start at t
  uint64_t lo = red[warp] + (x - local);
  for (uint64_t t = t0; t < t1; ++t) {
    const uint64_t hi = lo + row[t];
    for (uint64_t p = (lo + item_keys - 1) / item_keys; p * item_keys < hi && p < parts; ++p)
      items[base + p] = Item{b, (uint32_t)t, 0u, 0u};
    lo = hi;
  }
  __syncthreads();
  for (uint32_t p = tid; p < parts; p += 1024)
    items[base + p].t1 = (p + 1 < parts) ? items[base + p + 1].t0 : (uint32_t)num_tiles;
}

// ------------------------------------------------------------------ pass 2
// Two ways to spread an item's chunks (16-byte pieces of its segments) over
// the warps, chosen per item from the mean segment length:
//   short segments (uniform keys: ~17 chunks per tile): warp w takes the
//     item's tiles 32 at a time and lane l walks the segment of tile l chunk
//     by chunk, the warp stepping as long as its longest segment; when that
//     would leave most lanes idle (a few long segments among empty ones),
//     the 32 segments' chunks are numbered flat instead and lane l takes
//     chunks l, l + 32, ..., found by a binary search over the warp's scan;
//   long segments (a hot bucket, sorted or repeated keys): warp w takes
//     tiles w, w + 16, ... and its lanes stride through each segment.
// Either way the lanes stay busy.  Low parts need no range check:
// pass 1 dropped every key >= U.
constexpr uint32_t kP2Threads = 512;
constexpr uint32_t kP2Warps = kP2Threads / 32;
constexpr uint32_t kP2Unroll = 4;
constexpr uint32_t kP2LongSegment = 48;  // mean chunks per tile from which a warp takes one tile at a time

// Count one chunk per lane (all 32 lanes call this together).  A chunk of
// eight equal low parts (a hot or repeated key) is one item (key, 8) -- the
// CRN lane's local accumulation; when some lanes hold such items, equal ones
// are merged across the warp (match.any, the CRN's equality merge) and one
// lane adds their sum, so sorted or repeated keys do not pile 32 lanes onto
// one shared-memory address.
template <int MODE, bool kMerge = true>
__device__ __forceinline__ void count_chunk(const Sink<MODE>& s, const uint4& q, uint32_t vm, uint32_t lane) {
  const uint32_t k[8] = {q.x & 0xffffu, q.x >> 16, q.y & 0xffffu, q.y >> 16,
                         q.z & 0xffffu, q.z >> 16, q.w & 0xffffu, q.w >> 16};
  if (!kMerge) {  // short segments: runs of one low part are rare, plain adds
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i)
      if ((vm >> i) & 1u) s.add(k[i], 1u);
    return;
  }
  const bool same8 = vm == 0xffu && q.x == q.y && q.x == q.z && q.x == q.w && k[0] == k[1];
  const uint32_t m = __ballot_sync(0xffffffffu, same8);
  if (same8) {
    const uint32_t peers = __match_any_sync(m, k[0]);
    if ((peers & ((1u << lane) - 1u)) == 0) s.add(k[0], 8u * (uint32_t)__popc(peers));
  } else {
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i)
      if ((vm >> i) & 1u) s.add(k[i], 1u);
  }
}

// bits [from, to) of the chunk starting at tile position p0 that lie in the segment [a0, a1)
__device__ __forceinline__ uint32_t chunk_mask(uint32_t a0, uint32_t a1, uint32_t p0) {
  const uint32_t from = a0 > p0 ? a0 - p0 : 0u;
  const uint32_t to = a1 - p0 < 8u ? a1 - p0 : 8u;
  return ((1u << to) - 1u) & ~((1u << from) - 1u);
}

template <int MODE>
__global__ void __launch_bounds__(kP2Threads, 2) bucket_kernel(const uint16_t* __restrict__ low,
                                                               const uint16_t* __restrict__ toff, uint32_t B,
                                                               uint32_t L, uint32_t U, uint32_t* __restrict__ H,
                                                               const Item* __restrict__ items,
                                                               const uint32_t* nitems, uint32_t words_per_copy) {
  extern __shared__ __align__(16) uint32_t sh[];
  __shared__ uint32_t s_red[kP2Warps];
  if (blockIdx.x >= *nitems) return;
  const Item it = items[blockIdx.x];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t b_lo = (uint64_t)it.bucket << L;
  const uint32_t Ub = (uint32_t)(((uint64_t)U - b_lo) < (1ull << L) ? ((uint64_t)U - b_lo) : (1ull << L));
  zero_smem(sh, words_per_copy);
  // the item's chunk count, to pick the mapping
  uint32_t mine = 0;
  for (uint64_t t = it.t0 + tid; t < it.t1; t += kP2Threads) {
    const uint16_t* row = toff + t * (uint64_t)(B + 1);
    const uint32_t a0 = row[it.bucket], a1 = row[it.bucket + 1];
    mine += a1 > a0 ? ((a1 + 7u) >> 3) - (a0 >> 3) : 0u;
  }
  mine = __reduce_add_sync(0xffffffffu, mine);
  if (lane == 0) s_red[warp] = mine;
  __syncthreads();
  uint64_t chunks = 0;
#pragma unroll
  for (uint32_t w = 0; w < kP2Warps; ++w) chunks += s_red[w];
  const bool long_segments = chunks >= (uint64_t)kP2LongSegment * (it.t1 - it.t0);
  const Sink<MODE> s{sh, H + b_lo, Ub, 0u};
  const uint4* low4 = reinterpret_cast<const uint4*>(low);

  if (long_segments) {
    for (uint64_t t = it.t0 + warp; t < it.t1; t += kP2Warps) {
      const uint16_t* row = toff + t * (uint64_t)(B + 1);
      const uint32_t a0 = row[it.bucket], a1 = row[it.bucket + 1];
      if (a1 <= a0) continue;
      const uint32_t c_end = (a1 + 7u) >> 3;
      const uint4* tile4 = low4 + t * (uint64_t)(kP1Tile / 8);
      // the loop bound is warp-uniform: count_chunk is a warp collective
      for (uint32_t c0 = a0 >> 3; c0 < c_end; c0 += 32u * kP2Unroll) {
        uint4 q[kP2Unroll];
        uint32_t vm[kP2Unroll];
#pragma unroll
        for (uint32_t u = 0; u < kP2Unroll; ++u) {
          const uint32_t c = c0 + 32u * u + lane;
          vm[u] = 0;
          q[u] = make_uint4(0u, 0u, 0u, 0u);
          if (c < c_end) {
            vm[u] = chunk_mask(a0, a1, c * 8u);
            q[u] = __ldg(tile4 + c);
          }
        }
#pragma unroll
        for (uint32_t u = 0; u < kP2Unroll; ++u) count_chunk<MODE>(s, q[u], vm[u], lane);
      }
    }
  } else {
    for (uint64_t tb = it.t0 + (uint64_t)warp * 32u; tb < it.t1; tb += kP2Warps * 32u) {
      // lane l: the bucket's segment [a0, a1) of tile tb + l and its chunks [a0 / 8, ceil(a1 / 8))
      const uint64_t t = tb + lane;
      uint32_t a0 = 0, a1 = 0;
      if (t < it.t1) {
        const uint16_t* row = toff + t * (uint64_t)(B + 1);
        a0 = row[it.bucket];
        a1 = row[it.bucket + 1];
      }
      const uint32_t c_lo = a0 >> 3;
      const uint32_t nch = a1 > a0 ? ((a1 + 7u) >> 3) - c_lo : 0u;
      uint32_t steps = nch, incl = nch;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) steps = max(steps, __shfl_xor_sync(0xffffffffu, steps, d));
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= (uint32_t)d) incl += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      if (total >= 32u * kP2LongSegment) {
        // long segments in this batch (a hot bucket, sorted runs): the warp takes the 32 tiles one at a
        // time and its lanes stride through each segment, so equal chunks meet in one warp step
        for (uint32_t k = 0; k < 32u; ++k) {
          const uint32_t ka0 = __shfl_sync(0xffffffffu, a0, k), ka1 = __shfl_sync(0xffffffffu, a1, k);
          if (ka1 <= ka0) continue;  // warp-uniform
          const uint32_t c_end = (ka1 + 7u) >> 3;
          const uint4* tile4 = low4 + (tb + k) * (uint64_t)(kP1Tile / 8);
          for (uint32_t c0 = ka0 >> 3; c0 < c_end; c0 += 32u * kP2Unroll) {
            uint4 q[kP2Unroll];
            uint32_t vm[kP2Unroll];
#pragma unroll
            for (uint32_t u = 0; u < kP2Unroll; ++u) {
              const uint32_t c = c0 + 32u * u + lane;
              vm[u] = 0;
              q[u] = make_uint4(0u, 0u, 0u, 0u);
              if (c < c_end) {
                vm[u] = chunk_mask(ka0, ka1, c * 8u);
                q[u] = __ldg(tile4 + c);
              }
            }
#pragma unroll
            for (uint32_t u = 0; u < kP2Unroll; ++u) count_chunk<MODE>(s, q[u], vm[u], lane);
          }
        }
      } else if (2u * total >= 32u * steps) {
        // balanced: each lane walks its own segment (at least half the lanes busy at every step)
        const uint4* tile4 = low4 + (t < it.t1 ? t : it.t0) * (uint64_t)(kP1Tile / 8);
        for (uint32_t i = 0; i < steps; i += kP2Unroll) {  // warp-uniform bound: count_chunk is a warp collective
          uint4 q[kP2Unroll];
          uint32_t vm[kP2Unroll];
#pragma unroll
          for (uint32_t u = 0; u < kP2Unroll; ++u) {
            vm[u] = 0;
            q[u] = make_uint4(0u, 0u, 0u, 0u);
            if (i + u < nch) {
              const uint32_t c = c_lo + i + u;
              vm[u] = chunk_mask(a0, a1, c * 8u);
              q[u] = __ldg(tile4 + c);
            }
          }
#pragma unroll
          for (uint32_t u = 0; u < kP2Unroll; ++u) count_chunk<MODE, false>(s, q[u], vm[u], lane);
        }
      } else {
        // unbalanced (a few long segments among empty ones): number the 32 segments' chunks flat and let
        // lane l take chunks l, l + 32, ..., finding each chunk's tile by a 5-step binary search over the
        // scan held in the lanes
        const uint32_t excl = incl - nch;
        for (uint32_t j0 = 0; j0 < total; j0 += 32u * kP2Unroll) {
          uint4 q[kP2Unroll];
          uint32_t vm[kP2Unroll];
#pragma unroll
          for (uint32_t u = 0; u < kP2Unroll; ++u) {
            const uint32_t j = j0 + u * 32u + lane;
            uint32_t l = 0;  // the last lane with excl_l <= j (lanes without chunks are never it)
#pragma unroll
            for (uint32_t step = 16; step != 0; step >>= 1) {
              const uint32_t e = __shfl_sync(0xffffffffu, excl, l + step);
              if (e <= j) l += step;
            }
            const uint32_t sa = __shfl_sync(0xffffffffu, a0, l);
            const uint32_t sb = __shfl_sync(0xffffffffu, a1, l);
            const uint32_t el = __shfl_sync(0xffffffffu, excl, l);
            vm[u] = 0;
            q[u] = make_uint4(0u, 0u, 0u, 0u);
            if (j < total) {
              const uint32_t c = (sa >> 3) + (j - el);  // chunk within tile tb + l
              vm[u] = chunk_mask(sa, sb, c * 8u);
              q[u] = __ldg(low4 + (tb + l) * (uint64_t)(kP1Tile / 8) + c);
            }
          }
#pragma unroll
          for (uint32_t u = 0; u < kP2Unroll; ++u) count_chunk<MODE>(s, q[u], vm[u], lane);
        }
      }
    }
  }
  __syncthreads();
  flush_smem<MODE>(sh, 1, words_per_copy, Ub, H + b_lo, false);
}

}  // namespace

TwoLevelLayout two_level_layout(uint64_t n, uint32_t U) {
  TwoLevelLayout T;
  uint32_t lg = 0;
  while (lg < 32 && (1ull << lg) < U) ++lg;
  // Low bits per key: 64 buckets up to U = 2^20 and 128 beyond, while the pass-2 histogram (2^L
  // 32-bit counters) still fits 64 KB for two CTAs per SM; past that, packed 16-bit counters.
  T.L = lg <= 20 ? std::min<uint32_t>(14, std::max<uint32_t>(8, lg > 6 ? lg - 6 : 8))
                 : std::min<uint32_t>(16, lg - 7);
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
  T.off_tcnt = o;
  o = align_up(o + 2 * T.num_tiles * T.B, 256);
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
  (void)crn_mode;  // runs are merged by each pass itself
  char* base = static_cast<char*>(ws);
  uint16_t* low = reinterpret_cast<uint16_t*>(base + T.off_low);
  uint16_t* toff = reinterpret_cast<uint16_t*>(base + T.off_toff);
  uint16_t* tcnt = reinterpret_cast<uint16_t*>(base + T.off_tcnt);
  uint32_t* btot = reinterpret_cast<uint32_t*>(base + T.off_btot);
  Item* items = reinterpret_cast<Item*>(base + T.off_items);
  uint32_t* nitems = reinterpret_cast<uint32_t*>(base + T.off_nitems);

  cudaError_t e = cudaMemsetAsync(btot, 0, 4 * (size_t)T.B, stream);
  if (e != cudaSuccess) return e;
  const size_t p1_smem = 4 * (size_t)p1_words(T.B);
  int per_sm = 0;
  e = kernel_config(reinterpret_cast<const void*>(&partition_kernel), kP1Threads, p1_smem, false, &per_sm);
  if (e != cudaSuccess) return e;
  const uint64_t grid1 = std::min<uint64_t>(T.num_tiles, (uint64_t)dev.sms * std::max(per_sm, 1));
  partition_kernel<<<(unsigned)grid1, kP1Threads, p1_smem, stream>>>(keys, n, U, T.L, T.B, T.num_tiles, low, toff,
                                                                    tcnt, btot, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  uint32_t* pbase = reinterpret_cast<uint32_t*>(base + T.off_pbase);
  plan_kernel<<<1, 1024, 0, stream>>>(btot, T.B, T.item_keys, pbase, nitems);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  split_kernel<<<T.B, 1024, 0, stream>>>(tcnt, T.B, T.num_tiles, T.item_keys, pbase, items, T.max_items);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (!accumulate) e = cudaMemsetAsync(H, 0, (size_t)U * 4, stream);
  if (e != cudaSuccess) return e;
  const size_t p2_smem = (size_t)T.words_per_copy * 4;
  const uint32_t p2_threads = kP2Threads;
  const void* fn = T.p2_smem32 ? reinterpret_cast<const void*>(&bucket_kernel<MODE_SMEM32>)
                               : reinterpret_cast<const void*>(&bucket_kernel<MODE_SMEM16>);
  if (p2_smem > 48u * 1024u) {
    e = kernel_config(fn, (int)p2_threads, p2_smem, false, nullptr);
    if (e != cudaSuccess) return e;
  }
  const uint16_t* lowc = low;
  const uint16_t* toffc = toff;
  uint32_t B = T.B, L = T.L, UU = U, wpc = T.words_per_copy;
  const Item* itc = items;
  const uint32_t* nic = nitems;
  void* args[] = {&lowc, &toffc, &B, &L, &UU, &H, &itc, &nic, &wpc};
  return cudaLaunchKernel(fn, dim3((unsigned)T.max_items), dim3(p2_threads), args, p2_smem, stream);
}

}  // namespace dialsort
