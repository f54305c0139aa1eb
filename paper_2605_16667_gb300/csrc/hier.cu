// Two-level ingestion for universes of up to 2^21 bins: the "hierarchical
// partitioning" the paper names for large U (Sec. "Limitations"), shaped so
// that every count of Eq. (1) still lands in a shared-memory counter.
//
// A key k splits into a bucket b = k >> 15 and a low part k & (2^15 - 1);
// there are B = ceil(U / 2^15) <= 64 buckets.
//
//   pass 1 (hier_partition_kernel)  per 8192-key tile: count the tile's keys
//          per (bucket, lane) -- lane = the thread's lane within its warp, so
//          the 32 lanes of a warp never touch the same counter and every
//          counter access is conflict-free -- scan the counts into stage
//          slots (each bucket's segment starts on a 16-byte boundary), then
//          let every key take its slot with one atomic on its (bucket, lane)
//          cursor and store its low 16 bits there.  A warp whose 512 keys all
//          fall in one bucket (sorted runs, a repeated key) takes one cursor
//          step for all of them and stores them contiguously.  The staged
//          tile leaves by one bulk (TMA) store; seg[b][t] records where each
//          bucket's segment starts and how long it is.  The next tile's keys
//          are loaded while the current one is counted and placed.
//   split  (hier_split_kernel)  cuts the bucket-major sequence of segments
//          into one range per pass-2 CTA, each holding about n / G keys.
//   pass 2 (hier_count_kernel)  per range: a 2^15-bin shared-memory
//          histogram per bucket (Eq. (1) on the sub-universe), flushed into
//          H[b << 15 ...] by a bulk reduce-add (or bin by bin when few bins
//          are non-zero).  Eight equal low parts in one 16-byte chunk count
//          as one item (key, 8), and a lane keeps a running (key, count) pair
//          for repeated chunks: the local accumulation of a CRN lane (Sec.
//          "CRN Lane States"), so a hot key does not become a stream of adds
//          on one shared-memory word.
//
// Only shifts, masks and equality touch keys; the one magnitude test is key <
// U against the universe bound (for U a power of two, on the bitwise OR of a
// thread's keys).  Counting is exact: pass 1 only moves keys.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "recon_device.cuh"

namespace dialsort {

namespace {

constexpr uint32_t kLow = 15;                 // low bits per key
constexpr uint32_t kTile = 8192;              // keys per pass-1 tile
constexpr uint32_t kP1Threads = 512;
constexpr uint32_t kP1Warps = kP1Threads / 32;
constexpr uint32_t kKeysPerThread = kTile / kP1Threads;  // 16
constexpr uint32_t kP2Threads = 1024;
constexpr uint32_t kInvalid = 0xffffffffu;
constexpr uint32_t kMaxBuckets = 64;

__device__ __forceinline__ void red_s32(uint32_t a, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_s32(uint32_t a, uint32_t v) {
  uint32_t r;
  asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(r) : "r"(a), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ void st_s16(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"((uint16_t)v) : "memory");
}

// Pass-1 shared memory for BM bucket slots (BM = 32 or 64).
template <int BM>
struct P1Smem {
  uint32_t cnt[BM][32];  // keys per (bucket, lane) in this tile; zeroed by the scan
  uint32_t pos[BM][32];  // next stage slot per (bucket, lane)
  uint32_t agg[BM];      // keys of whole-warp (single-bucket) groups
  uint32_t aggpos[BM];   // next stage slot of the whole-warp part
  uint32_t tot[BM];      // keys per bucket in this tile
  uint32_t bacc[BM];     // this CTA's keys per bucket
  __align__(16) uint16_t stage[kTile + 8 * BM];
};

// Key quad j of this thread: keys [4 (128 w + 32 j + l), +4) of the tile (warp w, lane l);
// INVALID past n.
__device__ __forceinline__ void load_tile(const uint32_t* __restrict__ keys, uint64_t n, uint64_t t, uint32_t warp,
                                          uint32_t lane, uint4 (&kq)[4]) {
  const uint64_t p0 = t * kTile + (uint64_t)(warp * 128u + lane) * 4u;
  const uint4* q = reinterpret_cast<const uint4*>(keys + p0);
  if (p0 + 384u + 4u <= n) {
#pragma unroll
    for (int j = 0; j < 4; ++j) kq[j] = ld_stream_v4(q + 32 * j);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t p = p0 + 128u * j;
      if (p + 4 <= n) {
        kq[j] = ld_stream_v4(q + 32 * j);
      } else {
        kq[j].x = p < n ? keys[p] : kInvalid;
        kq[j].y = p + 1 < n ? keys[p + 1] : kInvalid;
        kq[j].z = p + 2 < n ? keys[p + 2] : kInvalid;
        kq[j].w = p + 3 < n ? keys[p + 3] : kInvalid;
      }
    }
  }
}

__device__ __forceinline__ uint32_t key_of(const uint4 (&kq)[4], int i) { return (&kq[i / 4].x)[i % 4]; }

template <int BM, bool POW2>
__global__ void __launch_bounds__(kP1Threads, 3) hier_partition_kernel(
    const uint32_t* __restrict__ keys, uint64_t n, uint32_t U, uint32_t B, uint64_t num_tiles, uint32_t S_t,
    uint16_t* __restrict__ low, uint32_t* __restrict__ seg, uint32_t* __restrict__ btot, uint32_t* err) {
  __shared__ P1Smem<BM> s;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  for (uint32_t i = tid; i < BM * 32u; i += kP1Threads) (&s.cnt[0][0])[i] = 0;
  for (uint32_t i = tid; i < (uint32_t)BM; i += kP1Threads) {
    s.agg[i] = 0;
    s.bacc[i] = 0;
  }
  const uint32_t cnt_a = smem_addr(&s.cnt[0][lane]);
  const uint32_t pos_a = smem_addr(&s.pos[0][lane]);
  const uint32_t stage_a = smem_addr(s.stage);
  bool bad = false;
  uint4 kc[4];
  uint64_t t = blockIdx.x;
  if (t < num_tiles) load_tile(keys, n, t, warp, lane, kc);
  __syncthreads();
  while (t < num_tiles) {
    const uint64_t tn = t + gridDim.x;
    const uint32_t len = (uint32_t)min((uint64_t)kTile, n - t * kTile);
    // Are all 16 keys of this thread real and below U?  Do they share one bucket?
    const uint32_t k0 = kc[0].x;
    uint32_t xo = 0, oo = 0;
#pragma unroll
    for (int i = 0; i < (int)kKeysPerThread; ++i) {
      xo |= key_of(kc, i) ^ k0;
      if (POW2) oo |= key_of(kc, i);
    }
    bool fast = len == kTile;
    if (POW2) {
      fast = fast && oo < U;  // U a power of two: the OR is below U exactly when every key is
    } else {
#pragma unroll
      for (int i = 0; i < (int)kKeysPerThread; ++i) fast = fast && key_of(kc, i) < U;
    }
    const uint32_t b0 = k0 >> kLow;
    const bool warp_one = __all_sync(0xffffffffu, fast && (xo >> kLow) == 0) && __shfl_sync(0xffffffffu, b0, 0) == b0;

    // ---- count
    if (warp_one) {
      if (lane == 0) red_s32(smem_addr(&s.agg[b0]), kKeysPerThread * 32u);
    } else if (fast) {
#pragma unroll
      for (int i = 0; i < (int)kKeysPerThread; ++i) red_s32(cnt_a + ((key_of(kc, i) >> kLow) << 7), 1u);
    } else {
#pragma unroll
      for (int i = 0; i < (int)kKeysPerThread; ++i) {
        const uint32_t key = key_of(kc, i);
        const uint32_t p = (warp * 128u + (i / 4) * 32u + lane) * 4u + (i % 4);
        const bool real = p < len, ok = key < U;
        bad |= real && !ok;
        if (real && ok) red_s32(cnt_a + ((key >> kLow) << 7), 1u);
      }
    }
    __syncthreads();
    if (tid == 0) bulk_wait_read();  // the previous tile's bulk store has read the stage
    // ---- in-bucket offsets: warp w scans the lanes' counts of buckets w, w + 16, ...
    for (uint32_t b = warp; b < B; b += kP1Warps) {
      const uint32_t c = s.cnt[b][lane];
      s.cnt[b][lane] = 0;
      uint32_t x = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= (uint32_t)d) x += y;
      }
      s.pos[b][lane] = x - c;
      if (lane == 31) {
        const uint32_t a = s.agg[b];
        s.agg[b] = 0;
        s.aggpos[b] = x;  // whole-warp keys follow the per-lane ones
        s.tot[b] = x + a;
      }
    }
    __syncthreads();
    // ---- bucket starts (each rounded up to 8 slots), in every warp: lane j holds buckets j and j + 32
    const uint32_t t0 = lane < B ? s.tot[lane] : 0u;
    const uint32_t t1 = (BM > 32 && lane + 32u < B) ? s.tot[lane + 32] : 0u;
    const uint32_t p0 = (t0 + 7u) & ~7u, p1 = (t1 + 7u) & ~7u;
    uint32_t x0 = p0, x1 = p1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y0 = __shfl_up_sync(0xffffffffu, x0, d);
      const uint32_t y1 = __shfl_up_sync(0xffffffffu, x1, d);
      if (lane >= (uint32_t)d) {
        x0 += y0;
        x1 += y1;
      }
    }
    const uint32_t sum0 = __shfl_sync(0xffffffffu, x0, 31);
    const uint32_t bb0 = x0 - p0, bb1 = sum0 + x1 - p1;
    const uint32_t padded_total = sum0 + __shfl_sync(0xffffffffu, x1, 31);
    for (uint32_t b = warp; b < B; b += kP1Warps) {
      const uint32_t bb = __shfl_sync(0xffffffffu, b < 32 ? bb0 : bb1, b & 31u);
      s.pos[b][lane] += bb;
      if (lane == 31) s.aggpos[b] += bb;
    }
    if (warp == 0) {
      if (lane < B) {
        seg[(uint64_t)lane * num_tiles + t] = (bb0 >> 3) | (t0 << 16);
        s.bacc[lane] += t0;
      }
      if (BM > 32 && lane + 32u < B) {
        seg[(uint64_t)(lane + 32) * num_tiles + t] = (bb1 >> 3) | (t1 << 16);
        s.bacc[lane + 32] += t1;
      }
    }
    __syncthreads();
    // ---- place: the cursor atomic returns each key's stage slot
    if (warp_one) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&s.aggpos[b0], kKeysPerThread * 32u);
      base = __shfl_sync(0xffffffffu, base, 0) + lane;
#pragma unroll
      for (int i = 0; i < (int)kKeysPerThread; ++i) st_s16(stage_a + (base + 32u * i) * 2u, key_of(kc, i));
    } else if (fast) {
#pragma unroll
      for (int i = 0; i < (int)kKeysPerThread; ++i) {
        const uint32_t key = key_of(kc, i);
        st_s16(stage_a + atom_s32(pos_a + ((key >> kLow) << 7), 1u) * 2u, key);
      }
    } else {
#pragma unroll
      for (int i = 0; i < (int)kKeysPerThread; ++i) {
        const uint32_t key = key_of(kc, i);
        const uint32_t p = (warp * 128u + (i / 4) * 32u + lane) * 4u + (i % 4);
        if (p < len && key < U) st_s16(stage_a + atom_s32(pos_a + ((key >> kLow) << 7), 1u) * 2u, key);
      }
    }
    fence_proxy_async_smem();  // the stage writes, before the bulk store reads them
    __syncthreads();
    if (tid == 0 && padded_total) bulk_store(low + t * S_t, s.stage, padded_total * 2u);
    if (tn < num_tiles) load_tile(keys, n, tn, warp, lane, kc);  // (three CTAs per SM hide the load latency)
    t = tn;
  }
  if (tid == 0) bulk_wait_all();
  if (bad) raise_error(err, ERRBIT_KEY_RANGE);
  __syncthreads();
  for (uint32_t b = tid; b < B; b += kP1Threads)
    if (s.bacc[b]) red_add_global(btot + b, s.bacc[b]);
}

// Work of pass 2, in key-equivalents: every key, plus a fixed cost per
// segment visited (reading its word, the window scan) and per non-empty
// bucket (zeroing and flushing a 2^15-bin histogram).  Ranges balanced by keys
// alone would hand one CTA every light bucket of a skewed input.
constexpr uint64_t kSegCost = 64;
constexpr uint64_t kBucketCost = 1u << 15;

__device__ __forceinline__ uint64_t bucket_cost(uint64_t nb, uint64_t num_tiles) {
  return nb ? nb + kSegCost * num_tiles + kBucketCost : 0;
}

// One CTA per bucket.  Pass-2 CTA k starts at the segment (b * num_tiles + t)
// where the cumulative work of the bucket-major segment order reaches
// floor(k W / G), W the total work.  Writes start[k] for every k whose target
// lies in this bucket; CTA 0 also writes start[0] and start[G].
__global__ void __launch_bounds__(1024) hier_split_kernel(const uint32_t* __restrict__ seg,
                                                          const uint32_t* __restrict__ btot, uint32_t B,
                                                          uint64_t num_tiles, uint32_t G,
                                                          uint64_t* __restrict__ start) {
  __shared__ uint64_t red[33];
  __shared__ uint64_t sP, sW;
  const uint32_t b = blockIdx.x, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (tid == 0) {
    uint64_t P = 0, W = 0;
    for (uint32_t j = 0; j < B; ++j) {
      const uint64_t c = bucket_cost(btot[j], num_tiles);
      if (j < b) P += c;
      W += c;
    }
    sP = P;
    sW = W;
    if (b == 0) {
      start[0] = 0;
      start[G] = (uint64_t)B * num_tiles;
      if (W == 0)
        for (uint32_t k = 1; k < G; ++k) start[k] = 0;  // nothing counted: every range is empty but the last
    }
  }
  __syncthreads();
  const uint64_t W = sW, nb = btot[b];
  if (W == 0 || nb == 0) return;
  const uint64_t P = sP + kBucketCost;  // the bucket's fixed cost comes first
  const uint64_t cb = bucket_cost(nb, num_tiles);
  uint64_t k_lo = (sP * G + W - 1) / W;                              // first k with floor(k W / G) >= sP
  const uint64_t k_hi = min((uint64_t)G, ((sP + cb) * G + W - 1) / W);  // first k at or past the bucket's end
  if (k_lo < 1) k_lo = 1;
  if (k_lo >= k_hi) return;
  // thread tid: a run of consecutive tiles
  const uint64_t per = (num_tiles + 1023) / 1024;
  const uint64_t ta = min((uint64_t)tid * per, num_tiles), tb = min(ta + per, num_tiles);
  const uint32_t* row = seg + (uint64_t)b * num_tiles;
  uint64_t local = 0;
  for (uint64_t t = ta; t < tb; ++t) local += (row[t] >> 16) + kSegCost;
  uint64_t x = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint64_t w0 = red[lane];
    uint64_t s2 = w0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, s2, d);
      if (lane >= (uint32_t)d) s2 += y;
    }
    red[lane] = s2 - w0;
  }
  __syncthreads();
  const uint64_t lo = P + red[warp] + (x - local), hi = lo + local;
  // targets before the bucket's first tile (inside its fixed cost) start at tile 0
  uint64_t k = k_lo;
  if (tid == 0)
    for (; k < k_hi && k * W / G < lo; ++k) start[k] = (uint64_t)b * num_tiles;
  if (hi <= lo) return;
  k = max(k_lo, (lo * G + W - 1) / W);
  uint64_t acc = lo, t = ta;
  for (; k < k_hi; ++k) {
    const uint64_t target = k * W / G;
    if (target >= hi) break;
    while (t < tb && acc + (row[t] >> 16) + kSegCost <= target) {
      acc += (row[t] >> 16) + kSegCost;
      ++t;
    }
    start[k] = (uint64_t)b * num_tiles + t;
  }
}

// A bucket holding more than kSharedShare / G of the keys is counted by many
// pass-2 CTAs; their histograms then go to private scratch slots (bulk stores)
// and hier_merge_kernel sums them, instead of many bulk reduce-adds meeting on
// the same lines of H.
constexpr uint64_t kSharedShare = 8;

__device__ __forceinline__ bool shared_bucket(uint64_t nb, uint64_t N, uint32_t G) { return nb * G > kSharedShare * N; }

// Pass-2 shared memory besides the 2^15-bin histogram (dynamic).
struct P2Smem {
  uint32_t wred[kP2Threads / 32];
  uint32_t cpre[kP2Threads + 2];  // first chunk of each non-empty segment of the window, then the window's
                                  // chunk count and a sentinel
  uint32_t csw[kP2Threads];       // their segment words
  uint16_t ctile[kP2Threads];     // their tiles, relative to the window
};

// Counts the low parts of bucket b in tiles [ta, tb) into hist (zeroed here, 2^15 bins).  On return hist
// is complete, visible to the whole CTA and fenced for a bulk copy to read it.  Windows of up to 1024
// tiles: one block scan numbers the window's non-empty segments and their chunks (16-byte pieces, 8 low
// parts each) flat; every warp then takes an equal contiguous range of chunks.  Within a warp step lane
// l takes chunk j0 + l: the segment boundaries falling inside the step are gathered into a 32-bit mask
// (one boundary per lane, redux.or), and a popcount of the mask below bit l gives the lane's segment.
__device__ __forceinline__ void count_piece(const uint16_t* __restrict__ low, const uint32_t* __restrict__ seg,
                                            uint32_t b, uint64_t ta, uint64_t tb, uint64_t num_tiles, uint32_t S_t,
                                            uint32_t* hist, P2Smem& sm) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  constexpr uint32_t bins = 1u << kLow;
  for (uint32_t i = tid * 4u; i < bins; i += kP2Threads * 4u) *reinterpret_cast<uint4*>(hist + i) = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  // a stored low part is the key's low 16 bits: bit 15 is the bucket's low bit
  const uint32_t hb_a = smem_addr(hist) - ((b & 1u) << kLow) * 4u;
  const uint32_t* row = seg + (uint64_t)b * num_tiles;
  uint32_t rkey = 0, rcnt = 0;
  for (uint64_t w0 = ta; w0 < tb; w0 += kP2Threads) {
    const uint32_t nw = (uint32_t)min((uint64_t)kP2Threads, tb - w0);
    const uint32_t sgw = tid < nw ? row[w0 + tid] : 0u;
    const uint32_t ch = ((sgw >> 16) + 7u) >> 3;
    const uint32_t packed = (ch << 11) | (ch ? 1u : 0u);  // chunks (21 bits) | non-empty segments (11 bits)
    uint32_t x = packed;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= (uint32_t)d) x += y;
    }
    __syncthreads();  // the previous window's tables are no longer read
    if (lane == 31) sm.wred[warp] = x;
    __syncthreads();
    uint32_t wbase = 0, total = 0;
    for (uint32_t w = 0; w < kP2Threads / 32; ++w) {
      const uint32_t v = sm.wred[w];
      if (w < warp) wbase += v;
      total += v;
    }
    const uint32_t excl = wbase + x - packed;
    if (ch) {
      const uint32_t i = excl & 0x7ffu;
      sm.cpre[i] = excl >> 11;
      sm.csw[i] = sgw;
      sm.ctile[i] = (uint16_t)tid;
    }
    const uint32_t nnz = total & 0x7ffu, nch = total >> 11;
    if (tid == 0) sm.cpre[nnz] = nch;
    if (tid == 1) sm.cpre[nnz + 1] = 0xffffffffu;  // sentinel past the last boundary
    __syncthreads();
    const uint32_t j_lo = (uint32_t)((uint64_t)nch * warp / (kP2Threads / 32));
    const uint32_t j_hi = (uint32_t)((uint64_t)nch * (warp + 1) / (kP2Threads / 32));
    if (j_lo >= j_hi) continue;
    // the segment holding chunk j_lo: the last e with cpre[e] <= j_lo (same in every lane)
    uint32_t e = 0;
    for (uint32_t step = kP2Threads / 2; step != 0; step >>= 1)
      if (e + step < nnz && sm.cpre[e + step] <= j_lo) e += step;
    constexpr int F = 4;  // chunks in flight per lane
    for (uint32_t j0 = j_lo; j0 < j_hi; j0 += 32u * F) {  // warp-uniform bound
      uint4 q[F];
      uint32_t nh[F];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const uint32_t jf = j0 + 32u * f, j = jf + lane;
        // boundaries cpre[e + 1 + k] (k = lane) inside [jf, jf + 32) -> mask bits; cpre[e + 1] >= jf
        const uint32_t bk = sm.cpre[min(e + 1u + lane, nnz + 1u)] - jf;
        const uint32_t m = __reduce_or_sync(0xffffffffu, bk < 32u ? 1u << bk : 0u);
        const uint32_t idx = e + __popc(m & (0xffffffffu >> (31u - lane)));
        e = __shfl_sync(0xffffffffu, idx, 31);
        q[f] = make_uint4(0u, 0u, 0u, 0u);
        nh[f] = 0;
        if (j < j_hi) {
          const uint32_t sgu = sm.csw[idx], c = j - sm.cpre[idx], cnt = sgu >> 16;
          nh[f] = cnt - c * 8u >= 8u ? 8u : cnt - c * 8u;
          q[f] = ld_stream_v4(
              reinterpret_cast<const uint4*>(low + (w0 + sm.ctile[idx]) * (uint64_t)S_t + (sgu & 0xffffu) * 8u) + c);
        }
      }
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const uint4 w = q[f];
        // eight equal low parts: one item (key, 8), accumulated in the lane while the key repeats
        if (nh[f] == 8u && w.x == w.y && w.x == w.z && w.x == w.w && (w.x & 0xffffu) == (w.x >> 16)) {
          if (w.x != rkey) {
            if (rcnt) red_s32(hb_a + (rkey & 0xffffu) * 4u, rcnt);
            rkey = w.x;
            rcnt = 0;
          }
          rcnt += 8u;
        } else if (nh[f] == 8u) {
          red_s32(hb_a + (w.x & 0xffffu) * 4u, 1u);
          red_s32(hb_a + (w.x >> 16) * 4u, 1u);
          red_s32(hb_a + (w.y & 0xffffu) * 4u, 1u);
          red_s32(hb_a + (w.y >> 16) * 4u, 1u);
          red_s32(hb_a + (w.z & 0xffffu) * 4u, 1u);
          red_s32(hb_a + (w.z >> 16) * 4u, 1u);
          red_s32(hb_a + (w.w & 0xffffu) * 4u, 1u);
          red_s32(hb_a + (w.w >> 16) * 4u, 1u);
        } else if (nh[f]) {
          const uint32_t k[8] = {w.x & 0xffffu, w.x >> 16, w.y & 0xffffu, w.y >> 16,
                                 w.z & 0xffffu, w.z >> 16, w.w & 0xffffu, w.w >> 16};
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if ((uint32_t)i < nh[f]) red_s32(hb_a + k[i] * 4u, 1u);
        }
      }
    }
  }
  if (rcnt) red_s32(hb_a + (rkey & 0xffffu) * 4u, rcnt);
  fence_proxy_async_smem();  // the histogram, before a bulk copy reads it
  __syncthreads();
}

// Adds hist (bins [0, Ub) of bucket b) into H[b 2^15 ...]: bin by bin when few bins are non-zero, else
// whole 16-byte pieces by four bulk reduce-adds (issued by threads 0-3, which then have a bulk group in
// flight) and the ragged end bin by bin.
__device__ __forceinline__ void flush_piece(const uint32_t* hist, uint32_t Ub, uint32_t* __restrict__ Hb,
                                            uint32_t* wred) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  uint32_t nz = 0;
  for (uint32_t i = tid; i < Ub; i += kP2Threads) nz += hist[i] != 0u;
  nz = __reduce_add_sync(0xffffffffu, nz);
  if (lane == 0) wred[warp] = nz;
  __syncthreads();
  nz = 0;
#pragma unroll
  for (uint32_t w = 0; w < kP2Threads / 32; ++w) nz += wred[w];
  if (nz * 16u <= Ub) {
    // few distinct keys (a hot bucket shared by many CTAs): add the non-zero bins one by one
    for (uint32_t i = tid; i < Ub; i += kP2Threads)
      if (hist[i]) red_add_global(Hb + i, hist[i]);
  } else {
    const uint32_t body = Ub & ~3u;
    if (tid < 4) {
      const uint32_t piece = (body / 4u) & ~3u;
      const uint32_t a = piece * tid, z = tid == 3 ? body : piece * (tid + 1);
      if (z > a) bulk_reduce_add_u32(Hb + a, hist + a, (z - a) * 4u);
    }
    for (uint32_t i = body + tid; i < Ub; i += kP2Threads)
      if (hist[i]) red_add_global(Hb + i, hist[i]);
  }
}

__global__ void __launch_bounds__(kP2Threads, 1) hier_count_kernel(
    const uint16_t* __restrict__ low, const uint32_t* __restrict__ seg, const uint64_t* __restrict__ start,
    const uint32_t* __restrict__ btot, uint32_t B, uint32_t U, uint64_t num_tiles, uint32_t S_t,
    uint32_t* __restrict__ H, uint32_t* __restrict__ part, uint32_t* __restrict__ part_used) {
  extern __shared__ __align__(128) uint32_t hist[];  // 2^15 bins
  __shared__ P2Smem sm;
  const uint32_t tid = threadIdx.x;
  constexpr uint32_t bins = 1u << kLow;
  uint64_t s = start[blockIdx.x];
  const uint64_t se = min(start[blockIdx.x + 1], (uint64_t)B * num_tiles);
  uint64_t N = 0;
  for (uint32_t j = 0; j < B; ++j) N += btot[j];
  bool pending = false;  // a bulk copy may still be reading hist
  while (s < se) {
    const uint32_t b = (uint32_t)(s / num_tiles);
    const uint64_t ta = s - (uint64_t)b * num_tiles;
    const uint64_t tb = min(num_tiles, ta + (se - s));
    s += tb - ta;
    if (btot[b] == 0) continue;  // an empty bucket (the same value in every thread)
    if (pending && tid < 4) bulk_wait_read();
    __syncthreads();
    count_piece(low, seg, b, ta, tb, num_tiles, S_t, hist, sm);
    const uint64_t blo = (uint64_t)b << kLow;
    const uint32_t Ub = (uint32_t)min((uint64_t)bins, (uint64_t)U - blo);
    if (shared_bucket(btot[b], N, gridDim.x)) {
      // scratch slot blockIdx.x + b: each (CTA, bucket) piece has its own (ranges are monotone in the bucket)
      const uint32_t slot = blockIdx.x + b;
      if (tid < 4) {
        bulk_store(part + (uint64_t)slot * bins + tid * (bins / 4), hist + tid * (bins / 4), bins);  // bins / 4 words
        pending = true;
      }
      if (tid == 0) part_used[slot] = b + 1u;  // slots of neighbouring buckets interleave: tag the bucket
      continue;
    }
    flush_piece(hist, Ub, H + blo, sm.wred);
    pending = true;
  }
  if (tid < 4) bulk_wait_all();
}

// Sums the scratch histograms of every shared bucket into H: CTA (b, c) takes
// bins [1024 c, 1024 c + 1024) of bucket b; the pieces of bucket b sit in slots
// i + b of the pass-2 CTAs i that counted part of it, each tagged b + 1 (the
// slot i + b of a CTA that counted another bucket b' carries the tag b' + 1).
__global__ void __launch_bounds__(256) hier_merge_kernel(const uint32_t* __restrict__ btot, uint32_t B, uint32_t U,
                                                         uint32_t G, const uint32_t* __restrict__ part,
                                                         const uint32_t* __restrict__ part_used,
                                                         uint32_t* __restrict__ H) {
  constexpr uint32_t bins = 1u << kLow;
  const uint32_t b = blockIdx.x, c = blockIdx.y, tid = threadIdx.x;
  __shared__ uint64_t sN;
  if (tid == 0) {
    uint64_t N = 0;
    for (uint32_t j = 0; j < B; ++j) N += btot[j];
    sN = N;
  }
  __syncthreads();
  if (!shared_bucket(btot[b], sN, G)) return;
  const uint64_t blo = (uint64_t)b << kLow;
  const uint32_t i0 = c * 1024u + tid * 4u;  // four bins per thread
  const uint32_t Ub = (uint32_t)min((uint64_t)bins, (uint64_t)U - blo);
  if (i0 >= Ub) return;
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  for (uint32_t i = 0; i < G; ++i) {
    if (part_used[i + b] != b + 1u) continue;  // slot i + b may hold a piece of another bucket
    const uint4 v = *reinterpret_cast<const uint4*>(part + (uint64_t)(i + b) * bins + i0);
    acc.x += v.x;
    acc.y += v.y;
    acc.z += v.z;
    acc.w += v.w;
  }
  const uint32_t a[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (i0 + j < Ub) H[blo + i0 + j] += a[j];  // the only writer of these bins
}

// ---------------------------------------------------------------- sort: counting fused with the projection
//
// For a sort, pass 2 and the projection (Eq. (2)) run in one persistent kernel whose CTAs take work
// items in one ticket order: count ranges of the bucket-major segment sequence (pass 2 as above, every
// piece reduce-added into H), interleaved with projection items -- one 1024-bin chunk of H each, which
// writes the chunk's runs of the output.  A bucket's projection items are placed after the last count
// range that touches the bucket (plus a delay of one grid's worth of tickets), so earlier buckets are
// projected while later ones are still being counted: the output writes overlap the low-part reads.
// A projection item waits (bounded) until every piece of its bucket has been added into H, then finds
// its chunk's start by decoupled look-back over the bucket's earlier chunks (a bucket's first key lands
// at the sum of the earlier buckets' keys, known from pass 1).  Every wait is for items with smaller
// tickets, which running CTAs hold: the waits end whatever the number of resident CTAs.
constexpr uint32_t kFusedMaxRanges = 1024;
constexpr uint32_t kChunksPerBucket = (1u << kLow) / kChunkBins;  // 32
constexpr uint32_t kFusedMaxChunks = kMaxBuckets * kChunksPerBucket;
constexpr uint32_t kProjItem = 0x80000000u;
constexpr uint32_t kNoItem = 0xffffffffu;

struct FusedCtl {
  uint32_t ticket;
  uint32_t nsched;
  uint32_t nlong;    // runs longer than kWarpRun keys, left to hier_long_kernel
  uint32_t npieces;  // their pieces of kLongPiece keys
};

// A run of more than kWarpRun keys (a hot key) is not painted by the chunk item's warp: one warp (one
// SM) would write it alone.  It goes to a list instead, cut into pieces of kLongPiece keys that
// hier_long_kernel paints with every SM after the fused kernel.  A chunk holding more than kChunkBudget
// keys (skewed keys: thousands of runs of thousands of keys) lists every run of more than kListRun keys,
// so that no chunk item writes more than about kChunkBudget keys itself.
constexpr uint32_t kWarpRun = 8192;
constexpr uint32_t kListRun = 512;
constexpr uint32_t kChunkBudget = 1u << 20;
constexpr uint32_t kLongPiece = 32768;
struct LongRun {
  uint32_t start, len, key, piece0;
};

// One CTA: pieces[b] (count ranges that touch non-empty bucket b), bbase[b] (keys of buckets < b), and the
// item order sched[0 .. nsched): range k as k, chunk c of the projection as kProjItem | c.
__global__ void __launch_bounds__(1024) hier_sched_kernel(const uint64_t* __restrict__ start, uint32_t K,
                                                          const uint32_t* __restrict__ btot, uint32_t B, uint32_t U,
                                                          uint64_t num_tiles, uint32_t delay, uint32_t* sched,
                                                          uint32_t* pieces, uint64_t* bbase, FusedCtl* ctl) {
  __shared__ uint32_t s_r[kMaxBuckets], s_nch[kMaxBuckets], s_off[kMaxBuckets], s_bt[kMaxBuckets];
  __shared__ uint64_t s_start[kFusedMaxRanges + 1];
  const uint32_t tid = threadIdx.x;
  for (uint32_t k = tid; k <= K; k += blockDim.x) s_start[k] = start[k];  // one round trip, then shared memory
  if (tid < B) s_bt[tid] = btot[tid];
  __syncthreads();
  if (tid < B) {
    const uint32_t b = tid;
    const uint64_t lo = (uint64_t)b * num_tiles, hi = lo + num_tiles;
    uint32_t l = 0, r = K;  // first range whose end lies past the bucket's first tile
    while (l < r) {
      const uint32_t m = (l + r) / 2;
      if (s_start[m + 1] > lo)
        r = m;
      else
        l = m + 1;
    }
    uint32_t cnt = 0, klast = 0;
    for (uint32_t k = l; k < K && s_start[k] < hi; ++k)
      if (s_start[k] < s_start[k + 1]) {
        ++cnt;
        klast = k;
      }
    const bool full = s_bt[b] != 0;
    pieces[b] = full ? cnt : 0u;
    s_r[b] = min(K - 1u, klast + delay);
    const uint32_t ub = (uint32_t)min((uint64_t)1u << kLow, (uint64_t)U - ((uint64_t)b << kLow));
    s_nch[b] = full ? (ub + kChunkBins - 1) / kChunkBins : 0u;
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t o = 0;
    uint64_t kb = 0;
    for (uint32_t b = 0; b < B; ++b) {
      s_off[b] = o;
      o += s_nch[b];
      bbase[b] = kb;
      kb += s_bt[b];
    }
    ctl->nsched = K + o;
  }
  __syncthreads();
  for (uint32_t t = tid; t < K; t += blockDim.x) {
    uint32_t idx = t;
    for (uint32_t b = 0; b < B; ++b)
      if (s_r[b] < t) idx += s_nch[b];
    sched[idx] = t;
  }
  for (uint32_t b = 0; b < B; ++b) {
    const uint32_t at = s_r[b] + 1u + s_off[b];
    for (uint32_t j = tid; j < s_nch[b]; j += blockDim.x) sched[at + j] = kProjItem | (b * kChunksPerBucket + j);
  }
}

// Projection item: chunk c (bins [1024 c, 1024 c + 1024)), one bin per thread.
__device__ __forceinline__ void project_chunk(uint32_t c, const uint32_t* __restrict__ H, uint32_t U,
                                              const uint32_t* __restrict__ pieces, const uint32_t* bdone,
                                              const uint64_t* __restrict__ bbase, uint64_t* desc, uint32_t* out,
                                              uint64_t n_cap, int out_aligned, FusedCtl* ctl, LongRun* longs,
                                              uint32_t* pmap, uint32_t* err, uint32_t* red, uint64_t* s_pre) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t b = c / kChunksPerBucket, j = c % kChunksPerBucket;
  if (tid == 0) {  // every piece of the bucket is in H
    uint32_t spins = 0;
    const uint32_t need = pieces[b];
    while (ld_acquire_u32(bdone + b) < need) {
      if (++spins > kSpinLimit) {
        raise_error(err, ERRBIT_TIMEOUT);
        break;
      }
      __nanosleep(128);
    }
  }
  __syncthreads();
  const uint64_t bin = (uint64_t)c * kChunkBins + tid;
  const uint32_t h = (tid < kChunkBins && bin < U) ? __ldcg(H + bin) : 0u;
  // block exclusive scan of the bins (a warp scan, then the warp totals)
  uint32_t x = h;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31) red[warp] = x;
  __syncthreads();
  uint32_t wb = 0, total = 0;
  for (uint32_t w = 0; w < kP2Threads / 32; ++w) {
    const uint32_t v = red[w];
    if (w < warp) wb += v;
    total += v;
  }
  const uint32_t excl = wb + x - h;
  if (tid == 0) {  // the chunk's start within its bucket: decoupled look-back over the bucket's chunks
    uint64_t pre = 0;
    if (j == 0) {
      st_release_u64(desc + c, kFlagInc | total);
    } else {
      st_release_u64(desc + c, kFlagAgg | total);
      uint32_t k = c - 1, spins = 0;
      for (;;) {
        const uint64_t d = ld_acquire_u64(desc + k);
        const uint64_t flag = d & ~kValMask;
        if (flag == 0) {
          if (++spins > kSpinLimit) {
            raise_error(err, ERRBIT_TIMEOUT);
            break;
          }
          __nanosleep(64);
          continue;
        }
        pre += d & kValMask;
        if (flag == kFlagInc || k % kChunksPerBucket == 0) break;
        --k;
      }
      st_release_u64(desc + c, kFlagInc | ((pre + total) & kValMask));
    }
    *s_pre = bbase[b] + pre;
  }
  __syncthreads();
  const uint64_t st = *s_pre + excl, en = min(st + h, n_cap);
  // a lane writes its run when short; longer runs are painted by the whole warp; the longest are listed
  // for hier_long_kernel
  if (h != 0 && h <= 4u)
    for (uint64_t p = st; p < en; ++p) out[p] = (uint32_t)bin;
  const uint32_t list_over = total > kChunkBudget ? kListRun : kWarpRun;  // the same in every thread
  if (h > list_over && st < en) {
    const uint32_t len = (uint32_t)(en - st), pieces_k = (len + kLongPiece - 1) / kLongPiece;
    const uint32_t i = atomicAdd(&ctl->nlong, 1u), p0 = atomicAdd(&ctl->npieces, pieces_k);
    longs[i] = LongRun{(uint32_t)st, len, (uint32_t)bin, p0};
    for (uint32_t q = 0; q < pieces_k; ++q) pmap[p0 + q] = i;
  }
  uint32_t lanes = __ballot_sync(0xffffffffu, h > 4u && h <= list_over && st < en);
  while (lanes) {
    const uint32_t src = (uint32_t)(__ffs(lanes) - 1);
    lanes &= lanes - 1;
    const uint64_t s0 = __shfl_sync(0xffffffffu, st, src), e0 = __shfl_sync(0xffffffffu, en, src);
    paint_run<uint32_t>(out, (uint32_t)s0, (uint32_t)e0, (uint32_t)(c * kChunkBins + src + warp * 32u), out_aligned,
                        lane, 32u);
  }
}

__global__ void __launch_bounds__(kP2Threads, 1) hier_sort_kernel(
    const uint16_t* __restrict__ low, const uint32_t* __restrict__ seg, const uint64_t* __restrict__ start,
    const uint32_t* __restrict__ btot, uint32_t B, uint32_t U, uint64_t num_tiles, uint32_t S_t,
    uint32_t* __restrict__ H, const uint32_t* __restrict__ sched, const uint32_t* __restrict__ pieces,
    uint32_t* bdone, const uint64_t* __restrict__ bbase, uint64_t* desc, uint32_t* __restrict__ out, uint64_t n_cap,
    int out_aligned, FusedCtl* ctl, LongRun* longs, uint32_t* pmap, uint32_t* err) {
  extern __shared__ __align__(128) uint32_t hist[];  // 2^15 bins
  __shared__ P2Smem sm;
  __shared__ uint32_t s_item;
  __shared__ uint64_t s_pre;
  const uint32_t tid = threadIdx.x;
  constexpr uint32_t bins = 1u << kLow;
  const uint32_t nsched = ctl->nsched;
  for (;;) {
    __syncthreads();  // the previous item is done with the shared words
    if (tid == 0) {
      const uint32_t t = atomicAdd(&ctl->ticket, 1u);
      s_item = t < nsched ? sched[t] : kNoItem;
    }
    __syncthreads();
    const uint32_t w = s_item;
    if (w == kNoItem) break;
    if (w & kProjItem) {
      project_chunk(w & ~kProjItem, H, U, pieces, bdone, bbase, desc, out, n_cap, out_aligned, ctl, longs, pmap,
                    err, sm.wred, &s_pre);
      continue;
    }
    uint64_t s = start[w];
    const uint64_t se = min(start[w + 1], (uint64_t)B * num_tiles);
    while (s < se) {
      const uint32_t b = (uint32_t)(s / num_tiles);
      const uint64_t ta = s - (uint64_t)b * num_tiles;
      const uint64_t tb = min(num_tiles, ta + (se - s));
      s += tb - ta;
      if (btot[b] == 0) continue;  // an empty bucket (the same value in every thread)
      __syncthreads();
      count_piece(low, seg, b, ta, tb, num_tiles, S_t, hist, sm);
      const uint64_t blo = (uint64_t)b << kLow;
      // (a bucket counted by many ranges is reduce-added into H too: scratch slots summed by the projection
      // items measured slower -- every chunk item then reads one slot per range)
      flush_piece(hist, (uint32_t)min((uint64_t)bins, (uint64_t)U - blo), H + blo, sm.wred);
      // the piece is in H (bulk adds complete and ordered before the release) before it is counted
      if (tid < 4) {
        bulk_wait_all();
        fence_proxy_async_global();
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(bdone + b, 1u);
    }
  }
}

// Paints the listed runs, a piece per warp, with every SM (pieces of one run in any order).
__global__ void __launch_bounds__(256) hier_long_kernel(const LongRun* __restrict__ longs,
                                                        const uint32_t* __restrict__ pmap, const FusedCtl* ctl,
                                                        uint32_t* __restrict__ out, int out_aligned) {
  const uint32_t npieces = ctl->npieces, lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * (blockDim.x / 32u);
  for (uint32_t p = blockIdx.x * (blockDim.x / 32u) + (threadIdx.x >> 5); p < npieces; p += warps) {
    const LongRun r = longs[pmap[p]];
    const uint32_t s = r.start + (p - r.piece0) * kLongPiece;
    const uint32_t e = min(s + kLongPiece, r.start + r.len);
    paint_run<uint32_t>(out, s, e, r.key, out_aligned, lane, 32u);
  }
}

}  // namespace

HierLayout hier_layout(uint64_t n, uint32_t U) {
  HierLayout T;
  T.B = (uint32_t)(((uint64_t)U + (1ull << kLow) - 1) >> kLow);
  T.BM = T.B <= 32 ? 32u : 64u;
  T.num_tiles = (n + kTile - 1) / kTile;
  T.S_t = kTile + 8u * T.BM;
  size_t o = 0;
  T.off_low = o;
  o = align_up(o + 2 * T.num_tiles * (size_t)T.S_t, 256);
  T.off_seg = o;
  o = align_up(o + 4 * T.num_tiles * (size_t)T.B, 256);
  T.off_btot = o;
  o = align_up(o + 4 * (size_t)kMaxBuckets, 256);
  T.off_start = o;
  o = align_up(o + 8 * ((size_t)kHierMaxCountCtas + 1), 256);
  T.G_max = hier_count_ctas(n, 1u << 30);
  T.off_used = o;
  o = align_up(o + 4 * ((size_t)T.G_max + T.B), 256);
  T.off_part = o;
  o = align_up(o + 4 * ((size_t)T.G_max + T.B) * (1u << kLow), 256);
  T.off_fclear = o;  // FusedCtl | bucket counters | one descriptor per 1024-bin chunk
  o = align_up(o + 256 + 4 * (size_t)kMaxBuckets + 8 * (size_t)kFusedMaxChunks, 256);
  T.fclear_bytes = o - T.off_fclear;
  T.off_fstart = o;
  o = align_up(o + 8 * ((size_t)kFusedMaxRanges + 1), 256);
  T.off_sched = o;
  o = align_up(o + 4 * ((size_t)kFusedMaxRanges + kFusedMaxChunks), 256);
  T.off_pieces = o;
  o = align_up(o + 4 * (size_t)kMaxBuckets, 256);
  T.off_bbase = o;
  o = align_up(o + 8 * (size_t)kMaxBuckets, 256);
  T.off_longs = o;  // at most n / kListRun listed runs, and n / kLongPiece + n / kListRun pieces
  o = align_up(o + sizeof(LongRun) * (n / kListRun + 1), 256);
  T.off_pmap = o;
  o = align_up(o + 4 * (n / kLongPiece + n / kListRun + 1), 256);
  T.total = o;
  return T;
}

uint32_t hier_count_ctas(uint64_t n, uint32_t sms) {
  // one 128 KB pass-2 CTA per SM, but at least 2^17 keys each
  const uint64_t by_n = std::max<uint64_t>(1, n >> 17);
  return (uint32_t)std::min<uint64_t>(std::min<uint64_t>(std::max<uint32_t>(sms, 1u), by_n), kHierMaxCountCtas);
}

bool hier_shape_fits(uint64_t n, uint32_t U, uint32_t key_bytes) {
  return key_bytes == 4 && n >= (1u << 20) && U > (1u << 16) && U <= (1u << 21);
}

bool hier_fits(uint64_t n, uint32_t U, uint32_t key_bytes, const void* keys) {
  return (reinterpret_cast<uintptr_t>(keys) & 15u) == 0 && hier_shape_fits(n, U, key_bytes);
}

namespace {
// Pass 1: bucket totals cleared, then the partition of every tile.
cudaError_t launch_partition(const uint32_t* keys, uint64_t n, uint32_t U, char* base, const HierLayout& T,
                             const DeviceInfo& dev, uint32_t* err, cudaStream_t stream) {
  uint16_t* low = reinterpret_cast<uint16_t*>(base + T.off_low);
  uint32_t* seg = reinterpret_cast<uint32_t*>(base + T.off_seg);
  uint32_t* btot = reinterpret_cast<uint32_t*>(base + T.off_btot);
  cudaError_t e = cudaMemsetAsync(btot, 0, 4 * (size_t)kMaxBuckets, stream);
  if (e != cudaSuccess) return e;
  const bool pow2 = (U & (U - 1)) == 0;
  const void* p1 = T.BM == 32 ? (pow2 ? reinterpret_cast<const void*>(&hier_partition_kernel<32, true>)
                                      : reinterpret_cast<const void*>(&hier_partition_kernel<32, false>))
                              : (pow2 ? reinterpret_cast<const void*>(&hier_partition_kernel<64, true>)
                                      : reinterpret_cast<const void*>(&hier_partition_kernel<64, false>));
  int per_sm = 0;
  e = kernel_config(p1, kP1Threads, 0, false, &per_sm);
  if (e != cudaSuccess) return e;
  const uint64_t grid1 = std::min<uint64_t>(T.num_tiles, (uint64_t)dev.sms * std::max(per_sm, 1));
  {
    uint32_t UU = U, B = T.B, S_t = T.S_t;
    uint64_t nn = n, nt = T.num_tiles;
    void* args[] = {const_cast<uint32_t**>(&keys), &nn, &UU, &B, &nt, &S_t, &low, &seg, &btot, &err};
    e = cudaLaunchKernel(p1, dim3((unsigned)grid1), dim3(kP1Threads), args, 0, stream);
  }
  return e;
}
}  // namespace

cudaError_t launch_hier(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H, void* ws, const HierLayout& T,
                        const DeviceInfo& dev, uint32_t* err, cudaStream_t stream, bool accumulate) {
  char* base = static_cast<char*>(ws);
  uint16_t* low = reinterpret_cast<uint16_t*>(base + T.off_low);
  uint32_t* seg = reinterpret_cast<uint32_t*>(base + T.off_seg);
  uint32_t* btot = reinterpret_cast<uint32_t*>(base + T.off_btot);
  uint64_t* start = reinterpret_cast<uint64_t*>(base + T.off_start);
  uint32_t* part_used = reinterpret_cast<uint32_t*>(base + T.off_used);
  uint32_t* part = reinterpret_cast<uint32_t*>(base + T.off_part);
  cudaError_t e = launch_partition(keys, n, U, base, T, dev, err, stream);
  if (e != cudaSuccess) return e;
  const uint32_t G = hier_count_ctas(n, (uint32_t)dev.sms);
  hier_split_kernel<<<T.B, 1024, 0, stream>>>(seg, btot, T.B, T.num_tiles, G, start);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (!accumulate && (e = cudaMemsetAsync(H, 0, (size_t)U * 4, stream)) != cudaSuccess) return e;
  const size_t p2_smem = (size_t)4 << kLow;
  e = kernel_config(reinterpret_cast<const void*>(&hier_count_kernel), kP2Threads, p2_smem, false, nullptr);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(part_used, 0, 4 * ((size_t)G + T.B), stream)) != cudaSuccess) return e;
  hier_count_kernel<<<G, kP2Threads, p2_smem, stream>>>(low, seg, start, btot, T.B, U, T.num_tiles, T.S_t, H, part,
                                                        part_used);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  hier_merge_kernel<<<dim3(T.B, (1u << kLow) / 1024u), 256, 0, stream>>>(btot, T.B, U, G, part, part_used, H);
  return cudaGetLastError();
}

cudaError_t launch_hier_sort(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H, uint32_t* out, void* ws,
                             const HierLayout& T, const DeviceInfo& dev, uint32_t* err, cudaStream_t stream,
                             cudaEvent_t* marks) {
  char* base = static_cast<char*>(ws);
  const uint16_t* low = reinterpret_cast<const uint16_t*>(base + T.off_low);
  const uint32_t* seg = reinterpret_cast<const uint32_t*>(base + T.off_seg);
  const uint32_t* btot = reinterpret_cast<const uint32_t*>(base + T.off_btot);
  FusedCtl* ctl = reinterpret_cast<FusedCtl*>(base + T.off_fclear);
  uint32_t* bdone = reinterpret_cast<uint32_t*>(base + T.off_fclear + 256);
  uint64_t* desc = reinterpret_cast<uint64_t*>(base + T.off_fclear + 256 + 4 * (size_t)kMaxBuckets);
  uint64_t* start = reinterpret_cast<uint64_t*>(base + T.off_fstart);
  uint32_t* sched = reinterpret_cast<uint32_t*>(base + T.off_sched);
  uint32_t* pieces = reinterpret_cast<uint32_t*>(base + T.off_pieces);
  uint64_t* bbase = reinterpret_cast<uint64_t*>(base + T.off_bbase);
  cudaError_t e = launch_partition(keys, n, U, base, T, dev, err, stream);
  if (e == cudaSuccess && marks) e = cudaEventRecord(marks[0], stream);
  if (e != cudaSuccess) return e;
  // count ranges: one per SM (measured faster than four: fewer pieces to flush), at least 2^17 keys each
  const uint32_t K = hier_count_ctas(n, (uint32_t)dev.sms);
  hier_split_kernel<<<T.B, 1024, 0, stream>>>(seg, btot, T.B, T.num_tiles, K, start);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(H, 0, (size_t)U * 4, stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(base + T.off_fclear, 0, T.fclear_bytes, stream)) != cudaSuccess) return e;
  const size_t smem = (size_t)4 << kLow;
  int per_sm = 0;
  e = kernel_config(reinterpret_cast<const void*>(&hier_sort_kernel), kP2Threads, smem, false, &per_sm);
  if (e != cudaSuccess) return e;
  const uint32_t grid = (uint32_t)std::max(1, dev.sms * std::max(per_sm, 1));
  hier_sched_kernel<<<1, 1024, 0, stream>>>(start, K, btot, T.B, U, T.num_tiles, grid, sched, pieces, bbase, ctl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (marks && (e = cudaEventRecord(marks[1], stream)) != cudaSuccess) return e;
  const int aligned = (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  LongRun* longs = reinterpret_cast<LongRun*>(base + T.off_longs);
  uint32_t* pmap = reinterpret_cast<uint32_t*>(base + T.off_pmap);
  hier_sort_kernel<<<grid, kP2Threads, smem, stream>>>(low, seg, start, btot, T.B, U, T.num_tiles, T.S_t, H, sched,
                                                      pieces, bdone, bbase, desc, out, n, aligned, ctl, longs, pmap,
                                                      err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (marks && (e = cudaEventRecord(marks[2], stream)) != cudaSuccess) return e;
  hier_long_kernel<<<dev.sms * 4, 256, 0, stream>>>(longs, pmap, ctl, out, aligned);
  return cudaGetLastError();
}

}  // namespace dialsort
