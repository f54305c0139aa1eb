// Device routines of step 2 (the ordered projection, Eq. (2)), shared by the
// single-instance kernels (reconstruct.cu) and the batched/served engine
// (engine.cu).  Each routine is executed by one 256-thread CTA.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace dialsort {

constexpr uint32_t kReconThreads = 256;  // threads of a CTA running these routines
constexpr uint64_t kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62, kValMask = (1ull << 62) - 1;

__device__ __forceinline__ void load_bins4(const uint32_t* H, uint64_t b0, uint32_t U, uint32_t (&h)[4]) {
  if (b0 + 3 < U) {
    const uint4 q = *reinterpret_cast<const uint4*>(H + b0);
    h[0] = q.x;
    h[1] = q.y;
    h[2] = q.z;
    h[3] = q.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = (b0 + j < U) ? H[b0 + j] : 0u;
  }
}

// Block-wide exclusive sum of one value per thread; returns the exclusive
// prefix and writes the block total to *total.  `red` needs blockDim/32 + 1 slots.
template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* red, T* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? red[lane] : T(0);
    T s = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= (uint32_t)d) s += y;
    }
    if (lane < nw) red[lane] = s - w;  // exclusive prefix of warp totals
    if (lane == nw - 1) red[nw] = s;
  }
  __syncthreads();
  const T excl = red[warp] + (x - v);
  *total = red[nw];
  __syncthreads();  // red may be reused by the caller
  return excl;
}

struct OffsetsSmem {
  uint64_t wsum[kReconThreads / 32];  // each warp's chunk total
  uint64_t gexcl;                     // the group's exclusive prefix
};

// Sum of one 1024-bin chunk by one warp (lane l: bins 128 r + 4 l .. + 3).
__device__ __forceinline__ uint64_t warp_chunk_sum(const uint32_t* __restrict__ H, uint32_t U, uint64_t c) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t sum = 0;
#pragma unroll
  for (uint32_t r = 0; r < kChunkBins / 128; ++r) {
    uint32_t h[4];
    load_bins4(H, c * kChunkBins + r * 128 + lane * 4ull, U, h);
    sum += (uint64_t)h[0] + h[1] + h[2] + h[3];
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
  return sum;
}

// Group g of the offset scan: chunks [8 g, 8 g + 8), one per warp.  Computes
// the group total, its exclusive prefix by decoupled look-back over
// desc[0..g), O[c] for its chunks (and O[num_chunks] in the last group), and
// the first chunk of every output tile whose first key falls in a chunk's run
// range.  The caller guarantees that every group below g is already held by a
// running CTA (groups are handed out in order), so the look-back ends.
__device__ __forceinline__ void offsets_group(const uint32_t* __restrict__ H, uint32_t U, uint64_t n_cap,
                                              uint64_t num_chunks, uint64_t g, uint64_t* desc, uint64_t* O,
                                              uint32_t* first_chunk, uint32_t* err, OffsetsSmem& sm) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  constexpr uint32_t kG = kReconThreads / 32;  // chunks per group
  const uint64_t c = g * kG + warp;
  const uint64_t mine = c < num_chunks ? warp_chunk_sum(H, U, c) : 0;
  if (lane == 0) sm.wsum[warp] = mine;
  __syncthreads();
  if (tid == 0) {
    uint64_t agg = 0;
    for (uint32_t w = 0; w < kG; ++w) agg += sm.wsum[w];
    uint64_t excl = 0;
    if (g == 0) {
      st_release_u64(desc, kFlagInc | (agg & kValMask));
    } else {
      st_release_u64(desc + g, kFlagAgg | (agg & kValMask));
      // look back over predecessors until one has published its inclusive prefix
      int64_t j = (int64_t)g - 1;
      uint32_t spins = 0;
      while (j >= 0) {
        const uint64_t d = ld_acquire_u64(desc + j);
        const uint64_t flag = d & ~kValMask;
        if (flag == 0) {
          if (++spins > kSpinLimit) {
            raise_error(err, ERRBIT_TIMEOUT);
            break;
          }
          __nanosleep(64);
          continue;
        }
        excl += d & kValMask;
        if (flag == kFlagInc) break;
        --j;
      }
      st_release_u64(desc + g, kFlagInc | ((excl + agg) & kValMask));
    }
    sm.gexcl = excl;
  }
  __syncthreads();
  if (c < num_chunks) {
    uint64_t lo = sm.gexcl;
    for (uint32_t w = 0; w < warp; ++w) lo += sm.wsum[w];
    if (lane == 0) {
      O[c] = lo;
      if (c == num_chunks - 1) {
        O[num_chunks] = lo + mine;
        if (lo + mine > n_cap) raise_error(err, ERRBIT_OVERFLOW);
      }
    }
    // tiles whose first key falls inside this chunk's run range [lo, lo + mine)
    const uint64_t hi = min(lo + mine, n_cap);
    if (mine != 0 && lo < hi) {
      const uint64_t t0 = (lo + kTileKeys - 1) / kTileKeys;
      const uint64_t t1 = (hi - 1) / kTileKeys;
      for (uint64_t t = t0 + lane; t <= t1; t += 32) first_chunk[t] = (uint32_t)c;
    }
  }
  __syncthreads();  // sm is reused by the caller's next item
}

__host__ __device__ inline uint64_t offset_groups(uint64_t num_chunks) {
  return (num_chunks + kReconThreads / 32 - 1) / (kReconThreads / 32);
}

// Bin-parallel projection for a sparse histogram (n well below U, where an
// output tile spans many chunks and one CTA would walk them all): item g
// takes chunks [8 g, 8 g + 8), one per warp, and every bin k writes its own
// run [start_k, start_k + H[k]) of Eq. (2) -- start_k from the chunk's offset
// O[c] and a warp scan of the chunk's bins.  A lane writes runs of up to four
// keys itself; longer runs are painted by the whole warp.  Positions at or
// past n_cap are not written (sum(H) > n_cap is reported by the offsets).
template <typename OutT>
__device__ __forceinline__ void expand_bins(const uint32_t* __restrict__ H, uint32_t U, uint64_t n_cap,
                                            uint64_t num_chunks, const uint64_t* __restrict__ O,
                                            OutT* __restrict__ out, uint64_t g,
                                            const OutT* __restrict__ inv = nullptr) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint64_t c = g * (kReconThreads / 32) + warp;
  if (c >= num_chunks) return;
  uint64_t run = O[c];
  if (O[c + 1] == run || run >= n_cap) return;  // an empty chunk, or one past the output (warp-uniform)
#pragma unroll 1
  for (uint32_t r = 0; r < kChunkBins / 128; ++r) {
    uint32_t h[4];
    const uint64_t b0 = c * kChunkBins + r * 128 + lane * 4ull;
    load_bins4(H, b0, U, h);
    const uint32_t t4 = h[0] + h[1] + h[2] + h[3];
    uint32_t x = t4;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= (uint32_t)d) x += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
    if (total == 0) continue;  // warp-uniform
    const uint64_t s0 = run + (x - t4);
    uint64_t st = s0;
    uint32_t longmask = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (h[j] != 0 && h[j] <= 4) {
        const OutT key = inv != nullptr ? inv[b0 + j] : (OutT)(b0 + j);
        for (uint32_t q = 0; q < h[j]; ++q)
          if (st + q < n_cap) out[st + q] = key;
      } else if (h[j] > 4) {
        longmask |= 1u << j;
      }
      st += h[j];
    }
    uint32_t lanes = __ballot_sync(0xffffffffu, longmask != 0);
    while (lanes) {  // long runs: the warp paints them one by one
      const uint32_t src = (uint32_t)(__ffs(lanes) - 1);
      lanes &= lanes - 1;
      const uint32_t lm = __shfl_sync(0xffffffffu, longmask, src);
      uint64_t ss = __shfl_sync(0xffffffffu, s0, src);
      const uint64_t sb = c * kChunkBins + r * 128 + src * 4ull;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t hj = __shfl_sync(0xffffffffu, h[j], src);
        if ((lm >> j) & 1u) {
          const OutT key = inv != nullptr ? inv[sb + j] : (OutT)(sb + j);
          for (uint32_t q = lane; q < hj; q += 32)
            if (ss + q < n_cap) out[ss + q] = key;
        }
        ss += hj;
      }
    }
    run += total;
    if (run >= n_cap) return;  // warp-uniform
  }
}

// Tiles crossed by at most this many short runs are painted run by run; others fill forward.
// Runs of kLongRun slots or more (at most four per tile) are painted by the whole CTA.
constexpr uint32_t kPaintRuns = 256;
constexpr uint32_t kLongRun = kTileKeys / 4;

struct ExpandSmem {
  uint32_t M[kTileKeys];  // key + 1 where a run starts, 0 elsewhere
  uint32_t red32[kReconThreads / 32 + 1];
  uint32_t nruns;         // short runs that cross the tile
  uint32_t nlong;         // long runs that cross the tile
  uint2 runs[kPaintRuns]; // (first slot | end slot << 16, key) of each short run, in no order
  uint2 longs[4];         // the same for the long runs
};

// Record a run crossing the tile: slots [s, e) hold key.
__device__ __forceinline__ void note_run(ExpandSmem& sm, uint32_t s, uint32_t e, uint32_t key) {
  if (e - s >= kLongRun) {
    const uint32_t i = atomicAdd(&sm.nlong, 1u);
    if (i < 4) sm.longs[i] = make_uint2(s | (e << 16), key);
  } else if (*reinterpret_cast<volatile uint32_t*>(&sm.nruns) <= kPaintRuns) {  // past the cap: stop counting
    const uint32_t i = atomicAdd(&sm.nruns, 1u);
    if (i < kPaintRuns) sm.runs[i] = make_uint2(s | (e << 16), key);
  }
}

// Slots [s, e) of the tile starting at dst get `key`: 16-byte stores over the aligned middle, plain
// stores at the ends; called by `lanes` threads together (a warp, or the CTA), `lane` in [0, lanes).
template <typename OutT>
__device__ __forceinline__ void paint_run(OutT* __restrict__ dst, uint32_t s, uint32_t e, uint32_t key,
                                          int out_aligned, uint32_t lane, uint32_t lanes) {
  constexpr uint32_t kPer = 16 / sizeof(OutT);  // keys per 16-byte store
  const uint32_t a = out_aligned ? (s + kPer - 1) / kPer * kPer : e;  // first aligned slot
  const uint32_t b = out_aligned ? e / kPer * kPer : e;                // end of the aligned middle
  if (a >= b) {  // no aligned middle: plain stores
    for (uint32_t i = s + lane; i < e; i += lanes) dst[i] = (OutT)key;
    return;
  }
  if (s + lane < a) dst[s + lane] = (OutT)key;  // head: fewer than kPer slots
  uint4 v;
  if (sizeof(OutT) == 4) {
    v = make_uint4(key, key, key, key);
  } else if (sizeof(OutT) == 2) {
    const uint32_t k2 = (key & 0xffffu) | (key << 16);
    v = make_uint4(k2, k2, k2, k2);
  } else {
    const uint32_t k4 = (key & 0xffu) * 0x01010101u;
    v = make_uint4(k4, k4, k4, k4);
  }
  uint4* d4 = reinterpret_cast<uint4*>(dst + a);
  for (uint32_t q = lane; q < (b - a) / kPer; q += lanes) d4[q] = v;
  if (b + lane < e) dst[b + lane] = (OutT)key;  // tail: fewer than kPer slots
}

// Output tile `tile` (keys [tile * 8192, ...)) of the projection.  Marks the
// slot where each run starts (slot 0 gets the run covering the tile's first
// key), fills forward ("latest mark wins"), and stores with 128-bit stores.
// With inv, index k is written as inv[k] (the inverse map of Prop. "General
// Self-Indexing Principle"); without it, as k.
template <typename OutT>
__device__ __forceinline__ void expand_tile(const uint32_t* __restrict__ H, uint32_t U, uint64_t n_cap,
                                            uint64_t num_chunks, const uint64_t* __restrict__ O,
                                            const uint32_t* __restrict__ first_chunk, OutT* __restrict__ out,
                                            int out_aligned, uint64_t tile, ExpandSmem& sm,
                                            const OutT* __restrict__ inv = nullptr) {
  uint32_t* M = sm.M;
  uint32_t* red32 = sm.red32;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t total = min(O[num_chunks], n_cap);
  const uint64_t tile_lo = tile * kTileKeys;
  if (tile_lo >= total) return;
  const uint64_t tile_hi = min(tile_lo + kTileKeys, total);
  const uint32_t len = (uint32_t)(tile_hi - tile_lo);

  // Mark run starts of every chunk overlapping [tile_lo, tile_hi).  A dense
  // tile overlaps one or two chunks: the whole CTA scans each (4 bins per
  // thread, one load each).  A sparse tile can overlap hundreds: the chunks
  // are shared out among the warps (warp w: c0 + w, c0 + w + 8, ...), each
  // warp scans its chunk with shuffles alone and skips an empty chunk without
  // reading its bins.  Every run crossing the tile is also noted (up to
  // kPaintRuns) so that a tile of few runs can be painted; a dense tile first
  // only notes runs and writes the marks in a second scan if it has too many.
  const uint64_t c0 = first_chunk[tile];
  const uint64_t num_tiles = (n_cap + kTileKeys - 1) / kTileKeys;
  // the next tile's first chunk bounds the chunks this tile can overlap
  const uint64_t c_last = (tile + 1 < num_tiles && tile_hi < total) ? first_chunk[tile + 1] : num_chunks - 1;
  const bool dense = c_last - c0 <= 1;
  uint4* M4 = reinterpret_cast<uint4*>(M);
  if (!dense)
    for (uint32_t i = tid; i < kTileKeys / 4; i += kReconThreads) M4[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    sm.nruns = 0;
    sm.nlong = 0;
  }
  __syncthreads();
  // dense tiles: notes (marks == false) or marks (marks == true) from one CTA-wide scan per chunk
  auto dense_scan = [&](bool marks) {
    for (uint64_t c = c0; c <= c_last && c < num_chunks; ++c) {
      const uint64_t oc = O[c];
      if (oc >= tile_hi) break;
      if (O[c + 1] == oc) continue;  // empty chunk
      uint32_t h[4];
      const uint64_t b0 = c * kChunkBins + tid * 4ull;
      load_bins4(H, b0, U, h);
      uint32_t chunk_total;
      uint32_t sc = block_exclusive_sum<uint32_t>(h[0] + h[1] + h[2] + h[3], red32, &chunk_total);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (h[j] != 0) {
          const uint64_t start = oc + sc, end = start + h[j];
          const uint32_t mark = (uint32_t)(b0 + j) + 1u;
          const uint32_t e = (uint32_t)((end < tile_hi ? end : tile_hi) - tile_lo);
          if (start >= tile_lo && start < tile_hi) {
            if (marks)
              M[start - tile_lo] = mark;
            else
              note_run(sm, (uint32_t)(start - tile_lo), e, mark - 1u);
          } else if (start < tile_lo && end > tile_lo) {
            if (marks)
              M[0] = mark;
            else
              note_run(sm, 0u, e, mark - 1u);
          }
        }
        sc += h[j];
      }
    }
  };
  if (dense) {
    dense_scan(false);
  } else {
    for (uint64_t c = c0 + warp; c < num_chunks; c += kReconThreads / 32) {
      const uint64_t oc = O[c];
      if (oc >= tile_hi) break;           // every later chunk starts later still
      if (O[c + 1] == oc) continue;       // empty chunk
      uint64_t run = oc;                  // start of the run of the next bin
#pragma unroll 1
      for (uint32_t r = 0; r < kChunkBins / 128; ++r) {
        if (run >= tile_hi) break;        // the rest of this chunk lies past the tile (warp-uniform)
        uint32_t h[4];
        const uint64_t b0 = c * kChunkBins + r * 128 + lane * 4ull;
        load_bins4(H, b0, U, h);
        const uint32_t t4 = h[0] + h[1] + h[2] + h[3];
        uint32_t x = t4;  // inclusive scan of the lanes' sums
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
          if (lane >= (uint32_t)d) x += y;
        }
        uint64_t start = run + (x - t4);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (h[j] != 0) {
            const uint64_t end = start + h[j];
            const uint32_t mark = (uint32_t)(b0 + j) + 1u;
            const uint32_t e = (uint32_t)((end < tile_hi ? end : tile_hi) - tile_lo);
            if (start >= tile_lo && start < tile_hi) {
              M[start - tile_lo] = mark;
              note_run(sm, (uint32_t)(start - tile_lo), e, mark - 1u);
            } else if (start < tile_lo && end > tile_lo) {
              M[0] = mark;
              note_run(sm, 0u, e, mark - 1u);
            }
          }
          start += h[j];
        }
        run += __shfl_sync(0xffffffffu, x, 31);
      }
    }
  }
  __syncthreads();

  OutT* dst = out + tile_lo;
  const uint32_t nruns = sm.nruns, nlong = sm.nlong;
  if (nruns <= kPaintRuns) {  // few runs: paint each with its key
    for (uint32_t r = warp; r < nruns; r += kReconThreads / 32) {
      const uint2 run = sm.runs[r];
      const uint32_t key = inv != nullptr ? (uint32_t)inv[run.y] : run.y;
      paint_run<OutT>(dst, run.x & 0xffffu, run.x >> 16, key, out_aligned, lane, 32u);
    }
    for (uint32_t r = 0; r < nlong && r < 4; ++r) {
      const uint2 run = sm.longs[r];
      const uint32_t key = inv != nullptr ? (uint32_t)inv[run.y] : run.y;
      paint_run<OutT>(dst, run.x & 0xffffu, run.x >> 16, key, out_aligned, tid, kReconThreads);
    }
    __syncthreads();  // sm is reused by the caller's next item
    return;
  }
  if (dense) {  // too many runs to paint: the marks, from a second scan
    for (uint32_t i = tid; i < kTileKeys / 4; i += kReconThreads) M4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    dense_scan(true);
    __syncthreads();
  }

  // Fill forward: every slot takes the latest mark at or before it.  Warp w
  // owns slots [1024 w, 1024 w + 1024); in round r lane l holds the quad at
  // 1024 w + 128 r + 4 l, so shared-memory reads are conflict-free and each
  // round's global store is 512 contiguous bytes.
  constexpr uint32_t kWarpSlots = kTileKeys / (kReconThreads / 32);  // 1024
  constexpr uint32_t kRounds = kWarpSlots / 128;                      // 8
  const uint32_t wq = warp * (kWarpSlots / 4);                        // first quad of this warp
  // pass 1: this warp's rightmost mark (scan rounds from the right)
  uint32_t agg = 0;
  for (int r = (int)kRounds - 1; r >= 0; --r) {
    const uint4 q = M4[wq + r * 32 + lane];
    const uint32_t last = q.w ? q.w : q.z ? q.z : q.y ? q.y : q.x;
    const uint32_t bal = __ballot_sync(0xffffffffu, last != 0);
    if (bal) {
      agg = __shfl_sync(0xffffffffu, last, 31 - __clz(bal));
      break;
    }
  }
  if (lane == 0) red32[warp] = agg;
  __syncthreads();
  uint32_t carry = 0;  // rightmost mark of the warps before this one
  for (int w2 = (int)warp - 1; w2 >= 0 && carry == 0; --w2) carry = red32[w2];

  for (uint32_t r = 0; r < kRounds; ++r) {
    const uint32_t slot = warp * kWarpSlots + r * 128 + lane * 4;
    uint4 q = M4[wq + r * 32 + lane];
    const uint32_t last = q.w ? q.w : q.z ? q.z : q.y ? q.y : q.x;
    uint32_t x = last;  // inclusive "rightmost non-zero" over lanes
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= (uint32_t)d && x == 0) x = y;
    }
    uint32_t c = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0 || c == 0) c = carry;
    const uint32_t round_last = __shfl_sync(0xffffffffu, x, 31);
    if (round_last) carry = round_last;
    const uint32_t m0 = q.x ? q.x : c;
    const uint32_t m1 = q.y ? q.y : m0;
    const uint32_t m2 = q.z ? q.z : m1;
    const uint32_t m3 = q.w ? q.w : m2;
    q = make_uint4(m0 - 1u, m1 - 1u, m2 - 1u, m3 - 1u);  // marks hold key + 1
    if (slot >= len) continue;
    if (inv != nullptr) q = make_uint4(inv[q.x], inv[q.y], inv[q.z], inv[q.w]);
    if (slot + 4 <= len && out_aligned) {
      if (sizeof(OutT) == 4) {
        *reinterpret_cast<uint4*>(dst + slot) = q;
      } else if (sizeof(OutT) == 2) {
        *reinterpret_cast<uint2*>(dst + slot) = make_uint2(q.x | (q.y << 16), q.z | (q.w << 16));
      } else {
        *reinterpret_cast<uint32_t*>(dst + slot) =
            (q.x & 0xffu) | ((q.y & 0xffu) << 8) | ((q.z & 0xffu) << 16) | (q.w << 24);
      }
    } else {
      dst[slot] = (OutT)q.x;
      if (slot + 1 < len) dst[slot + 1] = (OutT)q.y;
      if (slot + 2 < len) dst[slot + 2] = (OutT)q.z;
      if (slot + 3 < len) dst[slot + 3] = (OutT)q.w;
    }
  }
  __syncthreads();  // sm is reused by the caller's next item
}

}  // namespace dialsort
