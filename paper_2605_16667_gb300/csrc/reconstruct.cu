// Step 2 of DialSort: the ordered projection, Eq. (2) -- for k = 0..U-1 emit
// k exactly H[k] times.
//
// The sequential projection keeps one cursor; to write runs in parallel each
// run needs its start, sum_{j<k} H[j] (the cursor on reaching k).  The paper
// says DialSort needs no prefix sum; that holds for the single cursor only, so
// this file computes the starts at two granularities and keeps the fine one
// on chip:
//
//   offsets kernel  one CTA per 1024-bin chunk: the chunk's total, an
//                   exclusive scan across chunks by decoupled look-back, and,
//                   for every 8192-key output tile that starts inside the
//                   chunk's run range, the tile's first chunk.  Reads H once
//                   (4U bytes); writes 16 bytes per chunk and 4 per tile.
//   expand kernel   one CTA per output tile.  It walks the chunks that overlap
//                   the tile, scans each chunk's bins in shared memory to get
//                   run starts, and marks in a tile-sized buffer the slot where
//                   each run starts (slot 0 gets the run covering the tile's
//                   first key).  A fill-forward scan ("latest mark wins")
//                   turns marks into keys, which go out with 128-bit stores.
//
// No key is compared with another: searches and scans act on counts and
// output positions only.  Load balance is by output position, so one bin with
// H[k] = n (all keys equal) spreads over all tiles.
#include "common.cuh"
#include "internal.h"

namespace dialsort {

namespace {

constexpr uint32_t kScanThreads = 256;  // offsets kernel: 4 bins per thread
constexpr uint32_t kExpThreads = 256;   // expand kernel: 32 output keys per thread
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

__global__ void __launch_bounds__(kScanThreads) offsets_kernel(const uint32_t* __restrict__ H, uint32_t U,
                                                               uint64_t n_cap, uint64_t num_chunks,
                                                               uint32_t* ticket, uint64_t* desc, uint64_t* O,
                                                               uint32_t* first_chunk, uint32_t* err) {
  __shared__ uint64_t red[kScanThreads / 32 + 1];
  __shared__ uint64_t s_c, s_excl;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) s_c = atomicAdd(ticket, 1u);  // dynamic order: every lower chunk is already running or done
  __syncthreads();
  const uint64_t c = s_c;

  uint32_t h[4];
  load_bins4(H, c * kChunkBins + tid * 4ull, U, h);
  const uint64_t mine = (uint64_t)h[0] + h[1] + h[2] + h[3];
  uint64_t agg;
  block_exclusive_sum<uint64_t>(mine, red, &agg);

  if (tid == 0) {
    uint64_t excl = 0;
    if (c == 0) {
      st_release_u64(desc, kFlagInc | (agg & kValMask));
    } else {
      st_release_u64(desc + c, kFlagAgg | (agg & kValMask));
      // look back over predecessors until one has published its inclusive prefix
      int64_t j = (int64_t)c - 1;
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
      st_release_u64(desc + c, kFlagInc | ((excl + agg) & kValMask));
    }
    s_excl = excl;
    O[c] = excl;
    if (c == num_chunks - 1) {
      O[num_chunks] = excl + agg;
      if (excl + agg > n_cap) raise_error(err, ERRBIT_OVERFLOW);
    }
  }
  __syncthreads();
  // tiles whose first key falls inside this chunk's run range [excl, excl + agg)
  const uint64_t lo = s_excl;
  const uint64_t hi = min(lo + agg, n_cap);
  if (agg != 0 && lo < hi) {
    const uint64_t t0 = (lo + kTileKeys - 1) / kTileKeys;
    const uint64_t t1 = (hi - 1) / kTileKeys;
    for (uint64_t t = t0 + tid; t <= t1; t += kScanThreads) first_chunk[t] = (uint32_t)c;
  }
}

template <typename OutT>
__global__ void __launch_bounds__(kExpThreads) expand_kernel(const uint32_t* __restrict__ H, uint32_t U,
                                                             uint64_t n_cap, uint64_t num_chunks,
                                                             const uint64_t* __restrict__ O,
                                                             const uint32_t* __restrict__ first_chunk,
                                                             OutT* __restrict__ out, int out_aligned) {
  __shared__ __align__(16) uint32_t M[kTileKeys];  // key + 1 where a run starts, 0 elsewhere
  __shared__ uint32_t red32[kExpThreads / 32 + 1];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t total = min(O[num_chunks], n_cap);
  const uint64_t tile_lo = (uint64_t)blockIdx.x * kTileKeys;
  if (tile_lo >= total) return;
  const uint64_t tile_hi = min(tile_lo + kTileKeys, total);
  const uint32_t len = (uint32_t)(tile_hi - tile_lo);

  uint4* M4 = reinterpret_cast<uint4*>(M);
  for (uint32_t i = tid; i < kTileKeys / 4; i += kExpThreads) M4[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();

  // mark run starts of every chunk overlapping [tile_lo, tile_hi)
  for (uint64_t c = first_chunk[blockIdx.x]; c < num_chunks; ++c) {
    const uint64_t oc = O[c];
    if (oc >= tile_hi) break;
    if (O[c + 1] == oc) continue;  // empty chunk
    uint32_t h[4];
    const uint64_t b0 = c * kChunkBins + tid * 4ull;
    load_bins4(H, b0, U, h);
    uint32_t chunk_total;
    uint32_t s = block_exclusive_sum<uint32_t>(h[0] + h[1] + h[2] + h[3], red32, &chunk_total);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (h[j] != 0) {
        const uint64_t start = oc + s, end = start + h[j];
        const uint32_t mark = (uint32_t)(b0 + j) + 1u;
        if (start >= tile_lo && start < tile_hi)
          M[start - tile_lo] = mark;
        else if (start < tile_lo && end > tile_lo)
          M[0] = mark;
      }
      s += h[j];
    }
  }
  __syncthreads();

  // fill forward: every slot takes the latest mark at or before it
  constexpr uint32_t PER = kTileKeys / kExpThreads;  // 32 slots per thread, contiguous
  uint32_t v[PER];
#pragma unroll
  for (uint32_t q = 0; q < PER / 4; ++q) {
    const uint4 x = M4[tid * (PER / 4) + q];
    v[4 * q] = x.x;
    v[4 * q + 1] = x.y;
    v[4 * q + 2] = x.z;
    v[4 * q + 3] = x.w;
  }
  uint32_t last = 0;
#pragma unroll
  for (uint32_t j = 0; j < PER; ++j) last = v[j] ? v[j] : last;
  // inclusive "latest non-zero" scan over threads
  uint32_t x = last;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (uint32_t)d && x == 0) x = y;
  }
  if (lane == 31) red32[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kExpThreads / 32 ? red32[lane] : 0u;
    uint32_t s = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= (uint32_t)d && s == 0) s = y;
    }
    const uint32_t prev = __shfl_up_sync(0xffffffffu, s, 1);
    if (lane < kExpThreads / 32) red32[lane] = lane ? prev : 0u;  // exclusive over warps
  }
  __syncthreads();
  uint32_t carry = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) carry = 0;
  if (carry == 0) carry = red32[warp];
#pragma unroll
  for (uint32_t j = 0; j < PER; ++j) {
    carry = v[j] ? v[j] : carry;
    v[j] = carry - 1u;
  }
#pragma unroll
  for (uint32_t q = 0; q < PER / 4; ++q)
    M4[tid * (PER / 4) + q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  __syncthreads();

  OutT* dst = out + tile_lo;
  if (sizeof(OutT) == 4) {
    uint32_t i = 0;
    if (out_aligned) {
      uint4* d4 = reinterpret_cast<uint4*>(dst);
      const uint32_t quads = len / 4;
      for (uint32_t qd = tid; qd < quads; qd += kExpThreads) d4[qd] = M4[qd];
      i = quads * 4;
    }
    for (uint32_t k = i + tid; k < len; k += kExpThreads) dst[k] = (OutT)M[k];
  } else {
    uint32_t i = 0;
    if (out_aligned) {
      uint4* d4 = reinterpret_cast<uint4*>(dst);
      const uint32_t octs = len / 8;
      for (uint32_t o = tid; o < octs; o += kExpThreads) {
        const uint4 a = M4[2 * o], b = M4[2 * o + 1];
        d4[o] = make_uint4(a.x | (a.y << 16), a.z | (a.w << 16), b.x | (b.y << 16), b.z | (b.w << 16));
      }
      i = octs * 8;
    }
    for (uint32_t k = i + tid; k < len; k += kExpThreads) dst[k] = (OutT)M[k];
  }
}

}  // namespace

ReconLayout recon_layout(uint32_t U, uint64_t n) {
  ReconLayout L;
  L.num_chunks = (U + (uint64_t)kChunkBins - 1) / kChunkBins;
  L.num_tiles = (n + kTileKeys - 1) / kTileKeys;
  size_t o = 0;
  L.off_ticket = o;
  o = align_up(o + 4, 256);
  L.off_desc = o;
  o = align_up(o + 8 * L.num_chunks, 256);
  L.clear_bytes = o;
  L.off_offsets = o;
  o = align_up(o + 8 * (L.num_chunks + 1), 256);
  L.off_first = o;
  o = align_up(o + 4 * std::max<uint64_t>(L.num_tiles, 1), 256);
  L.total = o;
  return L;
}

cudaError_t launch_offsets(const uint32_t* H, uint32_t U, uint64_t n, void* ws, const ReconLayout& L,
                           uint32_t* err, cudaStream_t stream) {
  char* base = static_cast<char*>(ws);
  cudaError_t e = cudaMemsetAsync(base, 0, L.clear_bytes, stream);
  if (e != cudaSuccess) return e;
  offsets_kernel<<<(unsigned)L.num_chunks, kScanThreads, 0, stream>>>(
      H, U, n, L.num_chunks, reinterpret_cast<uint32_t*>(base + L.off_ticket),
      reinterpret_cast<uint64_t*>(base + L.off_desc), reinterpret_cast<uint64_t*>(base + L.off_offsets),
      reinterpret_cast<uint32_t*>(base + L.off_first), err);
  return cudaGetLastError();
}

cudaError_t launch_expand(const uint32_t* H, uint32_t U, uint64_t n, void* out, uint32_t out_bytes, void* ws,
                          const ReconLayout& L, cudaStream_t stream) {
  if (L.num_tiles == 0) return cudaSuccess;
  char* base = static_cast<char*>(ws);
  const uint64_t* O = reinterpret_cast<const uint64_t*>(base + L.off_offsets);
  const uint32_t* first = reinterpret_cast<const uint32_t*>(base + L.off_first);
  const int aligned = (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  if (out_bytes == 4)
    expand_kernel<uint32_t><<<(unsigned)L.num_tiles, kExpThreads, 0, stream>>>(
        H, U, n, L.num_chunks, O, first, static_cast<uint32_t*>(out), aligned);
  else
    expand_kernel<uint16_t><<<(unsigned)L.num_tiles, kExpThreads, 0, stream>>>(
        H, U, n, L.num_chunks, O, first, static_cast<uint16_t*>(out), aligned);
  return cudaGetLastError();
}

}  // namespace dialsort
