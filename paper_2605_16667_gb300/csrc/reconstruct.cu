// Step 2 of DialSort: the ordered projection, Eq. (2) -- for k = 0..U-1 emit
// k exactly H[k] times.
//
// The sequential projection keeps one cursor; to write runs in parallel each
// run needs its start, sum_{j<k} H[j] (the cursor on reaching k).  The paper
// says DialSort needs no prefix sum; that holds for the single cursor only, so
// this file computes the starts at two granularities and keeps the fine one
// on chip:
//
//   offsets kernel  one CTA per group of eight 1024-bin chunks (a warp per
//                   chunk): chunk totals, an exclusive scan across groups by
//                   decoupled look-back, each chunk's run start O[c] and, for
//                   every 8192-key output tile that starts inside a chunk's run
//                   range, the tile's first chunk.  Reads H once (4U bytes);
//                   writes about 9 bytes per chunk and 4 per tile.
//   expand kernel   one CTA per output tile.  Its warps share out the chunks
//                   that overlap the tile, scan each chunk's bins with warp
//                   shuffles to get run starts, and mark in a tile-sized buffer
//                   the slot where each run starts (slot 0 gets the run
//                   covering the tile's first key).  A fill-forward scan
//                   ("latest mark wins") turns marks into keys, which go out
//                   with 128-bit stores.
//
// No key is compared with another: searches and scans act on counts and
// output positions only.  Load balance is by output position, so one bin with
// H[k] = n (all keys equal) spreads over all tiles.
#include <cstddef>

#include "recon_device.cuh"

namespace dialsort {

namespace {

__global__ void __launch_bounds__(kReconThreads) offsets_kernel(const uint32_t* __restrict__ H, uint32_t U,
                                                                uint64_t n_cap, uint64_t num_chunks,
                                                                uint32_t* ticket, uint64_t* desc, uint64_t* O,
                                                                uint32_t* first_chunk, uint32_t* err) {
  __shared__ OffsetsSmem sm;
  __shared__ uint32_t s_g;
  if (threadIdx.x == 0) s_g = atomicAdd(ticket, 1u);  // dynamic order: every lower group is already running or done
  __syncthreads();
  offsets_group(H, U, n_cap, num_chunks, s_g, desc, O, first_chunk, err, sm);
}

template <typename OutT>
__global__ void __launch_bounds__(kReconThreads, 6) expand_kernel(const uint32_t* __restrict__ H, uint32_t U,
                                                                  uint64_t n_cap, uint64_t num_chunks,
                                                                  const uint64_t* __restrict__ O,
                                                                  const uint32_t* __restrict__ first_chunk,
                                                                  OutT* __restrict__ out, int out_aligned,
                                                                  const OutT* __restrict__ inv) {
  __shared__ __align__(16) ExpandSmem sm;
  expand_tile<OutT>(H, U, n_cap, num_chunks, O, first_chunk, out, out_aligned, blockIdx.x, sm, inv);
}


// ---------------------------------------------------------------- fused projection
// The offsets and the expansion in one launch.  Work items are handed out in
// one ticket order: first the groups of eight 1024-bin chunks of the offset
// scan (chunk sums chained by decoupled look-back: O[c], and each output
// tile's first chunk), then the 8192-key output tiles.  A CTA holding a tile
// first waits (bounded) until every group is done; every group has a lower
// ticket, so it is held by a running CTA or finished, and the wait ends
// without any assumption about how many CTAs are resident.
// With phase_mask = 1 only the groups are handed out: the offsets step timed
// on its own.
struct ProjSmem {
  __align__(16) ExpandSmem ex;  // first, 16-byte aligned: its tile buffer is read and written as uint4
  OffsetsSmem off;
  uint32_t k;  // ticket
};
static_assert(offsetof(ProjSmem, ex) % 16 == 0, "the expansion buffer must be 16-byte aligned");

// Counters of one projection (in the zeroed part of the workspace).
struct ProjCtl {
  uint32_t ticket;       // next work item
  uint32_t groups_done;  // finished groups of the offset scan
};

template <typename OutT>
__global__ void __launch_bounds__(kReconThreads) project_kernel(const uint32_t* __restrict__ H, uint32_t U,
                                                                uint64_t n_cap, uint64_t num_chunks, ProjCtl* ctl,
                                                                uint64_t* desc, uint64_t* O, uint32_t* first_chunk,
                                                                OutT* __restrict__ out, int out_aligned,
                                                                const OutT* __restrict__ inv, uint32_t* err,
                                                                int phase_mask, int by_bins) {
  __shared__ __align__(16) ProjSmem sm;
  const uint32_t tid = threadIdx.x;
  const uint64_t groups = offset_groups(num_chunks);
  // expansion items: output tiles, or (a sparse H, by_bins) the offsets' chunk groups again
  const uint64_t tiles = !(phase_mask & 2) ? 0 : by_bins ? groups : (n_cap + kTileKeys - 1) / kTileKeys;
  bool waited = false;
  for (;;) {
    if (tid == 0) sm.k = atomicAdd(&ctl->ticket, 1u);
    __syncthreads();
    const uint64_t k = sm.k;
    __syncthreads();
    if (k >= groups + tiles) break;
    if (k < groups) {
      offsets_group(H, U, n_cap, num_chunks, k, desc, O, first_chunk, err, sm.off);
      __threadfence();  // every thread's O and table writes, before the group counts as done
      __syncthreads();
      if (tid == 0) atomicAdd(&ctl->groups_done, 1u);
      continue;
    }
    if (!waited) {  // the offsets are complete before any tile is expanded
      if (tid == 0) {
        uint32_t spins = 0;
        while (*reinterpret_cast<volatile uint32_t*>(&ctl->groups_done) < groups) {
          if (++spins > kSpinLimit) {
            raise_error(err, ERRBIT_TIMEOUT);
            break;
          }
          __nanosleep(64);
        }
        __threadfence();
      }
      __syncthreads();
      waited = true;
    }
    if (by_bins)
      expand_bins<OutT>(H, U, n_cap, num_chunks, O, out, k - groups, inv);
    else
      expand_tile<OutT>(H, U, n_cap, num_chunks, O, first_chunk, out, out_aligned, k - groups, sm.ex, inv);
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
  o = align_up(o + 8 * offset_groups(L.num_chunks), 256);
  L.clear_bytes = o;
  L.off_offsets = o;
  o = align_up(o + 8 * (L.num_chunks + 1), 256);
  L.off_first = o;
  o = align_up(o + 4 * std::max<uint64_t>(L.num_tiles, 1), 256);
  L.total = o;
  return L;
}

// Self-test of the bounded look-back wait: one CTA scans group 1 of a 16-chunk
// histogram whose group 0 is never scanned (the ticket starts at 1), so its
// wait for group 0's descriptor runs out and records ERRBIT_TIMEOUT.
size_t offsets_selftest_bytes() { return recon_layout(16 * kChunkBins, 0).total + 4 * 16 * (size_t)kChunkBins; }

cudaError_t launch_offsets_selftest(void* ws, uint32_t* err, cudaStream_t stream) {
  const uint32_t U = 16 * kChunkBins;
  const ReconLayout L = recon_layout(U, 0);
  char* base = static_cast<char*>(ws);
  uint32_t* H = reinterpret_cast<uint32_t*>(base + L.total);
  cudaError_t e = cudaMemsetAsync(base, 0, L.total + 4 * (size_t)U, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + L.off_ticket, 1, 1, stream);  // ticket = 1
  if (e != cudaSuccess) return e;
  offsets_kernel<<<1, kReconThreads, 0, stream>>>(H, U, 0, L.num_chunks,
                                                  reinterpret_cast<uint32_t*>(base + L.off_ticket),
                                                  reinterpret_cast<uint64_t*>(base + L.off_desc),
                                                  reinterpret_cast<uint64_t*>(base + L.off_offsets),
                                                  reinterpret_cast<uint32_t*>(base + L.off_first), err);
  return cudaGetLastError();
}

cudaError_t launch_offsets(const uint32_t* H, uint32_t U, uint64_t n, void* ws, const ReconLayout& L,
                           uint32_t* err, cudaStream_t stream) {
  char* base = static_cast<char*>(ws);
  cudaError_t e = cudaMemsetAsync(base, 0, L.clear_bytes, stream);
  if (e != cudaSuccess) return e;
  offsets_kernel<<<(unsigned)offset_groups(L.num_chunks), kReconThreads, 0, stream>>>(
      H, U, n, L.num_chunks, reinterpret_cast<uint32_t*>(base + L.off_ticket),
      reinterpret_cast<uint64_t*>(base + L.off_desc), reinterpret_cast<uint64_t*>(base + L.off_offsets),
      reinterpret_cast<uint32_t*>(base + L.off_first), err);
  return cudaGetLastError();
}

cudaError_t launch_expand(const uint32_t* H, uint32_t U, uint64_t n, void* out, uint32_t out_bytes, void* ws,
                          const ReconLayout& L, cudaStream_t stream, const void* inv) {
  if (L.num_tiles == 0) return cudaSuccess;
  char* base = static_cast<char*>(ws);
  const uint64_t* O = reinterpret_cast<const uint64_t*>(base + L.off_offsets);
  const uint32_t* first = reinterpret_cast<const uint32_t*>(base + L.off_first);
  const int aligned = (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  // 6 CTAs of 32 KB per SM need the large shared-memory carve-out
  const void* fn = out_bytes == 4   ? reinterpret_cast<const void*>(&expand_kernel<uint32_t>)
                   : out_bytes == 2 ? reinterpret_cast<const void*>(&expand_kernel<uint16_t>)
                                    : reinterpret_cast<const void*>(&expand_kernel<uint8_t>);
  cudaError_t e = kernel_config(fn, kReconThreads, 0, true, nullptr);
  if (e != cudaSuccess) return e;
  if (out_bytes == 4)
    expand_kernel<uint32_t><<<(unsigned)L.num_tiles, kReconThreads, 0, stream>>>(
        H, U, n, L.num_chunks, O, first, static_cast<uint32_t*>(out), aligned, static_cast<const uint32_t*>(inv));
  else if (out_bytes == 2)
    expand_kernel<uint16_t><<<(unsigned)L.num_tiles, kReconThreads, 0, stream>>>(
        H, U, n, L.num_chunks, O, first, static_cast<uint16_t*>(out), aligned, static_cast<const uint16_t*>(inv));
  else
    expand_kernel<uint8_t><<<(unsigned)L.num_tiles, kReconThreads, 0, stream>>>(
        H, U, n, L.num_chunks, O, first, static_cast<uint8_t*>(out), aligned, static_cast<const uint8_t*>(inv));
  return cudaGetLastError();
}

}  // namespace dialsort

namespace dialsort {

cudaError_t launch_projection(const uint32_t* H, uint32_t U, uint64_t n, void* out, uint32_t out_bytes, void* ws,
                              const ReconLayout& L, const DeviceInfo& dev, uint32_t* err, cudaStream_t stream,
                              const void* inv, int phase_mask) {
  char* base = static_cast<char*>(ws);
  cudaError_t e = cudaMemsetAsync(base, 0, L.clear_bytes, stream);  // counters, descriptors
  if (e != cudaSuccess) return e;
  const void* fn = out_bytes == 4   ? reinterpret_cast<const void*>(&project_kernel<uint32_t>)
                   : out_bytes == 2 ? reinterpret_cast<const void*>(&project_kernel<uint16_t>)
                                    : reinterpret_cast<const void*>(&project_kernel<uint8_t>);
  // six CTAs of 35 KB per SM need the large shared-memory carve-out
  int per_sm = 0;
  e = kernel_config(fn, kReconThreads, 0, true, &per_sm);
  if (e != cudaSuccess) return e;
  // a sparse H (fewer keys than bins / 4): bin-parallel expansion over the chunk groups
  const int by_bins = 4 * n < (uint64_t)U ? 1 : 0;
  const uint64_t work = offset_groups(L.num_chunks) +
                        (phase_mask & 2 ? (by_bins ? offset_groups(L.num_chunks) : L.num_tiles) : 0);
  const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)dev.sms * std::max(per_sm, 1), std::max<uint64_t>(work, 1));
  ProjCtl* ctl = reinterpret_cast<ProjCtl*>(base + L.off_ticket);  // in the zeroed region
  uint64_t* desc = reinterpret_cast<uint64_t*>(base + L.off_desc);
  uint64_t* O = reinterpret_cast<uint64_t*>(base + L.off_offsets);
  uint32_t* first = reinterpret_cast<uint32_t*>(base + L.off_first);
  const int aligned = (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  if (out_bytes == 4)
    project_kernel<uint32_t><<<grid, kReconThreads, 0, stream>>>(H, U, n, L.num_chunks, ctl, desc, O, first,
                                                                 static_cast<uint32_t*>(out), aligned,
                                                                 static_cast<const uint32_t*>(inv), err, phase_mask,
                                                                 by_bins);
  else if (out_bytes == 2)
    project_kernel<uint16_t><<<grid, kReconThreads, 0, stream>>>(H, U, n, L.num_chunks, ctl, desc, O, first,
                                                                 static_cast<uint16_t*>(out), aligned,
                                                                 static_cast<const uint16_t*>(inv), err, phase_mask,
                                                                 by_bins);
  else
    project_kernel<uint8_t><<<grid, kReconThreads, 0, stream>>>(H, U, n, L.num_chunks, ctl, desc, O, first,
                                                                static_cast<uint8_t*>(out), aligned,
                                                                static_cast<const uint8_t*>(inv), err, phase_mask,
                                                                by_bins);
  return cudaGetLastError();
}

}  // namespace dialsort
