// A whole DialSort of a small input in one launch.
//
// A small sort is short on work and long on launches: zeroing H, the count,
// the offset scan and the expansion each wait for the previous one.  Here one
// kernel hands out their work items in one ticket order, each phase's items
// after all of the previous phase's:
//   zero   H = 0 (Eq. (1) starts from H = 0);
//   count  Eq. (1) on a range of the keys: a shared-memory sub-histogram
//          (U <= 4096 bins) filled with the warp CRN merging equal keys, then
//          added into H;
//   group  the offsets: eight 1024-bin chunks summed and chained to the
//          earlier groups by decoupled look-back;
//   tile   Eq. (2) on an 8192-key output tile.
// An item of one phase first waits (bounded; ERRBIT_TIMEOUT if it runs out)
// until every item of the previous phase is done.  Those items have lower
// tickets, so they are held by running CTAs or finished: the waits end
// whatever the number of resident CTAs.  The same dynamic shared memory
// serves the sub-histogram, the offset buffers and the expansion buffers.
#include <algorithm>
#include <cstddef>

#include "hist_device.cuh"
#include "internal.h"
#include "recon_device.cuh"

namespace dialsort {

namespace {

constexpr uint64_t kSmallMaxKeys = 1ull << 22;
// where the offset buffers start in the dynamic shared memory (after the expansion buffers, 16-byte aligned)
constexpr size_t kOffSmemAt = (sizeof(ExpandSmem) + 15) / 16 * 16;

struct SmallSync {
  uint32_t ticket;  // next work item
  uint32_t done[3]; // finished items of the zero, count and group phases
};

// Thread 0 waits until at least `target` items of a phase are done; then the CTA goes on.
__device__ __forceinline__ void wait_phase(uint32_t* done, uint32_t target, uint32_t* err) {
  if (threadIdx.x == 0) {
    uint32_t spins = 0;
    while (*reinterpret_cast<volatile uint32_t*>(done) < target) {
      if (++spins > kSpinLimit) {
        raise_error(err, ERRBIT_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

// An item is done: every thread's writes are fenced before the count goes up.
__device__ __forceinline__ void item_done(uint32_t* done) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(done, 1u);
}

template <typename KeyT, int MODE>
__global__ void __launch_bounds__(kReconThreads) small_sort_kernel(
    const KeyT* __restrict__ keys, uint64_t n, uint32_t U, uint32_t* H, uint32_t words_per_copy, uint32_t crn_mode,
    uint32_t count_items, SmallSync* sync, uint64_t* desc, uint64_t* O, uint32_t* first_chunk, uint64_t num_chunks,
    KeyT* __restrict__ out, int out_aligned, uint32_t* err) {
  extern __shared__ __align__(16) uint32_t sh[];
  __shared__ uint32_t s_k;
  const uint32_t tid = threadIdx.x, warp = tid >> 5;
  constexpr uint32_t kZeroBins = 4096;
  const uint32_t zero_items = (U + kZeroBins - 1) / kZeroBins;
  const uint32_t groups = (uint32_t)offset_groups(num_chunks);
  const uint64_t tiles = (n + kTileKeys - 1) / kTileKeys;
  const uint64_t c0 = zero_items, g0 = c0 + count_items, t0 = g0 + groups, end = t0 + tiles;
  ExpandSmem& ex = *reinterpret_cast<ExpandSmem*>(sh);
  OffsetsSmem& off = *reinterpret_cast<OffsetsSmem*>(reinterpret_cast<char*>(sh) + kOffSmemAt);
  for (;;) {
    if (tid == 0) s_k = atomicAdd(&sync->ticket, 1u);
    __syncthreads();
    const uint64_t k = s_k;
    __syncthreads();
    if (k >= end) break;
    if (k < c0) {  // zero: bins [4096 k, 4096 k + 4096)
      for (uint64_t b = k * kZeroBins + tid; b < U && b < (k + 1) * kZeroBins; b += kReconThreads) H[b] = 0u;
      item_done(&sync->done[0]);
    } else if (k < g0) {  // count: keys [c n / C, (c + 1) n / C)
      const uint64_t c = k - c0;
      const uint64_t lo = n * c / count_items, hi = n * (c + 1) / count_items;
      zero_smem(sh, words_per_copy);
      wait_phase(&sync->done[0], zero_items, err);  // also orders the zeroing of sh
      const Sink<MODE> s{sh, H, U, 0u};
      bool bad = false;
      ingest_span<KeyT, MODE>(keys + lo, hi - lo, U, s, warp * 32u, kReconThreads, true, crn_mode, bad);
      if (bad) raise_error(err, ERRBIT_KEY_RANGE);
      __syncthreads();
      flush_smem<MODE>(sh, 1, words_per_copy, U, H, false);
      item_done(&sync->done[1]);
    } else if (k < t0) {  // an offset-scan group
      wait_phase(&sync->done[1], count_items, err);
      offsets_group(H, U, n, num_chunks, k - g0, desc, O, first_chunk, err, off);
      item_done(&sync->done[2]);
    } else {  // an output tile
      wait_phase(&sync->done[2], groups, err);
      expand_tile<KeyT>(H, U, n, num_chunks, O, first_chunk, out, out_aligned, k - t0, ex,
                        static_cast<const KeyT*>(nullptr));
    }
  }
}

template <typename KeyT, int MODE>
const void* small_kernel() {
  return reinterpret_cast<const void*>(&small_sort_kernel<KeyT, MODE>);
}

}  // namespace

bool small_sort_fits(uint64_t n, uint32_t U, uint32_t key_bytes) {
  // up to 4096 bins: 16 KB sub-histograms, and a merge of U adds per count item cheap enough to give
  // every input its CTAs (larger universes at these sizes count in L2, the single-pass global regime)
  return n > 0 && n <= kSmallMaxKeys && U <= 4096u && (key_bytes == 4 || key_bytes == 2);
}

cudaError_t launch_small_sort(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H, void* out,
                              void* rws, const ReconLayout& L, const DeviceInfo& dev, uint32_t* err,
                              cudaStream_t stream) {
  const uint32_t wpc = (uint32_t)align_up(U, 4);  // 32-bit counters (U <= 4096: 16 KB)
  const size_t smem = std::max<size_t>((size_t)wpc * 4, kOffSmemAt + align_up(sizeof(OffsetsSmem), 16));
  const void* fn = key_bytes == 4 ? small_kernel<uint32_t, MODE_SMEM32>() : small_kernel<uint16_t, MODE_SMEM32>();
  int per_sm = 0;
  cudaError_t e = kernel_config(fn, kReconThreads, smem, true, &per_sm);
  if (e != cudaSuccess) return e;
  // count items: for throughput few enough that the sub-histogram merges (U adds each) stay below about
  // n / 8; for latency at least one per output tile and per 2048 keys, up to 32
  const uint64_t by_merge = std::max<uint64_t>(1, n / (8ull * U));
  const uint64_t by_latency = std::min<uint64_t>(32, std::max<uint64_t>(L.num_tiles, (n + 2047) / 2048));
  const uint64_t resident = (uint64_t)dev.sms * std::max(per_sm, 1);
  const uint32_t count_items = (uint32_t)std::max<uint64_t>(1, std::min(std::max(by_merge, by_latency), resident));
  const uint64_t items = (U + 4095) / 4096 + count_items + offset_groups(L.num_chunks) + L.num_tiles;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min(items, resident));
  char* base = static_cast<char*>(rws);
  e = cudaMemsetAsync(base, 0, L.clear_bytes, stream);  // ticket, phase counters, descriptors
  if (e != cudaSuccess) return e;
  SmallSync* sync = reinterpret_cast<SmallSync*>(base + L.off_ticket);
  uint64_t* desc = reinterpret_cast<uint64_t*>(base + L.off_desc);
  uint64_t* O = reinterpret_cast<uint64_t*>(base + L.off_offsets);
  uint32_t* first = reinterpret_cast<uint32_t*>(base + L.off_first);
  const int aligned = (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  if (key_bytes == 4)
    small_sort_kernel<uint32_t, MODE_SMEM32><<<grid, kReconThreads, smem, stream>>>(
        static_cast<const uint32_t*>(keys), n, U, H, wpc, 2u, count_items, sync, desc, O, first, L.num_chunks,
        static_cast<uint32_t*>(out), aligned, err);
  else
    small_sort_kernel<uint16_t, MODE_SMEM32><<<grid, kReconThreads, smem, stream>>>(
        static_cast<const uint16_t*>(keys), n, U, H, wpc, 2u, count_items, sync, desc, O, first, L.num_chunks,
        static_cast<uint16_t*>(out), aligned, err);
  return cudaGetLastError();  // crn 2 above: the adaptive CRN
}

}  // namespace dialsort
