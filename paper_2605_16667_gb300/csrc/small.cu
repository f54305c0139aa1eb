// A whole DialSort of a small input in one cooperative launch.
//
// A small sort is short on work and long on launches: zeroing H, the count,
// the offset scan and the expansion each wait for the previous one.  Here one
// kernel runs them as phases separated by grid-wide barriers (all CTAs are
// resident: cooperative launch; every wait is bounded and records
// ERRBIT_TIMEOUT if it runs out):
//   phase 0  zero H (Eq. (1) starts from H = 0);
//   phase 1  Eq. (1): every CTA counts its share of the keys into a
//            shared-memory sub-histogram (U <= 4096 bins), with the warp CRN
//            merging equal keys, and adds it into H;
//   phase 2  the offsets: chunk sums chained by decoupled look-back;
//   phase 3  Eq. (2): the CTAs claim 8192-key output tiles and expand them.
// The same dynamic shared memory serves the sub-histogram and, afterwards,
// the offset and expansion buffers.
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
  uint32_t arrived;  // grid barrier count (barrier k waits for k * gridDim.x arrivals)
  uint32_t group;    // offset-scan ticket
  uint32_t tile;     // expansion ticket
};

__device__ __forceinline__ void grid_wait(uint32_t* arrived, uint32_t target, uint32_t* err) {
  __threadfence();  // this thread's writes, before the arrival
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(arrived, 1u);
    uint32_t spins = 0;
    while (*reinterpret_cast<volatile uint32_t*>(arrived) < target) {
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

template <typename KeyT, int MODE>
__global__ void __launch_bounds__(kReconThreads) small_sort_kernel(
    const KeyT* __restrict__ keys, uint64_t n, uint32_t U, uint32_t* H, uint32_t words_per_copy, uint32_t crn_mode,
    SmallSync* sync, uint64_t* desc, uint64_t* O, uint32_t* first_chunk, uint64_t num_chunks, KeyT* __restrict__ out,
    int out_aligned, uint32_t* err) {
  extern __shared__ __align__(16) uint32_t sh[];
  __shared__ uint32_t s_t;
  const uint32_t tid = threadIdx.x, warp = tid >> 5;
  const uint32_t G = gridDim.x;
  // ---- phase 0: H = 0, and this CTA's sub-histogram
  for (uint64_t b = (uint64_t)blockIdx.x * kReconThreads + tid; b < U; b += (uint64_t)G * kReconThreads) H[b] = 0u;
  zero_smem(sh, words_per_copy);
  grid_wait(&sync->arrived, G, err);
  // ---- phase 1: count
  {
    const Sink<MODE> s{sh, H, U, 0u};
    bool bad = false;
    ingest_span<KeyT, MODE>(keys, n, U, s, (uint64_t)blockIdx.x * kReconThreads + warp * 32u,
                            (uint64_t)G * kReconThreads, blockIdx.x == G - 1, crn_mode, bad);
    if (bad) raise_error(err, ERRBIT_KEY_RANGE);
    __syncthreads();
    flush_smem<MODE>(sh, 1, words_per_copy, U, H, false);
  }
  grid_wait(&sync->arrived, 2 * G, err);
  // ---- phase 2: offsets (the buffers now overlay the sub-histogram)
  ExpandSmem& ex = *reinterpret_cast<ExpandSmem*>(sh);
  OffsetsSmem& off = *reinterpret_cast<OffsetsSmem*>(reinterpret_cast<char*>(sh) + kOffSmemAt);
  const uint64_t groups = offset_groups(num_chunks);
  for (;;) {
    if (tid == 0) s_t = atomicAdd(&sync->group, 1u);
    __syncthreads();
    const uint64_t g = s_t;
    __syncthreads();
    if (g >= groups) break;
    offsets_group(H, U, n, num_chunks, g, desc, O, first_chunk, err, off);
  }
  grid_wait(&sync->arrived, 3 * G, err);
  // ---- phase 3: expansion
  const uint64_t num_tiles = (n + kTileKeys - 1) / kTileKeys;
  for (;;) {
    if (tid == 0) s_t = atomicAdd(&sync->tile, 1u);
    __syncthreads();
    const uint64_t t = s_t;
    __syncthreads();
    if (t >= num_tiles) break;
    expand_tile<KeyT>(H, U, n, num_chunks, O, first_chunk, out, out_aligned, t, ex, static_cast<const KeyT*>(nullptr));
  }
}

template <typename KeyT, int MODE>
const void* small_kernel() {
  return reinterpret_cast<const void*>(&small_sort_kernel<KeyT, MODE>);
}

}  // namespace

bool small_sort_fits(uint64_t n, uint32_t U, uint32_t key_bytes) {
  // up to 4096 bins: 16 KB sub-histograms, and a merge of U adds per CTA cheap enough to give every
  // input its CTAs (larger universes at these sizes count in L2, the single-pass global regime)
  return n > 0 && n <= kSmallMaxKeys && U <= 4096u && (key_bytes == 4 || key_bytes == 2);
}

cudaError_t launch_small_sort(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H, void* out,
                              void* rws, const ReconLayout& L, const DeviceInfo& dev, uint32_t* err,
                              cudaStream_t stream) {
  // 32-bit counters while they fit in 64 KB, packed 16-bit counters beyond
  const bool u32 = (uint64_t)align_up(U, 4) * 4 <= 64u * 1024u;
  const uint32_t wpc = (uint32_t)(u32 ? align_up(U, 4) : align_up((U + 1u) / 2u, 4));
  const size_t smem = std::max<size_t>((size_t)wpc * 4,
                                       kOffSmemAt + align_up(sizeof(OffsetsSmem), 16));
  const void* fn = key_bytes == 4 ? (u32 ? small_kernel<uint32_t, MODE_SMEM32>() : small_kernel<uint32_t, MODE_SMEM16>())
                                  : (u32 ? small_kernel<uint16_t, MODE_SMEM32>() : small_kernel<uint16_t, MODE_SMEM16>());
  int per_sm = 0;
  cudaError_t e = kernel_config(fn, kReconThreads, smem, false, &per_sm);
  if (e != cudaSuccess) return e;
  // CTAs: for throughput, few enough that the sub-histogram merges (U adds per CTA) stay below about
  // n / 8; for latency, at least one per output tile and per 2048 keys, up to 32 (at most 32 * 4096
  // merge adds)
  const uint64_t by_merge = std::max<uint64_t>(1, n / (8ull * U));
  const uint64_t by_latency = std::min<uint64_t>(32, std::max<uint64_t>(L.num_tiles, (n + 2047) / 2048));
  uint64_t grid = std::max(by_merge, by_latency);
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (uint64_t)dev.sms * std::max(per_sm, 1)));
  char* base = static_cast<char*>(rws);
  e = cudaMemsetAsync(base, 0, L.clear_bytes, stream);  // barrier count, tickets, descriptors
  if (e != cudaSuccess) return e;
  SmallSync* sync = reinterpret_cast<SmallSync*>(base + L.off_ticket);
  uint64_t* desc = reinterpret_cast<uint64_t*>(base + L.off_desc);
  uint64_t* O = reinterpret_cast<uint64_t*>(base + L.off_offsets);
  uint32_t* first = reinterpret_cast<uint32_t*>(base + L.off_first);
  uint64_t nn = n, nc = L.num_chunks;
  uint32_t UU = U, crn = 2, wpcv = wpc;  // crn 2: the adaptive CRN
  int aligned = (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  void* args[] = {const_cast<void**>(&keys), &nn, &UU, &H, &wpcv, &crn, &sync, &desc, &O,
                  &first, &nc, &out, &aligned, &err};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kReconThreads), args, smem, stream);
}

}  // namespace dialsort
