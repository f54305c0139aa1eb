// Host-side declarations shared by the translation units of libdialsort.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dialsort.h"

namespace dialsort {

struct DeviceInfo {
  int device = -1;
  int sms = 0;
  size_t smem_optin = 0;  // max dynamic shared memory per CTA (opt-in)
  uint32_t* err = nullptr;  // device address of the per-device error word
  bool pageable = false;    // kernels may dereference pageable host memory (coherent host page tables)
};

// The address a kernel dereferences for a caller's pointer: device or managed
// memory of this device as is, page-locked host memory through its mapped
// address, pageable host memory only where dev.pageable.  INVALID_ARG for
// memory this device cannot reach.
dialsort_status_t kernel_address(const void* p, const DeviceInfo& dev, const void** q, bool* in_host = nullptr);

// Per-device properties and error word; initialised once per device, with
// that device current.  Returns nullptr when no device is usable.
const DeviceInfo* device_info();

// Launch set-up of a kernel on the current device, done once per (device, kernel): its dynamic
// shared-memory limit raised to the device's opt-in maximum and, with carveout_max, the shared-memory
// carve-out preferred; *per_sm (optional) receives its resident CTAs per SM for the given block size and
// dynamic shared memory, also computed once per configuration.
cudaError_t kernel_config(const void* fn, int threads, size_t dyn_smem, bool carveout_max, int* per_sm);

// Fully resolved launch choices for step 1.
struct HistPlan {
  uint32_t regime = DIALSORT_REGIME_GLOBAL_CRN;
  uint32_t crn = 2;  // 0 off, 1 on, 2 adaptive (hist.cu CrnMode)
  uint32_t blocks = 0;
  uint32_t threads = 1024;
  uint32_t replicas = 1;
  uint32_t cluster = 1;
  uint32_t words_per_copy = 0;  // 32-bit words per shared-memory sub-histogram copy
  size_t smem_bytes = 0;        // dynamic shared memory per CTA
  bool tuned = false;           // taken from the measured tuning table
};

// Fills every field of a plan (the autotuner); cfg fields that are non-zero
// are taken as given.  Returns INVALID_ARG when a forced choice cannot work.
// With use_table and an all-automatic cfg, the measured tuning table's entry
// for (n, U, key_bytes, skew_hint) is tried first (plan->tuned says so).
dialsort_status_t plan_histogram(uint64_t n, uint32_t U, uint32_t key_bytes, uint32_t skew_hint,
                                 const dialsort_hist_config_t* cfg, const DeviceInfo& dev, HistPlan* plan,
                                 bool use_table = true);

// The tuning table's entry nearest to (n, U) for this key width and skew
// class, as launch choices (blocks left 0; blocks_per_sm separately, 0 =
// automatic).  False when the table has nothing near.
bool tuned_choice(uint64_t n, uint32_t U, uint32_t key_bytes, uint32_t skew, dialsort_hist_config_t* cfg,
                  uint32_t* blocks_per_sm);
// The skew class (dialsort_skew_class_t) of the probe's counts {samples,
// equal neighbours, neighbour pairs, top multiplicity}.
uint32_t skew_class_of(const uint32_t stats[4], uint32_t U);

// Step 1 kernels (H must already be zero).  hist.cu
// phi (optional): index = phi[key] for keys < M (see KeyMap); key_bytes 1, 2 or 4.
cudaError_t launch_histogram(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H,
                             const HistPlan& plan, uint32_t* err, cudaStream_t stream,
                             const uint32_t* phi = nullptr, uint32_t M = 0);

// Two-level ingestion for large universes.  hist2.cu
struct TwoLevelLayout {
  uint32_t L = 0, B = 0;          // low bits per key; buckets = ceil(U / 2^L)
  uint64_t num_tiles = 0, item_keys = 0, max_items = 0;
  size_t off_low = 0, off_toff = 0, off_tcnt = 0, off_btot = 0, off_items = 0, off_nitems = 0, off_pbase = 0;
  size_t total = 0;
  bool p2_smem32 = true;          // pass-2 histograms in 32-bit counters (else packed 16-bit)
  uint32_t words_per_copy = 0;
};
TwoLevelLayout two_level_layout(uint64_t n, uint32_t U);
// Whether the two-level path applies (uint32 keys, 16-byte aligned, enough keys, bucket count in range).
bool two_level_shape_fits(uint64_t n, uint32_t U, uint32_t key_bytes);
bool two_level_fits(uint64_t n, uint32_t U, uint32_t key_bytes, const void* keys);
cudaError_t launch_two_level(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H, void* ws,
                             const TwoLevelLayout& T, uint32_t crn_mode, const DeviceInfo& dev, uint32_t* err,
                             cudaStream_t stream, bool accumulate);

// Two-level ingestion with per-(bucket, lane) partition counters for 2^16 < U <= 2^21.  hier.cu
struct HierLayout {
  uint32_t B = 0, BM = 0;        // buckets of 2^15 bins; bucket slots of the partition kernel (32 or 64)
  uint64_t num_tiles = 0;        // 8192-key tiles
  uint32_t S_t = 0;              // staged entries per tile in the workspace
  uint32_t G_max = 0;            // pass-2 CTAs the scratch has room for
  size_t off_low = 0, off_seg = 0, off_btot = 0, off_start = 0, off_used = 0, off_part = 0;
  // the sort's fused count + projection: cleared words (ticket, bucket counters, look-back descriptors),
  // then its count ranges, item order, pieces per bucket and bucket bases
  size_t off_fclear = 0, fclear_bytes = 0, off_fstart = 0, off_sched = 0, off_pieces = 0, off_bbase = 0;
  size_t off_longs = 0, off_pmap = 0;  // runs too long for one warp, and the map of their pieces
  size_t total = 0;
};
constexpr uint32_t kHierMaxCountCtas = 256;  // pass-2 CTAs (one per SM) at most
// Pass-2 CTAs for n keys on a GPU with `sms` SMs (no more than the workspace has room for).
uint32_t hier_count_ctas(uint64_t n, uint32_t sms);
HierLayout hier_layout(uint64_t n, uint32_t U);
bool hier_shape_fits(uint64_t n, uint32_t U, uint32_t key_bytes);
bool hier_fits(uint64_t n, uint32_t U, uint32_t key_bytes, const void* keys);
cudaError_t launch_hier(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H, void* ws, const HierLayout& T,
                        const DeviceInfo& dev, uint32_t* err, cudaStream_t stream, bool accumulate);
// The whole sort of uint32 keys in the two-level form: pass 1, then counting fused with the projection
// (Eq. (2)) into out (n_cap keys); H receives the histogram.
// marks (or NULL): three events recorded after pass 1, after the split and schedule, and after the fused
// kernel (the long-run painter follows).
cudaError_t launch_hier_sort(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H, uint32_t* out, void* ws,
                             const HierLayout& T, const DeviceInfo& dev, uint32_t* err, cudaStream_t stream,
                             cudaEvent_t* marks = nullptr);

// Self-tests of the bounded device waits (a wait that is made to run out).
size_t offsets_selftest_bytes();
cudaError_t launch_offsets_selftest(void* ws, uint32_t* err, cudaStream_t stream);
size_t radix_selftest_bytes();
cudaError_t launch_radix_selftest(void* ws, uint32_t* err, cudaStream_t stream);

// Step 2.  reconstruct.cu
constexpr uint32_t kChunkBins = 1024;  // bins per offset-scan chunk
constexpr uint32_t kTileKeys = 8192;   // output keys per expansion tile

struct ReconLayout {
  uint64_t num_chunks = 0, num_tiles = 0;
  size_t off_ticket = 0, off_desc = 0, off_offsets = 0, off_first = 0;
  size_t clear_bytes = 0;  // bytes at the start of the workspace zeroed before each scan
  size_t total = 0;
};
ReconLayout recon_layout(uint32_t U, uint64_t n);

cudaError_t launch_offsets(const uint32_t* H, uint32_t U, uint64_t n, void* ws, const ReconLayout& L,
                           uint32_t* err, cudaStream_t stream);
// The projection with its offsets in one launch (offset-scan groups, then output tiles, in one ticket
// order).  phase_mask 1: the offsets only (O[] and the tile table written); 3: both.
cudaError_t launch_projection(const uint32_t* H, uint32_t U, uint64_t n, void* out, uint32_t out_bytes, void* ws,
                              const ReconLayout& L, const DeviceInfo& dev, uint32_t* err, cudaStream_t stream,
                              const void* inv = nullptr, int phase_mask = 3);
// A whole sort of a small input (n <= 2^22, U <= 4096) in one launch (zero H, count, offsets, expand;
// rws is the reconstruction scratch).  small.cu
bool small_sort_fits(uint64_t n, uint32_t U, uint32_t key_bytes);
cudaError_t launch_small_sort(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H, void* out,
                              void* rws, const ReconLayout& L, const DeviceInfo& dev, uint32_t* err,
                              cudaStream_t stream);
// inv (optional): index k is written as inv[k] (an array of out_bytes-wide values); out_bytes 1, 2 or 4.
cudaError_t launch_expand(const uint32_t* H, uint32_t U, uint64_t n, void* out, uint32_t out_bytes, void* ws,
                          const ReconLayout& L, cudaStream_t stream, const void* inv = nullptr);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The status every entry point returns for a CUDA runtime result.
inline dialsort_status_t from_cuda(cudaError_t e) { return e == cudaSuccess ? DIALSORT_OK : DIALSORT_ERR_CUDA; }

}  // namespace dialsort
