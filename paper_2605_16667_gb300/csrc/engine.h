// Shared definitions of the request engine (engine.cu) and the server (serve.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace dialsort {
namespace eng {

constexpr uint32_t kThreads = 256;       // worker CTA size (the step-2 routines assume 256)
constexpr uint32_t kZeroWords = 16384;   // H words zeroed per zero item (64 KB; batched: x kBatchedZeroScale)
constexpr uint32_t kWindow = 256;        // requests examined per work search (one per thread)
constexpr uint32_t kQuickCtas = 32;      // served mode: CTAs that watch the doorbell (fast pick-up)
constexpr uint32_t kHistSmem = 48 * 1024;  // dynamic shared memory for shared-memory histogram items
// Batched mode: a claim costs a few microseconds of L2 round trips, so its items carry more work (the
// zero phase's words, the offsets groups, the output tiles (or sparse chunk groups) and the histogram's
// keys, times these factors; measured on the batched configuration: 9.1 ms with 4 / 4 / 8 / 4, 8.4 ms
// with these).  Served mode keeps small items: one request then spreads over every CTA.
constexpr uint32_t kBatchedZeroScale = 16;
constexpr uint32_t kBatchedOffsPerItem = 16;
constexpr uint32_t kBatchedExpandPerItem = 32;
constexpr uint32_t kBatchedHistScale = 4;

// Two-level ingestion inside the engine (universes past the shared-memory
// sub-histogram, up to 2^22 bins): bucket = key >> 14.  A partition item
// groups the in-range keys of one 8192-key tile by bucket and writes their
// low 14 bits (uint16) to the request's scratch, with one segment word per
// (tile, bucket); a histogram item then counts one bucket's low parts over a
// range of tiles in packed 16-bit shared-memory counters (32 KB) and adds
// them into H.
constexpr uint32_t kPartKeys = 8192;
constexpr uint32_t kBucketBits = 14;
constexpr uint32_t kMaxBuckets = 256;
constexpr uint32_t MODE_TWO_LEVEL_ENG = 3;  // Req.mode beside hist_device.cuh's HistMode values

// Phases in order; a request skips those with no items.
enum Phase : uint32_t {
  PH_FREE = 0,
  PH_ZERO = 1,
  PH_PART = 2,  // two-level only: partition tiles by bucket
  PH_HIST = 3,
  PH_OFFS = 4,
  PH_EXPAND = 5,
  PH_DONE = 6
};
constexpr uint32_t kPhases = 5;  // work phases PH_ZERO .. PH_EXPAND

// Immutable description of one request (device memory).
struct Req {
  const void* keys;
  uint32_t* H;
  void* out;          // nullptr: histogram only
  uint64_t* desc;     // look-back descriptors (zeroed before the request starts)
  uint64_t* O;        // chunk offsets
  uint32_t* first;    // first chunk of each output tile
  uint64_t n;
  uint64_t item_keys; // keys per histogram item
  uint32_t U;
  uint32_t key_bytes;
  uint32_t mode;      // hist_device.cuh HistMode
  uint32_t crn;       // hist_device.cuh CrnMode
  uint32_t replicas;
  uint32_t words_per_copy;
  uint32_t owned;     // the single histogram item stores every bin of H (H needs no zeroing)
  uint32_t out_aligned;
  uint32_t count[kPhases];  // items of the zero, partition, histogram, offsets and expand phases
  uint32_t first_phase;
  uint32_t zero_H;    // the zero phase clears H[0..U) before clearing desc
  uint32_t buckets;   // two-level: buckets of 2^kBucketBits bins
  uint32_t by_bins;   // the expand phase is bin-parallel (expand_bins: a sparse H), over the offsets groups
  uint32_t zero_words_item;  // H / descriptor words per zero item
  uint32_t offs_per_item;    // offsets groups per offsets item
  uint32_t expand_per_item;  // output tiles (or sparse chunk groups) per expand item
  uint16_t* low;      // two-level: low parts, kPartKeys per partition tile
  uint32_t* seg;      // two-level: per (tile, bucket) start | count << 16 within the tile
};

// Mutable progress of one request (device memory).  One 64-bit word holds
// the low 32 bits of the request's admission sequence number, its phase and
// the number of items of that phase handed out:
//     word = seq32 << 32 | phase << 24 | next          (next < 2^24)
// A CTA claims with a plain atomicAdd(word, 1) and reads what it claimed from
// the returned value, so every claim is self-describing: if the phase moved
// on, or (served mode) the slot was given to a new request, between the CTA's
// look and its add, the CTA has claimed a genuine item of the new phase or
// request and does that one.  A claim whose phase is not a work phase, or
// whose index is past the phase's item count, claims nothing.
struct State {
  unsigned long long word;
  unsigned long long seq;       // admission order (smaller = older = served first)
  unsigned long long t_done;    // %globaltimer when the request finished
  uint32_t done[kPhases];       // items finished, per phase
  uint32_t err;                 // error bits of this request
  uint32_t pad[4];
};
static_assert(sizeof(State) == 64, "State is one 64-byte record");

__host__ __device__ inline unsigned long long pack_word(uint64_t seq, uint32_t phase, uint32_t next) {
  return ((unsigned long long)(uint32_t)seq << 32) | ((unsigned long long)(phase & 0xffu) << 24) |
         (unsigned long long)(next & 0xffffffu);
}
__host__ __device__ inline uint32_t word_phase(unsigned long long w) { return (uint32_t)(w >> 24) & 0xffu; }
__host__ __device__ inline uint32_t word_next(unsigned long long w) { return (uint32_t)w & 0xffffffu; }
__host__ __device__ inline uint32_t word_seq(unsigned long long w) { return (uint32_t)(w >> 32); }

// Completion record in host-mapped memory (served mode).
struct Completion {
  volatile uint64_t seq_done;  // = State.seq + 1 once the request is finished
  volatile uint64_t t_done;
  volatile uint32_t err;
  uint32_t pad[3];
};

// Control words in host-mapped memory (served mode).
struct HostCtl {
  volatile uint32_t stop;      // host: workers exit once nothing is left to do
  volatile uint32_t running;   // device: CTAs currently inside the worker loop
  uint32_t pad[14];
};

// Control words in device memory.
struct Ctl {
  uint32_t tail;                 // batched mode: every request below tail is finished
  uint32_t pad0;
  unsigned long long last_work;  // %globaltimer of the latest claimed item (any CTA)
  unsigned long long bell;       // served mode: admissions so far, written by DMA after each slot is published
  uint32_t pad[58];
};

struct Launch {
  const Req* reqs;
  State* st;
  Ctl* ctl;
  Completion* comp;   // served mode only
  HostCtl* host;      // served mode only
  uint32_t* err;      // device error word
  uint32_t count;     // batched: number of requests; served: ring slots
  uint32_t served;    // 0 batched, 1 served
  uint64_t idle_ns;   // served: exit after this long without work; batched: give up (timeout) after this long
};

// Host-side planning of one request's items (the autotuner for the engine).
struct ReqPlanInput {
  const void* keys;
  uint32_t* H;
  void* out;
  uint64_t n;
  uint32_t U;
  uint32_t key_bytes;
  uint32_t skew = 0;    // dialsort_skew_class_t, 0 = unknown
  uint32_t regime = 0;  // dialsort_regime_t to force, 0 = automatic
  bool served = false;  // served mode: small items (latency); batched: larger items (throughput)
};
// False when a forced regime cannot apply to the request.
bool plan_request(const ReqPlanInput& in, Req* r);
// Bytes of scratch the request needs, 256-aligned: two-level ingestion (low
// parts, segment words), then reconstruction (desc, O, first).
size_t request_scratch_bytes(const Req& r);
// Points desc / O / first into `base` (the request's scratch region).
void place_request_scratch(Req* r, char* base);

cudaError_t launch_engine(const Launch& L, uint32_t grid, cudaStream_t stream);
uint32_t engine_grid(const DeviceInfo& dev);

}  // namespace eng
}  // namespace dialsort
