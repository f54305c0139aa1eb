// Shared definitions of the request engine (engine.cu) and the server (serve.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace dialsort {
namespace eng {

constexpr uint32_t kThreads = 256;       // worker CTA size (the step-2 routines assume 256)
constexpr uint32_t kZeroWords = 16384;   // H words zeroed per zero item (64 KB)
constexpr uint32_t kWindow = 256;        // requests examined per work search (one per thread)
constexpr uint32_t kHistSmem = 48 * 1024;  // dynamic shared memory for shared-memory histogram items

enum Phase : uint32_t { PH_FREE = 0, PH_ZERO = 1, PH_HIST = 2, PH_OFFS = 3, PH_EXPAND = 4, PH_DONE = 5 };

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
  uint32_t owned;     // the single histogram item stores every bin of H (no zero phase)
  uint32_t out_aligned;
  uint32_t count[4];  // items of the zero, histogram, offsets and expand phases
  uint32_t first_phase;
  uint32_t pad;
};

// Mutable progress of one request (device memory).  `phase` is published last.
// A claim word holds (low 32 bits of seq) << 32 | items handed out: in served
// mode slots are reused, and a CTA claims with a compare-and-swap that fails
// if the slot now holds a different request.
struct State {
  unsigned long long claim[4];  // per phase: zero, histogram, offsets, expand
  unsigned long long seq;       // admission order (smaller = older = served first)
  unsigned long long t_done;    // %globaltimer when the request finished
  uint32_t phase;
  uint32_t done[4];             // items finished, per phase
  uint32_t err;                 // error bits of this request
  uint32_t pad[2];
};

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
  uint32_t tail;   // batched mode: every request below tail is finished
  uint32_t pad[63];
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
};
void plan_request(const ReqPlanInput& in, Req* r);
// Bytes of reconstruction scratch (desc, O, first) the request needs, 256-aligned.
size_t request_scratch_bytes(const Req& r);
// Points desc / O / first into `base` (the request's scratch region).
void place_request_scratch(Req* r, char* base);

cudaError_t launch_engine(const Launch& L, uint32_t grid, cudaStream_t stream);
uint32_t engine_grid(const DeviceInfo& dev);

}  // namespace eng
}  // namespace dialsort
