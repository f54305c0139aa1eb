// The request engine: one persistent kernel whose CTAs pull work items of many
// independent DialSort requests (zero H, histogram a key range, one chunk of
// the offset scan, one output tile of the projection) and move each request
// through its phases.  It serves two forms:
//
//   batched  thousands of instances are planned on the host, uploaded, and
//            run by ONE launch (memcpy + memset + kernel, so the whole batch
//            can be captured in a CUDA graph); the kernel exits when every
//            instance is finished.
//   served   a host scheduler (serve.cu) admits requests into a ring of
//            slots while the kernel runs; the kernel picks them up, finishes
//            them out of order, and reports completions in host-mapped memory.
//
// Work search: each CTA looks at a window of up to 256 requests (one per
// thread), takes the OLDEST request that still has unclaimed items in its
// current phase, and claims an item with one atomicAdd on the request's
// state word (see State in engine.h: the returned word names the claimed
// phase and item).  Items of a phase are claimed in order, which is what the
// decoupled look-back of the offsets phase needs (every earlier chunk is
// already held by a running CTA).  The CTA that finishes a phase's last item
// publishes the next phase (exchange after a fence), so later phases see
// every write of earlier ones.  Every wait is bounded in time (%globaltimer):
// idle CTAs sleep with back-off and leave once the whole engine has had no
// work for `idle_ns` (recording ERRBIT_TIMEOUT in batched mode, where that
// can only mean something went wrong).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "engine.h"
#include "hist_device.cuh"
#include "recon_device.cuh"

namespace dialsort {
namespace eng {

namespace {

enum Cmd : uint32_t { CMD_WORK = 0, CMD_RETRY = 1, CMD_SLEEP = 2, CMD_EXIT = 3 };

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) { return *(const volatile uint32_t*)p; }
__device__ __forceinline__ uint64_t ld_volatile_u64(const unsigned long long* p) {
  return *(const volatile unsigned long long*)p;
}

// Copy a request description into shared memory through L2 (never a stale
// L1 line: in served mode the host rewrites a slot's description by DMA).
__device__ __forceinline__ void load_req(const Req* src, Req* dst) {
  static_assert(sizeof(Req) % 8 == 0, "Req is copied in 8-byte words");
  const volatile unsigned long long* s = reinterpret_cast<const volatile unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (uint32_t i = threadIdx.x; i < sizeof(Req) / 8; i += blockDim.x) d[i] = s[i];
}

__host__ __device__ __forceinline__ uint64_t num_chunks_of(const Req& r) {
  return ((uint64_t)r.U + kChunkBins - 1) / kChunkBins;
}

// Offsets groups (look-back descriptors) of a sorting request; its offsets items take offs_per_item each.
__host__ __device__ __forceinline__ uint64_t offs_groups_of(const Req& r) {
  return r.count[PH_OFFS - 1] ? offset_groups(num_chunks_of(r)) : 0;
}

__device__ __forceinline__ uint32_t next_phase(const Req& r, uint32_t ph) {
  for (uint32_t p = ph + 1; p <= PH_EXPAND; ++p)
    if (r.count[p - 1]) return p;
  return PH_DONE;
}

// The zero phase clears, in zero_words_item-word items, the concatenation of H
// (when the histogram phase adds into it) and the look-back descriptors of
// the offsets phase.  Doing this on the device keeps admission free of
// kernels (a memset could not start while the engine occupies every SM).
__device__ void zero_words(uint32_t* p, uint64_t w0, uint64_t w1) {  // p 16-byte aligned
  uint64_t a = (w0 + 3) & ~3ull;
  if (a > w1) a = w1;
  const uint64_t b = a + ((w1 - a) & ~3ull);
  for (uint64_t w = w0 + threadIdx.x; w < a; w += blockDim.x) p[w] = 0u;
  uint4* p4 = reinterpret_cast<uint4*>(p);
  for (uint64_t q = a / 4 + threadIdx.x; q < b / 4; q += blockDim.x) p4[q] = make_uint4(0u, 0u, 0u, 0u);
  for (uint64_t w = b + threadIdx.x; w < w1; w += blockDim.x) p[w] = 0u;
}

__device__ void zero_item(const Req& r, uint32_t item) {
  const uint64_t h_words = r.zero_H ? (uint64_t)r.U : 0;
  const uint64_t d_words = r.desc ? 2ull * offs_groups_of(r) : 0;  // one descriptor per offsets group
  const uint64_t w0 = (uint64_t)item * r.zero_words_item;
  const uint64_t w1 = min(w0 + r.zero_words_item, h_words + d_words);
  if (w0 < h_words) zero_words(r.H, w0, min(w1, h_words));
  if (w1 > h_words) zero_words(reinterpret_cast<uint32_t*>(r.desc), max(w0, h_words) - h_words, w1 - h_words);
}

template <typename KeyT, int MODE>
__device__ void hist_item(const Req& r, uint32_t item, uint32_t* sh, uint32_t* err, State* st) {
  const uint64_t begin = (uint64_t)item * r.item_keys;
  const uint64_t end = min(begin + r.item_keys, r.n);
  const uint32_t warp = threadIdx.x >> 5;
  // the global sink keeps bins [0, S) in shared memory (hot keys), the rest in L2
  const uint32_t S = MODE == MODE_GLOBAL ? min(r.words_per_copy, r.U) : 0u;
  zero_smem(sh, r.replicas * r.words_per_copy);
  __syncthreads();
  const Sink<MODE> s{sh + (warp % r.replicas) * r.words_per_copy, r.H, r.U, S};
  bool bad = false;
  ingest_span<KeyT, MODE>(static_cast<const KeyT*>(r.keys) + begin, end - begin, r.U, s, warp * 32u, blockDim.x,
                          true, r.crn, bad);
  if (bad) {
    raise_error(err, ERRBIT_KEY_RANGE);
    atomicOr(&st->err, ERRBIT_KEY_RANGE);
  }
  __syncthreads();
  flush_smem<MODE>(sh, r.replicas, r.words_per_copy, MODE == MODE_GLOBAL ? S : r.U, r.H,
                   MODE != MODE_GLOBAL && r.owned != 0);
}

__device__ void run_hist(const Req& r, uint32_t item, uint32_t* sh, uint32_t* err, State* st) {
  if (r.key_bytes == 4) {
    if (r.mode == MODE_SMEM32)
      hist_item<uint32_t, MODE_SMEM32>(r, item, sh, err, st);
    else if (r.mode == MODE_SMEM16)
      hist_item<uint32_t, MODE_SMEM16>(r, item, sh, err, st);
    else
      hist_item<uint32_t, MODE_GLOBAL>(r, item, sh, err, st);
  } else {
    if (r.mode == MODE_SMEM32)
      hist_item<uint16_t, MODE_SMEM32>(r, item, sh, err, st);
    else if (r.mode == MODE_SMEM16)
      hist_item<uint16_t, MODE_SMEM16>(r, item, sh, err, st);
    else
      hist_item<uint16_t, MODE_GLOBAL>(r, item, sh, err, st);
  }
}

// ---- two-level ingestion (see kPartKeys in engine.h)

// Partition item t: the in-range keys of tile t grouped by bucket.  Counts go
// to per-(bucket, lane) shared counters (a lane's adds never collide with its
// warp neighbours'), an exclusive scan turns them into stage positions, and a
// second read of the tile (an L1/L2 hit) places each key's low part.  The
// stage is written out whole: 16 KB per tile, coalesced.
template <typename KeyT>
__device__ void part_item(const Req& r, uint32_t t, uint8_t* dyn, uint32_t* err, State* st) {
  __shared__ uint32_t wsum[kThreads / 32];
  uint32_t* cnt = reinterpret_cast<uint32_t*>(dyn);                            // [B][32]
  uint16_t* stage = reinterpret_cast<uint16_t*>(dyn + kMaxBuckets * 32 * 4);  // kPartKeys low parts
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, B = r.buckets, U = r.U;
  const uint64_t base = (uint64_t)t * kPartKeys;
  const uint32_t len = (uint32_t)(r.n - base < kPartKeys ? r.n - base : kPartKeys);
  const KeyT* keys = static_cast<const KeyT*>(r.keys) + base;
  const uint32_t E = B * 32u;
  for (uint32_t i = tid; i < E; i += kThreads) cnt[i] = 0u;
  __syncthreads();
  bool bad = false;
  for (uint32_t i = tid; i < len; i += kThreads) {
    const uint32_t k = keys[i];
    if (k < U)
      atomicAdd(&cnt[(k >> kBucketBits) * 32u + lane], 1u);
    else
      bad = true;
  }
  if (bad) {
    raise_error(err, ERRBIT_KEY_RANGE);
    atomicOr(&st->err, ERRBIT_KEY_RANGE);
  }
  __syncthreads();
  // exclusive scan over (bucket, lane): each thread sums a run of `per` counters
  const uint32_t per = (E + kThreads - 1) / kThreads, i0 = min(E, tid * per), i1 = min(E, i0 + per);
  uint32_t sum = 0;
  for (uint32_t i = i0; i < i1; ++i) sum += cnt[i];
  uint32_t inc = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= (uint32_t)d) inc += o;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t before = 0, total = 0;
  for (uint32_t w = 0; w < kThreads / 32; ++w) {
    if (w < warp) before += wsum[w];
    total += wsum[w];
  }
  uint32_t run = before + inc - sum;
  for (uint32_t i = i0; i < i1; ++i) {
    const uint32_t c = cnt[i];
    cnt[i] = run;
    run += c;
  }
  __syncthreads();
  uint32_t* seg = r.seg + (uint64_t)t * B;
  for (uint32_t b = tid; b < B; b += kThreads) {
    const uint32_t start = cnt[b * 32u], end = b + 1 < B ? cnt[(b + 1) * 32u] : total;
    seg[b] = start | ((end - start) << 16);
  }
  __syncthreads();  // every segment start read before the places move the counters
  for (uint32_t i = tid; i < len; i += kThreads) {
    const uint32_t k = keys[i];
    if (k < U) stage[atomicAdd(&cnt[(k >> kBucketBits) * 32u + lane], 1u)] = (uint16_t)(k & ((1u << kBucketBits) - 1u));
  }
  __syncthreads();
  const uint4* s4 = reinterpret_cast<const uint4*>(stage);
  uint4* d4 = reinterpret_cast<uint4*>(r.low + base);
  for (uint32_t q = tid; q < (total + 7u) / 8u; q += kThreads) d4[q] = s4[q];
}

// Histogram item of the two-level form: bucket b over tiles [t0, t1) (item =
// g * B + b).  Each warp walks the segments of its tiles; the low parts go
// through the same ingestion step as every other regime (per-lane run, warp
// CRN by the request's choice) into packed 16-bit counters, which are then
// added into H[b 2^14 ...].
__device__ void count_item(const Req& r, uint32_t item, uint32_t* sh, uint32_t* err, State* st) {
  const uint32_t B = r.buckets, tiles = r.count[PH_PART - 1], groups = r.count[PH_HIST - 1] / B;
  const uint32_t b = item % B, g = item / B, lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t t0 = (uint32_t)((uint64_t)tiles * g / groups), t1 = (uint32_t)((uint64_t)tiles * (g + 1) / groups);
  const uint32_t W = 1u << kBucketBits, Wb = min(W, r.U - b * W);
  constexpr uint32_t kWords = (1u << kBucketBits) / 2u;
  zero_smem(sh, kWords);
  __syncthreads();
  uint32_t* Hb = r.H + (uint64_t)b * W;
  const Sink<MODE_SMEM16> s{sh, Hb, Wb, 0u};
  uint32_t score = 0;
  bool bad = false;
  for (uint32_t t = t0 + warp; t < t1; t += kThreads / 32) {
    const uint32_t sg = __ldg(r.seg + (uint64_t)t * B + b);
    const uint32_t start = sg & 0xffffu, c = sg >> 16;
    const uint16_t* lo = r.low + (uint64_t)t * kPartKeys + start;
    for (uint32_t j = 0; j < c; j += 32) {  // c is warp-uniform: the warp stays together
      const bool v = j + lane < c;
      uint32_t k[1] = {v ? (uint32_t)lo[j + lane] : 0u};
      ingest<1, MODE_SMEM16>(k, v, s, Wb, bad, r.crn, score);
    }
  }
  if (bad) {  // cannot happen (low parts are below Wb); kept as a guard
    raise_error(err, ERRBIT_KEY_RANGE);
    atomicOr(&st->err, ERRBIT_KEY_RANGE);
  }
  __syncthreads();
  flush_smem<MODE_SMEM16>(sh, 1, kWords, Wb, Hb, false);
}

__global__ void __launch_bounds__(kThreads, 4) engine_kernel(Launch L) {
  extern __shared__ __align__(16) uint8_t dyn[];
  __shared__ uint64_t s_best[kThreads / 32];
  __shared__ uint32_t s_prefix[kThreads / 32];
  __shared__ uint32_t s_base, s_slot, s_ph, s_item, s_tag, s_cmd, s_exit;
  __shared__ __align__(16) Req s_req;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  uint64_t idle_since = 0;  // thread 0 only
  uint32_t backoff = 500;   // ns; doubles while idle (every thread keeps the same value)
  uint32_t round = 0;       // work searches so far (scrambles the batched-mode choice)
  unsigned long long seen_bell = 0;  // thread 0 only: the doorbell value at the last ring scan

  for (;;) {
    // ---- find the oldest request with an unclaimed item, claim one.  The
    // first barrier makes sure every thread has read last round's shared words
    // before thread 0 rewrites them.
    __syncthreads();
    ++round;
    if (tid == 0) {
      s_base = L.served ? 0u : ld_volatile_u32(&L.ctl->tail);
      s_cmd = CMD_SLEEP;
    }
    __syncthreads();
    if (!L.served && s_base >= L.count) break;  // every request is finished
    for (uint32_t wb = s_base; wb < L.count; wb += kWindow) {
      const uint32_t len = min(kWindow, L.count - wb);
      uint64_t key = ~0ull;
      bool done = true;
      if (tid < len) {
        const uint32_t slot = wb + tid;
        const unsigned long long w = ld_volatile_u64(&L.st[slot].word);
        const uint32_t ph = word_phase(w);
        done = (ph == PH_DONE);
        if (ph >= PH_ZERO && ph <= PH_EXPAND && word_next(w) < ld_volatile_u32(&L.reqs[slot].count[ph - 1]))
        {
          // An order scrambled per CTA and per round, so that hundreds of CTAs spread over the
          // requests with work instead of all contending for one request's next item (one claim per
          // round).  Batched: any request of the window.  Served: among the oldest cohort of 32
          // admissions with work (older cohorts first keeps the tail latency).
          const uint64_t mix = (uint32_t)(((tid + 1u) * 0x9E3779B1u) ^ (blockIdx.x * 0x85EBCA6Bu) ^
                                          (round * 0xC2B2AE35u)) >> 8;
          key = L.served ? (((uint64_t)(word_seq(w) >> 5) << 32) | (mix << 8) | tid) : ((mix << 8) | tid);
        }
      }
      const uint32_t notdone = __ballot_sync(0xffffffffu, !done);
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const uint64_t o = __shfl_xor_sync(0xffffffffu, key, d);
        key = o < key ? o : key;
      }
      if (lane == 0) {
        s_best[warp] = key;
        s_prefix[warp] = notdone ? (uint32_t)(__ffs(notdone) - 1) : 32u;
      }
      __syncthreads();
      if (tid == 0) {
        uint64_t best = ~0ull;
        for (uint32_t w = 0; w < kThreads / 32; ++w) best = s_best[w] < best ? s_best[w] : best;
        if (!L.served && wb == s_base) {
          uint32_t pre = 0;  // finished requests at the front of the window
          for (uint32_t w = 0; w < kThreads / 32; ++w) {
            pre += s_prefix[w];
            if (s_prefix[w] < 32u) break;
          }
          pre = min(pre, len);
          if (pre) atomicMax(&L.ctl->tail, wb + pre);
        }
        if (best != ~0ull) {
          const uint32_t slot = wb + (uint32_t)(best & 0xffu);
          // the returned word says what was claimed (see State)
          const unsigned long long old = atomicAdd(&L.st[slot].word, 1ull);
          const uint32_t ph = word_phase(old), item = word_next(old);
          s_cmd = CMD_RETRY;
          if (ph >= PH_ZERO && ph <= PH_EXPAND && item < ld_volatile_u32(&L.reqs[slot].count[ph - 1])) {
            __threadfence();  // acquire: see every write of the request's earlier phases
            s_slot = slot;
            s_ph = ph;
            s_item = item;
            s_tag = word_seq(old);
            s_cmd = CMD_WORK;
            L.ctl->last_work = globaltimer();
          }
        }
      }
      __syncthreads();
      if (s_cmd != CMD_SLEEP || L.served) break;  // served mode: the ring is one window
    }
    const uint32_t cmd = s_cmd;  // thread 0 writes it again only after the next loop-top barrier

    // ---- nothing to do: wait (bounded), or leave.  Served mode: in the first kQuickCtas CTAs thread 0
    // watches the doorbell word (one load per poll, every 200 ns) and the ring is scanned again as soon
    // as it rings, or after 64 quiet polls; the other CTAs, and batched mode, sleep with back-off.
    if (cmd == CMD_SLEEP) {
      if (tid == 0) {
        s_exit = 0;
        for (uint32_t polls = 0;; ++polls) {
          const uint64_t now = globaltimer();
          if (idle_since == 0) idle_since = now;
          const uint64_t last = *(volatile unsigned long long*)&L.ctl->last_work;
          if (L.served && L.host->stop) {
            s_exit = 1;
            break;
          }
          if (now - idle_since > L.idle_ns && (now > last ? now - last : 0) > L.idle_ns) {
            // the whole engine, not just this CTA, has had no work for idle_ns
            if (!L.served) raise_error(L.err, ERRBIT_TIMEOUT);
            s_exit = 1;
            break;
          }
          // batched mode, and served-mode CTAs outside the quick pool: back-off (they join a long
          // request within its first phases; a short one is done by the pool)
          if (!L.served || blockIdx.x >= kQuickCtas) {
            __nanosleep(backoff);
            break;
          }
          const unsigned long long b = *(volatile unsigned long long*)&L.ctl->bell;
          if (b != seen_bell) {
            seen_bell = b;
            break;
          }
          if (polls >= 64) break;
          __nanosleep(200);
        }
      }
      __syncthreads();
      if (s_exit) break;
      backoff = min(backoff * 2u, 16000u);
      continue;
    }
    if (cmd == CMD_RETRY) {  // another CTA took the item: let the claimers spread out
      __nanosleep(100 + 32 * (blockIdx.x & 7u));
      continue;
    }
    backoff = 500;
    if (tid == 0) idle_since = 0;

    // ---- do the item
    const uint32_t slot = s_slot, ph = s_ph, item = s_item;
    load_req(&L.reqs[slot], &s_req);
    __syncthreads();
    const Req& r = s_req;
    State* st = &L.st[slot];
    switch (ph) {
      case PH_ZERO:
        zero_item(r, item);
        break;
      case PH_PART:
        if (r.key_bytes == 4)
          part_item<uint32_t>(r, item, dyn, L.err, st);
        else
          part_item<uint16_t>(r, item, dyn, L.err, st);
        break;
      case PH_HIST:
        if (r.mode == MODE_TWO_LEVEL_ENG)
          count_item(r, item, reinterpret_cast<uint32_t*>(dyn), L.err, st);
        else
          run_hist(r, item, reinterpret_cast<uint32_t*>(dyn), L.err, st);
        break;
      case PH_OFFS: {  // offs_per_item consecutive groups, in order (a group looks back only at earlier ones)
        const uint64_t g1 = min((uint64_t)(item + 1) * r.offs_per_item, offs_groups_of(r));
        for (uint64_t g = (uint64_t)item * r.offs_per_item; g < g1; ++g)
          offsets_group(r.H, r.U, r.n, num_chunks_of(r), g, r.desc, r.O, r.first, L.err,
                        *reinterpret_cast<OffsetsSmem*>(dyn));
        break;
      }
      default: {  // expand_per_item output tiles (or chunk groups of a sparse H) per item
        const uint64_t units = r.by_bins ? offset_groups(num_chunks_of(r)) : (r.n + kTileKeys - 1) / kTileKeys;
        const uint64_t u1 = min((uint64_t)(item + 1) * r.expand_per_item, units);
        for (uint64_t u = (uint64_t)item * r.expand_per_item; u < u1; ++u) {
          if (r.by_bins) {
            if (r.key_bytes == 4)
              expand_bins<uint32_t>(r.H, r.U, r.n, num_chunks_of(r), r.O, static_cast<uint32_t*>(r.out), u);
            else
              expand_bins<uint16_t>(r.H, r.U, r.n, num_chunks_of(r), r.O, static_cast<uint16_t*>(r.out), u);
          } else {
            if (r.key_bytes == 4)
              expand_tile<uint32_t>(r.H, r.U, r.n, num_chunks_of(r), r.O, r.first, static_cast<uint32_t*>(r.out),
                                    r.out_aligned, u, *reinterpret_cast<ExpandSmem*>(dyn));
            else
              expand_tile<uint16_t>(r.H, r.U, r.n, num_chunks_of(r), r.O, r.first, static_cast<uint16_t*>(r.out),
                                    r.out_aligned, u, *reinterpret_cast<ExpandSmem*>(dyn));
            __syncthreads();  // the tile's shared buffers are reused by the next
          }
        }
        break;
      }
    }

    // ---- report; the last item of a phase publishes the next phase
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const uint32_t cnt = r.count[ph - 1];
      if (atomicAdd(&st->done[ph - 1], 1u) + 1u == cnt) {
        __threadfence();
        const uint32_t np = next_phase(r, ph);
        if (np == PH_DONE) {
          const uint64_t t = globaltimer();
          st->t_done = t;
          if (L.served) {
            Completion* c = &L.comp[slot];
            c->err = ld_volatile_u32(&st->err);
            c->t_done = t;
            __threadfence_system();
            c->seq_done = ld_volatile_u64(&st->seq) + 1;
          }
        }
        atomicExch(&st->word, pack_word(s_tag, np, 0));
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- host side

bool plan_request(const ReqPlanInput& in, Req* r) {
  std::memset(r, 0, sizeof(Req));
  r->keys = in.keys;
  r->H = in.H;
  r->out = in.out;
  r->n = in.n;
  r->U = in.U;
  r->key_bytes = in.key_bytes;
  // the CRN by skew class: off when equal keys rarely meet, on for runs, adaptive per warp otherwise
  // (the tuning table's CRN choices were measured on the single-instance kernels, whose CTA shapes and
  // shared-memory hot prefix differ, so they are not carried over)
  r->crn = in.skew == DIALSORT_SKEW_LOW ? CRN_OFF : in.skew == DIALSORT_SKEW_RUNS ? CRN_ON : CRN_ADAPTIVE;
  const uint64_t cap32 = kHistSmem / 4, cap16 = 2 * (kHistSmem / 4);
  const uint64_t U = in.U, n = in.n;
  const bool fits32 = align_up(U, 4) <= cap32, fits16 = align_up((U + 1) / 2, 4) <= cap16 / 2;
  const bool fits_tl = U <= ((uint64_t)kMaxBuckets << kBucketBits);
  uint32_t mode;
  switch (in.regime) {
    case DIALSORT_REGIME_AUTO:
      // (the two-level form is taken only when forced: measured inside the engine on instances of up
      // to 2^24 keys, whose H stays in L2, one L2 atomic per key was faster at every (n, U) tried)
      if (n >= 2 * U && fits32)
        mode = MODE_SMEM32;
      else if (n >= 2 * U && fits16)
        mode = MODE_SMEM16;
      else
        mode = MODE_GLOBAL;
      break;
    case DIALSORT_REGIME_SMEM32:
      if (!fits32) return false;
      mode = MODE_SMEM32;
      break;
    case DIALSORT_REGIME_SMEM16:
      if (!fits16) return false;
      mode = MODE_SMEM16;
      break;
    case DIALSORT_REGIME_GLOBAL_CRN:
    case DIALSORT_REGIME_GLOBAL:
      mode = MODE_GLOBAL;
      if (in.regime == DIALSORT_REGIME_GLOBAL) r->crn = CRN_OFF;
      break;
    case DIALSORT_REGIME_TWO_LEVEL:
      if (!fits_tl) return false;
      mode = MODE_TWO_LEVEL_ENG;
      break;
    default:
      return false;
  }
  r->mode = mode;
  r->replicas = 1;
  if (mode == MODE_TWO_LEVEL_ENG) {
    r->buckets = (uint32_t)((U + (1u << kBucketBits) - 1) >> kBucketBits);
    r->words_per_copy = (1u << kBucketBits) / 2u;
  } else if (mode == MODE_SMEM32) {
    r->words_per_copy = (uint32_t)align_up(U, 4);
    uint32_t rep = 1;
    while (rep < 8 && (uint64_t)r->words_per_copy * 4 * rep * 2 <= kHistSmem) rep *= 2;
    r->replicas = rep;
  } else if (mode == MODE_SMEM16) {
    r->words_per_copy = (uint32_t)align_up((U + 1) / 2, 4);
  } else {
    r->words_per_copy = (uint32_t)std::min<uint64_t>(align_up(U, 4), kHistSmem / 4);  // shared hot prefix
  }
  uint32_t n_hist;
  if (r->mode == MODE_TWO_LEVEL_ENG) {
    // partition tiles, then bucket x tile-group items with about 8 x 2^14 keys each or more (the
    // merge of a group's counters stays below 1/8 of its keys' work)
    const uint64_t tiles = (n + kPartKeys - 1) / kPartKeys;
    const uint64_t per_bucket = n / r->buckets;
    const uint64_t groups = std::max<uint64_t>(1, std::min<uint64_t>(tiles, per_bucket / (8ull << kBucketBits)));
    r->item_keys = kPartKeys;
    r->count[PH_PART - 1] = (uint32_t)tiles;
    n_hist = (uint32_t)(groups * r->buckets);
  } else {
    if (r->mode == MODE_GLOBAL)
      r->item_keys = 65536ull * (in.served ? 1u : kBatchedHistScale);
    else
      r->item_keys = align_up(std::max<uint64_t>(32768ull * (in.served ? 1u : kBatchedHistScale),
                                                 8ull * U * r->replicas), 8192);
    n_hist = (uint32_t)((n + r->item_keys - 1) / r->item_keys);
  }
  r->owned = (r->mode == MODE_SMEM32 && n_hist == 1) ? 1u : 0u;
  r->zero_H = r->owned ? 0u : 1u;
  r->count[PH_HIST - 1] = n_hist;
  const bool sort = in.out != nullptr && n > 0;
  const uint32_t groups = sort ? (uint32_t)offset_groups((U + kChunkBins - 1) / kChunkBins) : 0u;
  r->zero_words_item = kZeroWords * (in.served ? 1u : kBatchedZeroScale);
  r->offs_per_item = in.served ? 1u : kBatchedOffsPerItem;
  r->expand_per_item = in.served ? 1u : kBatchedExpandPerItem;
  r->count[PH_OFFS - 1] = (groups + r->offs_per_item - 1) / r->offs_per_item;
  // a sparse H (fewer keys than bins / 4): each offsets group of chunks writes its own bins' runs, so the
  // Theta(U) walk is spread over U / 8192 items instead of the few output tiles
  r->by_bins = (sort && 4 * n < U) ? 1u : 0u;
  const uint64_t units = r->by_bins ? groups : (n + kTileKeys - 1) / kTileKeys;
  r->count[PH_EXPAND - 1] = !sort ? 0u : (uint32_t)((units + r->expand_per_item - 1) / r->expand_per_item);
  const uint64_t zero_words = (r->zero_H ? U : 0) + 2ull * groups;
  r->count[PH_ZERO - 1] = (uint32_t)((zero_words + r->zero_words_item - 1) / r->zero_words_item);
  r->out_aligned = (reinterpret_cast<uintptr_t>(in.out) & 15u) == 0;
  r->first_phase = PH_DONE;
  for (uint32_t p = PH_ZERO; p <= PH_EXPAND; ++p)
    if (r->count[p - 1]) {
      r->first_phase = p;
      break;
    }
  return true;
}

// scratch of a sorting request: look-back descriptors (one per offsets group),
// chunk offsets O[0..chunks] and the first chunk of every output tile
namespace {
size_t two_level_scratch_bytes(const Req& r) {
  if (r.mode != MODE_TWO_LEVEL_ENG) return 0;
  const uint64_t tiles = r.count[PH_PART - 1];
  return align_up(tiles * kPartKeys * 2, 256) + align_up(tiles * r.buckets * 4, 256);
}
}  // namespace

size_t request_scratch_bytes(const Req& r) {
  const uint64_t groups = offs_groups_of(r), tiles = (r.n + kTileKeys - 1) / kTileKeys;
  const size_t tl = two_level_scratch_bytes(r);
  if (groups == 0) return tl;
  const uint64_t chunks = num_chunks_of(r);
  return tl + align_up(8 * groups, 256) + align_up(8 * (chunks + 1), 256) +
         align_up(4 * std::max<uint64_t>(tiles, 1), 256);
}

void place_request_scratch(Req* r, char* base) {
  r->low = nullptr;
  r->seg = nullptr;
  if (r->mode == MODE_TWO_LEVEL_ENG) {
    const uint64_t tiles = r->count[PH_PART - 1];
    r->low = reinterpret_cast<uint16_t*>(base);
    r->seg = reinterpret_cast<uint32_t*>(base + align_up(tiles * kPartKeys * 2, 256));
    base += two_level_scratch_bytes(*r);
  }
  const uint64_t groups = offs_groups_of(*r);
  if (groups == 0) {
    r->desc = nullptr;
    r->O = nullptr;
    r->first = nullptr;
    return;
  }
  const uint64_t chunks = num_chunks_of(*r);
  r->desc = reinterpret_cast<uint64_t*>(base);
  base += align_up(8 * groups, 256);
  r->O = reinterpret_cast<uint64_t*>(base);
  base += align_up(8 * (chunks + 1), 256);
  r->first = reinterpret_cast<uint32_t*>(base);
}

size_t engine_smem_bytes() { return std::max<size_t>(kHistSmem, sizeof(ExpandSmem)); }

namespace {
constexpr int kMaxDev = 64;
std::once_flag g_engine_once[kMaxDev];
uint32_t g_engine_grid[kMaxDev];
cudaError_t g_engine_err[kMaxDev];

// Kernel attributes and the resident grid, set up once per device (so later
// launches, e.g. inside a stream capture, make no attribute calls).
void engine_setup(const DeviceInfo& dev) {
  std::call_once(g_engine_once[dev.device], [&dev] {
    const size_t smem = engine_smem_bytes();
    int per_sm = 0;
    cudaError_t e = cudaFuncSetAttribute(engine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel, kThreads, smem);
    g_engine_err[dev.device] = e;
    g_engine_grid[dev.device] = (uint32_t)(dev.sms * std::max(per_sm, 1));
  });
}
}  // namespace

uint32_t engine_grid(const DeviceInfo& dev) {
  engine_setup(dev);
  return g_engine_grid[dev.device];
}

cudaError_t launch_engine(const Launch& L, uint32_t grid, cudaStream_t stream) {
  const DeviceInfo* dev = device_info();
  if (!dev) return cudaErrorNoDevice;
  engine_setup(*dev);
  if (g_engine_err[dev->device] != cudaSuccess) return g_engine_err[dev->device];
  engine_kernel<<<grid, kThreads, engine_smem_bytes(), stream>>>(L);
  return cudaGetLastError();
}

}  // namespace eng
}  // namespace dialsort

// ---------------------------------------------------------------- batched C ABI

using namespace dialsort;
using namespace dialsort::eng;

struct dialsort_batch_s {
  uint32_t count = 0;
  std::vector<uint32_t> order;  // table position -> caller's instance index (largest work first)
  std::vector<size_t> scratch_off;
  Req* h_reqs = nullptr;        // pinned
  State* h_states = nullptr;    // pinned
  size_t off_reqs = 0, off_states = 0, off_ctl = 0, off_scratch = 0, scratch_bytes = 0, total = 0;
  void* planned_ws = nullptr;   // workspace the request table was last pointed at
};

namespace {

bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

dialsort_status_t check_instance(const dialsort_instance_t& x) {
  if (x.key_bytes != 4 && x.key_bytes != 2) return DIALSORT_ERR_INVALID_ARG;
  if (x.U == 0 || x.n >= (1ull << 32)) return DIALSORT_ERR_INVALID_ARG;
  if (x.key_bytes == 2 && x.U > 65536u) return DIALSORT_ERR_INVALID_ARG;
  if (x.n > 0 && (x.keys == nullptr || !aligned_to(x.keys, x.key_bytes))) return DIALSORT_ERR_INVALID_ARG;
  if (x.H == nullptr || !aligned_to(x.H, 16)) return DIALSORT_ERR_INVALID_ARG;
  if (x.out != nullptr && !aligned_to(x.out, x.key_bytes)) return DIALSORT_ERR_INVALID_ARG;
  return DIALSORT_OK;
}

void free_batch(dialsort_batch_s* b) {
  if (!b) return;
  if (b->h_reqs) cudaFreeHost(b->h_reqs);
  if (b->h_states) cudaFreeHost(b->h_states);
  delete b;
}

}  // namespace

extern "C" {

dialsort_status_t dialsort_batch_create(const dialsort_instance_t* inst, uint32_t count, int sort,
                                        dialsort_batch_t* out) {
  if (out == nullptr || (count > 0 && inst == nullptr)) return DIALSORT_ERR_INVALID_ARG;
  *out = nullptr;
  for (uint32_t i = 0; i < count; ++i) {
    dialsort_status_t s = check_instance(inst[i]);
    if (s != DIALSORT_OK) return s;
    if (sort && inst[i].n > 0 && inst[i].out == nullptr) return DIALSORT_ERR_INVALID_ARG;
  }
  dialsort_batch_s* b = new (std::nothrow) dialsort_batch_s();
  if (!b) return DIALSORT_ERR_INVALID_ARG;
  b->count = count;
  const size_t nreq = std::max<uint32_t>(count, 1);
  if (cudaMallocHost(&b->h_reqs, sizeof(Req) * nreq) != cudaSuccess ||
      cudaMallocHost(&b->h_states, sizeof(State) * nreq) != cudaSuccess) {
    free_batch(b);
    return DIALSORT_ERR_CUDA;
  }
  // plan every instance, then order the table by estimated work (largest first)
  std::vector<Req> plans(count);
  std::vector<double> cost(count);
  for (uint32_t i = 0; i < count; ++i) {
    ReqPlanInput in{inst[i].keys, inst[i].H,  sort ? inst[i].out : nullptr, inst[i].n,
                    inst[i].U,    inst[i].key_bytes, inst[i].skew <= 3 ? inst[i].skew : 0u, inst[i].regime};
    if (!plan_request(in, &plans[i])) {
      free_batch(b);
      return DIALSORT_ERR_INVALID_ARG;
    }
    cost[i] = (double)inst[i].n * inst[i].key_bytes * (sort ? 2.0 : 1.0) + 12.0 * inst[i].U;
  }
  b->order.resize(count);
  for (uint32_t i = 0; i < count; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](uint32_t a, uint32_t c) { return cost[a] > cost[c]; });
  size_t off = 0;
  b->off_reqs = off;
  off = align_up(off + sizeof(Req) * nreq, 256);
  b->off_states = off;
  off = align_up(off + sizeof(State) * nreq, 256);
  b->off_ctl = off;
  off = align_up(off + sizeof(Ctl), 256);
  b->off_scratch = off;
  b->scratch_off.resize(count);
  size_t s = 0;
  for (uint32_t p = 0; p < count; ++p) {
    b->h_reqs[p] = plans[b->order[p]];
    b->scratch_off[p] = s;
    s += request_scratch_bytes(b->h_reqs[p]);
  }
  b->scratch_bytes = s;
  b->total = align_up(off + s, 256);
  for (uint32_t p = 0; p < count; ++p) {
    std::memset(&b->h_states[p], 0, sizeof(State));
    b->h_states[p].seq = p;
    b->h_states[p].word = pack_word(p, b->h_reqs[p].first_phase, 0);
  }
  *out = b;
  return DIALSORT_OK;
}

size_t dialsort_batch_workspace_size(dialsort_batch_t b) { return b ? b->total : 0; }

dialsort_status_t dialsort_batch_launch(dialsort_batch_t b, void* ws, size_t ws_bytes, void* stream) {
  if (b == nullptr || ws == nullptr || !aligned_to(ws, 256) || ws_bytes < b->total) return DIALSORT_ERR_WORKSPACE;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  if (b->planned_ws != ws) {
    for (uint32_t p = 0; p < b->count; ++p) place_request_scratch(&b->h_reqs[p], base + b->off_scratch + b->scratch_off[p]);
    b->planned_ws = ws;
  }
  if (b->count == 0) return DIALSORT_OK;
  cudaError_t e = cudaMemcpyAsync(base + b->off_reqs, b->h_reqs, sizeof(Req) * b->count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + b->off_states, b->h_states, sizeof(State) * b->count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + b->off_ctl, 0, sizeof(Ctl), st);
  if (e != cudaSuccess) return DIALSORT_ERR_CUDA;
  Launch L{};
  L.reqs = reinterpret_cast<const Req*>(base + b->off_reqs);
  L.st = reinterpret_cast<State*>(base + b->off_states);
  L.ctl = reinterpret_cast<Ctl*>(base + b->off_ctl);
  L.err = dev->err;
  L.count = b->count;
  L.served = 0;
  L.idle_ns = 2000000000ull;
  return launch_engine(L, engine_grid(*dev), st) == cudaSuccess ? DIALSORT_OK : DIALSORT_ERR_CUDA;
}

dialsort_status_t dialsort_batch_destroy(dialsort_batch_t b) {
  free_batch(b);
  return DIALSORT_OK;
}

dialsort_status_t dialsort_batch_describe(dialsort_batch_t b, uint32_t index, dialsort_hist_config_t* cfg,
                                          uint32_t* items) {
  if (b == nullptr || cfg == nullptr || index >= b->count) return DIALSORT_ERR_INVALID_ARG;
  uint32_t p = 0;
  while (p < b->count && b->order[p] != index) ++p;
  const Req& r = b->h_reqs[p];
  const uint32_t regime = r.mode == MODE_SMEM32           ? DIALSORT_REGIME_SMEM32
                          : r.mode == MODE_SMEM16         ? DIALSORT_REGIME_SMEM16
                          : r.mode == MODE_TWO_LEVEL_ENG  ? DIALSORT_REGIME_TWO_LEVEL
                                                          : DIALSORT_REGIME_GLOBAL_CRN;
  const uint32_t crn_cfg = r.crn == CRN_ON ? 1u : r.crn == CRN_OFF ? 2u : 3u;
  *cfg = dialsort_hist_config_t{regime, crn_cfg, 0u, kThreads, r.replicas, 1u, 0u};
  if (items) {  // zero, histogram (two-level: partition + count), offsets, expand
    items[0] = r.count[PH_ZERO - 1];
    items[1] = r.count[PH_PART - 1] + r.count[PH_HIST - 1];
    items[2] = r.count[PH_OFFS - 1];
    items[3] = r.count[PH_EXPAND - 1];
  }
  return DIALSORT_OK;
}

size_t dialsort_batched_workspace_size(const dialsort_instance_t* inst, uint32_t count, int sort) {
  dialsort_batch_t b = nullptr;
  if (dialsort_batch_create(inst, count, sort, &b) != DIALSORT_OK) return 0;
  const size_t t = b->total;
  free_batch(b);
  return t;
}

dialsort_status_t dialsort_batched(const dialsort_instance_t* inst, uint32_t count, int sort, void* ws,
                                   size_t ws_bytes, void* stream) {
  dialsort_batch_t b = nullptr;
  dialsort_status_t s = dialsort_batch_create(inst, count, sort, &b);
  if (s != DIALSORT_OK) return s;
  s = dialsort_batch_launch(b, ws, ws_bytes, stream);
  // the host tables must outlive the asynchronous copies that read them
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess && s == DIALSORT_OK)
    s = DIALSORT_ERR_CUDA;
  free_batch(b);
  return s;
}

dialsort_status_t dialsort_histogram_batched(const dialsort_instance_t* inst, uint32_t count, void* ws,
                                             size_t ws_bytes, void* stream) {
  return dialsort_batched(inst, count, 0, ws, ws_bytes, stream);
}

dialsort_status_t dialsort_sort_batched(const dialsort_instance_t* inst, uint32_t count, void* ws, size_t ws_bytes,
                                        void* stream) {
  return dialsort_batched(inst, count, 1, ws, ws_bytes, stream);
}

}  // extern "C"
