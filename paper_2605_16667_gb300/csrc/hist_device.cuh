// Device routines of step 1 (ingestion, Eq. (1), with the warp-level CRN),
// shared by the single-instance kernel (hist.cu) and the batched/served
// engine (engine.cu).
#pragma once

#include "common.cuh"

namespace dialsort {

enum HistMode : int { MODE_SMEM32 = 0, MODE_SMEM16 = 1, MODE_GLOBAL = 2 };

template <int MODE>
struct Sink;

template <>
struct Sink<MODE_SMEM32> {
  uint32_t* sh;
  uint32_t* H;
  uint32_t U;
  uint32_t S;  // unused here
  __device__ __forceinline__ void add(uint32_t key, uint32_t c) const { atomicAdd(sh + key, c); }
};

// Two 16-bit counters per word: bin 2w in bits 0..15, bin 2w+1 in bits 16..31.
// The word holds (A + 2^16 B) mod 2^32 for true counts A (low bin) and B (high
// bin).  Every add uses a count c < 2^16, so it crosses at most one multiple of
// 2^16 in either field, and the value the atomic returns says exactly whether
// it did:
//   low carry  ((old & 0xffff) + c > 0xffff, low-bin adds only): A gained 2^16
//              that the low field cannot hold, and the high field gained 1
//              that is not B's.  Record H[2w] += 2^16, H[2w+1] -= 1.
//   word wrap  (old + delta >= 2^32): the high field passed a multiple of
//              2^16.  Record H[2w+1] += 2^16.
// At the end, H[2w] += low field and H[2w+1] += high field.  The records are
// modular adds, so H ends exact whatever the interleaving.
template <>
struct Sink<MODE_SMEM16> {
  uint32_t* sh;
  uint32_t* H;
  uint32_t U;
  uint32_t S;  // unused here
  __device__ __forceinline__ void add(uint32_t key, uint32_t c) const {
    const uint32_t hi_bin = key & 1u;
    const uint32_t delta = hi_bin ? (c << 16) : c;
    const uint32_t old = atomicAdd(sh + (key >> 1), delta);
    if (!hi_bin && (old & 0xffffu) + c > 0xffffu) {
      red_add_global(H + key, 0x10000u);
      if (key + 1 < U) red_add_global(H + key + 1, 0xffffffffu);
    }
    if ((uint64_t)old + delta > 0xffffffffull) {
      if ((key | 1u) < U) red_add_global(H + (key | 1u), 0x10000u);
    }
  }
};

template <>
// Adds go straight to the L2-resident H, except for the low bins [0, S),
// which are counted in shared memory and merged at the end: when a few keys
// are hot they are usually the small ones (Zipf), and a hot key at one L2
// address serialises every add to it.
struct Sink<MODE_GLOBAL> {
  uint32_t* sh;
  uint32_t* H;
  uint32_t U;
  uint32_t S;
  __device__ __forceinline__ void add(uint32_t key, uint32_t c) const {
    if (key < S)
      atomicAdd(sh + key, c);
    else
      red_add_global(H + key, c);
  }
};

// Optional map from a raw key to its index (Prop. "General Self-Indexing
// Principle": phi, an order-preserving map of the key domain onto [0, U)).
// phi == nullptr: the key is its own index.  A raw key x >= M, or one whose
// phi[x] is 0xffffffff (not in the domain), maps to 0xffffffff, which the
// range check then reports like any key >= U.
struct KeyMap {
  const uint32_t* phi;
  uint32_t M;
  __device__ __forceinline__ uint32_t operator()(uint32_t x) const {
    return phi == nullptr ? x : (x < M ? __ldg(phi + x) : 0xffffffffu);
  }
};

template <typename KeyT>
struct Vec;
template <>
struct Vec<uint32_t> {
  static constexpr int K = 4;
  __device__ __forceinline__ static void unpack(const uint4& q, uint32_t (&k)[4]) {
    k[0] = q.x;
    k[1] = q.y;
    k[2] = q.z;
    k[3] = q.w;
  }
};
template <>
struct Vec<uint8_t> {
  static constexpr int K = 16;
  __device__ __forceinline__ static void unpack(const uint4& q, uint32_t (&k)[16]) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      k[4 * i] = w[i] & 0xffu;
      k[4 * i + 1] = (w[i] >> 8) & 0xffu;
      k[4 * i + 2] = (w[i] >> 16) & 0xffu;
      k[4 * i + 3] = w[i] >> 24;
    }
  }
};
template <>
struct Vec<uint16_t> {
  static constexpr int K = 8;
  __device__ __forceinline__ static void unpack(const uint4& q, uint32_t (&k)[8]) {
    k[0] = q.x & 0xffffu;
    k[1] = q.x >> 16;
    k[2] = q.y & 0xffffu;
    k[3] = q.y >> 16;
    k[4] = q.z & 0xffffu;
    k[5] = q.z >> 16;
    k[6] = q.w & 0xffffu;
    k[7] = q.w >> 16;
  }
};

enum CrnMode : uint32_t { CRN_OFF = 0, CRN_ON = 1, CRN_ADAPTIVE = 2 };

// Adaptive CRN: a warp turns match.any on only while most of its lanes hold
// the same key.  The probe is cheap -- how many lanes hold the same first key
// as their left neighbour, once per vector of keys -- and feeds a moving score
// (fixed point, decay 1/8) that is the same in every lane, so the decision is
// warp-uniform.  The score settles at 64 x (equal neighbours per probe); the
// CRN is used from 16 per probe on for shared-memory sinks (4 for the L2
// sink, where a hot key serialises at one address).  Measured on this GPU, match.any costs
// about 6 clocks per distinct key among the 32 lanes, while a shared-memory
// atomic pays one pass per lane that hits the same address: merging wins only
// when few distinct keys share a warp (all equal, long sorted runs), not for
// a hot key among many (Zipf), where it was ~15x slower than plain atomics.
template <int MODE>
struct CrnThreshold {
  static constexpr uint32_t value = 64 * 16;
};
// an L2 address takes one add at a time: merge equal keys sooner
template <>
struct CrnThreshold<MODE_GLOBAL> {
  static constexpr uint32_t value = 64 * 4;
};

// Ingest the KPV keys one lane holds; bit j of vmask says whether key j is
// real.  Must be called by all 32 lanes of the warp together (the CRN step
// is a warp collective); a lane with vmask == 0 contributes nothing.  Runs of
// equal keys are merged only across consecutive real keys.
template <int KPV, int MODE>
__device__ __forceinline__ void ingest_masked(const uint32_t (&k)[KPV], uint32_t vmask, const Sink<MODE>& s,
                                              uint32_t U, bool& bad, uint32_t crn_mode, uint32_t& score) {
  // the CRN decision is taken once per vector (warp-uniform); the adaptive
  // probe looks at the first key of every lane
  bool use_crn = crn_mode == CRN_ON;
  if (crn_mode == CRN_ADAPTIVE) {
    const bool a0 = (vmask & 1u) && k[0] < U;
    const uint32_t m0 = __ballot_sync(0xffffffffu, a0);
    const uint32_t left = __shfl_up_sync(0xffffffffu, k[0], 1);
    const uint32_t eq = __ballot_sync(0xffffffffu, a0 && left == k[0]) & (m0 << 1);
    score = score - (score >> 3) + 8u * (uint32_t)__popc(eq);
    use_crn = score >= CrnThreshold<MODE>::value;
  }
  if (!use_crn) {  // equal keys are rare here: one add per key
#pragma unroll
    for (int j = 0; j < KPV; ++j) {
      const bool real = (vmask >> j) & 1u;
      const bool in_range = k[j] < U;
      bad |= real && !in_range;
      if (real && in_range) s.add(k[j], 1u);
    }
    return;
  }
  // CRN path: runs of equal keys within the lane first (the optional local
  // accumulation of a CRN lane), then equal keys across the warp's lanes
  uint32_t cnt[KPV];
  uint32_t run = 1;
#pragma unroll
  for (int j = KPV - 1; j >= 0; --j) {
    if (j < KPV - 1) run = ((vmask >> (j + 1)) & 1u) && k[j + 1] == k[j] ? run + 1 : 1;
    cnt[j] = run;
  }
#pragma unroll
  for (int j = 0; j < KPV; ++j) {
    const bool real = (vmask >> j) & 1u;
    const bool start = real && (j == 0 || !((vmask >> (j - 1)) & 1u) || k[j] != k[j - 1]);
    const bool in_range = k[j] < U;
    bad |= start && !in_range;
    const bool act = start && in_range;
    const uint32_t m = __ballot_sync(0xffffffffu, act);
    if (m == 0) continue;
    if (act) {
      const uint32_t peers = __match_any_sync(m, k[j]);
      const uint32_t total = __reduce_add_sync(peers, cnt[j]);
      if ((peers & lanemask_lt()) == 0) s.add(k[j], total);
    }
  }
}

template <int KPV, int MODE>
__device__ __forceinline__ void ingest(const uint32_t (&k)[KPV], bool valid, const Sink<MODE>& s, uint32_t U,
                                       bool& bad, uint32_t crn_mode, uint32_t& score) {
  ingest_masked<KPV, MODE>(k, valid ? ((1u << KPV) - 1u) : 0u, s, U, bad, crn_mode, score);
}

// Ingest keys[0..n) with the threads of a grid (or of one CTA): thread t of
// `stride` threads starts at vector `first + lane` of its warp and steps by
// `stride` vectors.  `first` must be warp-uniform.  The scalar head (up to the
// first 16-byte boundary) and tail are ingested by the CTA for which
// `do_scalars` is true.  Returns through `bad` whether a key >= U was seen.
template <typename KeyT, int MODE>
__device__ __forceinline__ void ingest_span(const KeyT* __restrict__ keys, uint64_t n, uint32_t U,
                                            const Sink<MODE>& s, uint64_t first, uint64_t stride, bool do_scalars,
                                            uint32_t crn_mode, bool& bad, const KeyMap map = KeyMap{nullptr, 0u}) {
  constexpr int KPV = Vec<KeyT>::K;
  constexpr int UNR = 4;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t score = 0;
  const uint64_t mis = (reinterpret_cast<uintptr_t>(keys) & 15u) / sizeof(KeyT);
  const uint64_t head = mis ? ((uint64_t)(KPV - mis) < n ? (uint64_t)(KPV - mis) : n) : 0;
  const uint64_t nvec = (n - head) / KPV;
  const uint64_t tail0 = head + nvec * KPV;
  const uint64_t nscalar = head + (n - tail0);
  const uint4* body = reinterpret_cast<const uint4*>(keys + head);

  for (uint64_t v0 = first; v0 < nvec; v0 += UNR * stride) {
    uint4 q[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const uint64_t v = v0 + u * stride + lane;
      q[u] = (v < nvec) ? ld_stream_v4(body + v) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      uint32_t k[KPV];
      Vec<KeyT>::unpack(q[u], k);
      if (map.phi != nullptr) {
#pragma unroll
        for (int j = 0; j < KPV; ++j) k[j] = map(k[j]);
      }
      ingest<KPV, MODE>(k, v0 + u * stride + lane < nvec, s, U, bad, crn_mode, score);
    }
  }
  if (nscalar != 0 && do_scalars) {
    for (uint64_t i0 = warp * 32u; i0 < nscalar; i0 += blockDim.x) {
      const uint64_t i = i0 + lane;
      uint32_t k[1] = {0u};
      if (i < nscalar) k[0] = map(keys[i < head ? i : tail0 + (i - head)]);
      ingest<1, MODE>(k, i < nscalar, s, U, bad, crn_mode, score);
    }
  }
}

// Zero `words` 32-bit words of shared memory (a multiple of 4) with the CTA.
__device__ __forceinline__ void zero_smem(uint32_t* sh, uint32_t words) {
  uint4* sh4 = reinterpret_cast<uint4*>(sh);
  for (uint32_t i = threadIdx.x; i < words / 4u; i += blockDim.x) sh4[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Merge the CTA's shared-memory sub-histograms into H.  With `store` (only
// for MODE_SMEM32, when this CTA saw every key of the instance) every bin of
// H is written, zeros included, so H needs no zeroing beforehand; otherwise
// non-zero counts are added to H.
template <int MODE>
__device__ __forceinline__ void flush_smem(const uint32_t* sh, uint32_t replicas, uint32_t words_per_copy,
                                           uint32_t U, uint32_t* H, bool store) {
  if (MODE == MODE_SMEM32 || MODE == MODE_GLOBAL) {  // (the global sink: U = its shared prefix S)
    for (uint32_t b = threadIdx.x; b < U; b += blockDim.x) {
      uint32_t sum = 0;
      for (uint32_t r = 0; r < replicas; ++r) sum += sh[r * words_per_copy + b];
      if (store)
        H[b] = sum;
      else if (sum)
        red_add_global(H + b, sum);
    }
  } else if (MODE == MODE_SMEM16) {
    const uint32_t words = (U + 1u) / 2u;
    for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) {
      uint32_t lo = 0, hi = 0;
      for (uint32_t r = 0; r < replicas; ++r) {
        const uint32_t x = sh[r * words_per_copy + w];
        lo += x & 0xffffu;
        hi += x >> 16;
      }
      if (lo) red_add_global(H + 2u * w, lo);
      if (hi && 2u * w + 1u < U) red_add_global(H + 2u * w + 1u, hi);
    }
  }
}

}  // namespace dialsort
