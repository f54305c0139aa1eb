// Step 1 of DialSort: ingestion, Eq. (1) -- H[x] += 1 for every key x --
// with concurrent equal keys merged additively before they reach memory, as
// the Conflict Resolution Network does (Eqs. (3)-(4), Definition "CRN level
// transition", Lemma "CRN additive conservation").
//
// GPU form of the CRN.  A warp's 32 lanes are the CRN's input lanes.  Each
// lane first merges runs of equal keys inside its own 16-byte vector (the
// optional local accumulation of Sec. "CRN Lane States": a lane carries
// (k_i, c_i) with c_i > 1 when the same key repeats).  Then match.any groups
// all lanes holding the same key, redux.add sums their counts, and the lowest
// lane of each group applies one add of the sum.  This merges every equal key
// of the warp in one step, where the paper's pairwise tree needs ceil(log2 k)
// levels.  Only equality between keys is evaluated; the one magnitude test,
// key < U, compares a key with the universe bound, not with another key.
//
// Privatisation regimes (where the adds land):
//   SMEM32  per-CTA 32-bit sub-histograms in shared memory (optionally several
//           copies per CTA to spread contention), merged into H at the end.
//   SMEM16  per-CTA packed sub-histograms, two 16-bit counters per word.  A
//           carry out of a counter is detected exactly from the value the
//           atomic returns and moved to H at once (see Sink<MODE_SMEM16>).
//   GLOBAL  adds go straight to H, which stays resident in L2.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace dialsort {

enum HistMode : int { MODE_SMEM32 = 0, MODE_SMEM16 = 1, MODE_GLOBAL = 2 };

template <int MODE>
struct Sink;

template <>
struct Sink<MODE_SMEM32> {
  uint32_t* sh;
  uint32_t* H;
  uint32_t U;
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
struct Sink<MODE_GLOBAL> {
  uint32_t* sh;
  uint32_t* H;
  uint32_t U;
  __device__ __forceinline__ void add(uint32_t key, uint32_t c) const { red_add_global(H + key, c); }
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

// Adaptive CRN: a warp turns match.any on only while equal keys are common.
// The probe is cheap -- how many lanes hold the same key as their left
// neighbour -- and feeds a moving score (fixed point, decay 1/8) that is the
// same in every lane, so the decision is warp-uniform.  The score settles at
// 64 x (equal neighbours per round); the CRN is used from one per round on.
// match.any costs about 30x an atomic when all 32 keys differ, and merges
// hot keys when they do not.
constexpr uint32_t kCrnScoreOn = 64;

// Ingest the KPV keys one lane holds.  Must be called by all 32 lanes of the
// warp together (the CRN step is a warp collective); lanes with valid == false
// contribute nothing.
template <int KPV, int MODE>
__device__ __forceinline__ void ingest(const uint32_t (&k)[KPV], bool valid, const Sink<MODE>& s, uint32_t U,
                                       bool& bad, uint32_t crn_mode, uint32_t& score) {
  // run length starting at each position (consecutive equal keys in the lane)
  uint32_t cnt[KPV];
  uint32_t run = 1;
#pragma unroll
  for (int j = KPV - 1; j >= 0; --j) {
    if (j < KPV - 1) run = (k[j + 1] == k[j]) ? run + 1 : 1;
    cnt[j] = run;
  }
#pragma unroll
  for (int j = 0; j < KPV; ++j) {
    const bool start = valid && (j == 0 || k[j] != k[j - 1]);
    const bool in_range = k[j] < U;
    bad |= start && !in_range;
    const bool act = start && in_range;
    if (crn_mode == CRN_OFF) {
      if (act) s.add(k[j], cnt[j]);
      continue;
    }
    const uint32_t m = __ballot_sync(0xffffffffu, act);
    if (m == 0) continue;
    bool use_crn = true;
    if (crn_mode == CRN_ADAPTIVE) {
      const uint32_t left = __shfl_up_sync(0xffffffffu, k[j], 1);
      const uint32_t eq = __ballot_sync(0xffffffffu, act && left == k[j]) & (m << 1);
      score = score - (score >> 3) + 8u * (uint32_t)__popc(eq);
      use_crn = score >= kCrnScoreOn;
    }
    if (use_crn) {
      if (act) {
        const uint32_t peers = __match_any_sync(m, k[j]);
        const uint32_t total = __reduce_add_sync(peers, cnt[j]);
        if ((peers & lanemask_lt()) == 0) s.add(k[j], total);
      }
    } else if (act) {
      s.add(k[j], cnt[j]);
    }
  }
}

template <typename KeyT, int MODE>
__global__ void __launch_bounds__(1024) hist_kernel(const KeyT* __restrict__ keys, uint64_t n, uint32_t U,
                                                    uint32_t* __restrict__ H, uint32_t* err, uint32_t replicas,
                                                    uint32_t words_per_copy, uint32_t crn_mode) {
  constexpr int KPV = Vec<KeyT>::K;
  constexpr int UNR = 4;
  extern __shared__ __align__(16) uint32_t sh[];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;

  if (MODE != MODE_GLOBAL) {
    const uint32_t quads = replicas * words_per_copy / 4u;  // words_per_copy is a multiple of 4
    uint4* sh4 = reinterpret_cast<uint4*>(sh);
    for (uint32_t i = tid; i < quads; i += blockDim.x) sh4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
  }
  const Sink<MODE> s{sh + (warp % replicas) * words_per_copy, H, U};
  bool bad = false;
  uint32_t score = 0;

  // scalar head up to the first 16-byte boundary, vector body, scalar tail
  const uint64_t mis = (reinterpret_cast<uintptr_t>(keys) & 15u) / sizeof(KeyT);
  const uint64_t head = mis ? ((uint64_t)(KPV - mis) < n ? (uint64_t)(KPV - mis) : n) : 0;
  const uint64_t nvec = (n - head) / KPV;
  const uint64_t tail0 = head + nvec * KPV;
  const uint64_t nscalar = head + (n - tail0);
  const uint4* body = reinterpret_cast<const uint4*>(keys + head);

  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x + warp * 32u; v0 < nvec; v0 += UNR * stride) {
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
      ingest<KPV, MODE>(k, v0 + u * stride + lane < nvec, s, U, bad, crn_mode, score);
    }
  }

  if (nscalar != 0 && blockIdx.x == gridDim.x - 1) {
    for (uint64_t i0 = warp * 32u; i0 < nscalar; i0 += blockDim.x) {
      const uint64_t i = i0 + lane;
      uint32_t k[1] = {0u};
      if (i < nscalar) k[0] = keys[i < head ? i : tail0 + (i - head)];
      ingest<1, MODE>(k, i < nscalar, s, U, bad, crn_mode, score);
    }
  }
  if (bad) raise_error(err, ERRBIT_KEY_RANGE);

  if (MODE == MODE_SMEM32) {
    __syncthreads();
    for (uint32_t b = tid; b < U; b += blockDim.x) {
      uint32_t sum = 0;
      for (uint32_t r = 0; r < replicas; ++r) sum += sh[r * words_per_copy + b];
      if (sum) red_add_global(H + b, sum);
    }
  } else if (MODE == MODE_SMEM16) {
    __syncthreads();
    const uint32_t words = (U + 1u) / 2u;
    for (uint32_t w = tid; w < words; w += blockDim.x) {
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

// ---------------------------------------------------------------- host side

namespace {

template <typename KeyT, int MODE>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&hist_kernel<KeyT, MODE>);
}

const void* pick_kernel(uint32_t key_bytes, int mode) {
  if (key_bytes == 4) {
    switch (mode) {
      case MODE_SMEM32: return kernel_ptr<uint32_t, MODE_SMEM32>();
      case MODE_SMEM16: return kernel_ptr<uint32_t, MODE_SMEM16>();
      default: return kernel_ptr<uint32_t, MODE_GLOBAL>();
    }
  }
  switch (mode) {
    case MODE_SMEM32: return kernel_ptr<uint16_t, MODE_SMEM32>();
    case MODE_SMEM16: return kernel_ptr<uint16_t, MODE_SMEM16>();
    default: return kernel_ptr<uint16_t, MODE_GLOBAL>();
  }
}

int mode_of(uint32_t regime) {
  switch (regime) {
    case DIALSORT_REGIME_SMEM32: return MODE_SMEM32;
    case DIALSORT_REGIME_SMEM16: return MODE_SMEM16;
    default: return MODE_GLOBAL;
  }
}

}  // namespace

cudaError_t launch_histogram(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H,
                             const HistPlan& plan, uint32_t* err, cudaStream_t stream) {
  const void* fn = pick_kernel(key_bytes, mode_of(plan.regime));
  if (plan.smem_bytes > 48u * 1024u) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem_bytes);
    if (e != cudaSuccess) return e;
  }
  uint32_t replicas = plan.replicas, wpc = plan.words_per_copy, crn = plan.crn;
  void* args[] = {const_cast<void**>(&keys), &n, &U, &H, &err, &replicas, &wpc, &crn};
  return cudaLaunchKernel(fn, dim3(plan.blocks), dim3(plan.threads), args, plan.smem_bytes, stream);
}

// ---------------------------------------------------------------- autotuner

// Cost model (per CTA-resident SM, from the kernels above):
//   * shared-memory regimes pay a merge of words_per_copy * replicas words per
//     CTA at the end, i.e. blocks * U global adds in total; they win when that
//     is small next to n.
//   * the global regime pays one L2 atomic per key run (per distinct key of a
//     warp with the CRN on); with H resident in L2 it needs no merge at all.
dialsort_status_t plan_histogram(uint64_t n, uint32_t U, uint32_t key_bytes, uint32_t skew_hint,
                                 const dialsort_hist_config_t* cfg, const DeviceInfo& dev, HistPlan* plan) {
  dialsort_hist_config_t c = cfg ? *cfg : dialsort_hist_config_t{0, 0, 0, 0, 0, 0};
  HistPlan p;
  const size_t smem_cap = dev.smem_optin ? dev.smem_optin : 227u * 1024u;
  const uint32_t sms = dev.sms > 0 ? (uint32_t)dev.sms : 152u;

  if (c.threads != 0 && c.threads != 256 && c.threads != 512 && c.threads != 1024) return DIALSORT_ERR_INVALID_ARG;
  if (c.crn > 3) return DIALSORT_ERR_INVALID_ARG;

  uint32_t regime = c.regime;
  if (regime == DIALSORT_REGIME_CLUSTER) return DIALSORT_ERR_INVALID_ARG;  // not built in this library version
  if (regime > DIALSORT_REGIME_GLOBAL) return DIALSORT_ERR_INVALID_ARG;
  const uint64_t u32_words = align_up(U, 4);
  const uint64_t u16_words = align_up((U + 1ull) / 2ull, 4);
  if (regime == DIALSORT_REGIME_AUTO) {
    // merge cost of a smem regime with one CTA per SM, against the keys' own cost
    const bool merge_cheap = (uint64_t)sms * U * 8ull <= n;
    if (merge_cheap && u32_words * 4 <= smem_cap)
      regime = DIALSORT_REGIME_SMEM32;
    else if (merge_cheap && u16_words * 4 <= smem_cap)
      regime = DIALSORT_REGIME_SMEM16;
    else
      regime = skew_hint == 1 ? DIALSORT_REGIME_GLOBAL : DIALSORT_REGIME_GLOBAL_CRN;
  }
  p.regime = regime;
  // config: 0 auto, 1 on, 2 off, 3 adaptive.  Auto: adaptive, except off for the plain GLOBAL
  // regime or when the caller says keys rarely repeat.
  if (c.crn == 1)
    p.crn = CRN_ON;
  else if (c.crn == 2)
    p.crn = CRN_OFF;
  else if (c.crn == 3)
    p.crn = CRN_ADAPTIVE;
  else
    p.crn = (regime == DIALSORT_REGIME_GLOBAL || skew_hint == 1) ? CRN_OFF : CRN_ADAPTIVE;
  p.threads = c.threads ? c.threads : 1024;

  if (regime == DIALSORT_REGIME_SMEM32 || regime == DIALSORT_REGIME_SMEM16) {
    p.words_per_copy = (uint32_t)(regime == DIALSORT_REGIME_SMEM32 ? u32_words : u16_words);
    const size_t copy_bytes = (size_t)p.words_per_copy * 4;
    if (copy_bytes > smem_cap) return DIALSORT_ERR_INVALID_ARG;
    uint32_t warps = p.threads / 32;
    uint32_t rep = c.replicas;
    if (rep == 0) {
      // more copies for small universes: spreads equal-key contention across banks and copies
      rep = 1;
      while (rep * 2 <= warps && copy_bytes * rep * 2 <= 64u * 1024u) rep *= 2;
    }
    if (rep > warps || copy_bytes * rep > smem_cap) return DIALSORT_ERR_INVALID_ARG;
    p.replicas = rep;
    p.smem_bytes = copy_bytes * rep;
    // resident CTAs per SM by shared memory and threads (2048 threads per SM)
    uint32_t per_sm = std::max<uint32_t>(1u, std::min<uint32_t>((uint32_t)(228u * 1024u / (p.smem_bytes + 1024u)),
                                                                  2048u / p.threads));
    uint32_t blocks = sms * per_sm;
    // keep the end-of-kernel merge below about 1/8 of the keys
    uint64_t max_blocks = std::max<uint64_t>(1, n / (8ull * U * rep));
    if (blocks > max_blocks) blocks = (uint32_t)max_blocks;
    p.blocks = c.blocks ? c.blocks : blocks;
  } else {
    p.replicas = 1;
    p.words_per_copy = 0;
    p.smem_bytes = 0;
    uint64_t vec_per_thread = 16;  // aim for a handful of loop trips per thread
    uint64_t want = (n / (16 / key_bytes) + (uint64_t)p.threads * vec_per_thread - 1) / ((uint64_t)p.threads * vec_per_thread);
    uint64_t blocks = std::min<uint64_t>((uint64_t)sms * (2048u / p.threads), std::max<uint64_t>(1, want));
    p.blocks = c.blocks ? c.blocks : (uint32_t)blocks;
  }
  p.cluster = 1;
  *plan = p;
  return DIALSORT_OK;
}

}  // namespace dialsort
