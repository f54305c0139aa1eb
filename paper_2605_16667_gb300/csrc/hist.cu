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

#include "hist_device.cuh"
#include "internal.h"

namespace dialsort {

template <typename KeyT, int MODE>
__global__ void __launch_bounds__(1024) hist_kernel(const KeyT* __restrict__ keys, uint64_t n, uint32_t U,
                                                    uint32_t* __restrict__ H, uint32_t* err, uint32_t replicas,
                                                    uint32_t words_per_copy, uint32_t crn_mode, KeyMap map) {
  extern __shared__ __align__(16) uint32_t sh[];
  const uint32_t warp = threadIdx.x >> 5;
  // the global sink keeps bins [0, S) in shared memory (S = words_per_copy, capped at U)
  const uint32_t S = MODE == MODE_GLOBAL ? min(words_per_copy, U) : 0u;
  zero_smem(sh, replicas * words_per_copy);
  __syncthreads();
  const Sink<MODE> s{sh + (warp % replicas) * words_per_copy, H, U, S};
  bool bad = false;
  ingest_span<KeyT, MODE>(keys, n, U, s, (uint64_t)blockIdx.x * blockDim.x + warp * 32u,
                          (uint64_t)gridDim.x * blockDim.x, blockIdx.x == gridDim.x - 1, crn_mode, bad, map);
  if (bad) raise_error(err, ERRBIT_KEY_RANGE);
  __syncthreads();
  flush_smem<MODE>(sh, replicas, words_per_copy, MODE == MODE_GLOBAL ? S : U, H, false);
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
  if (key_bytes == 2) {
    switch (mode) {
      case MODE_SMEM32: return kernel_ptr<uint16_t, MODE_SMEM32>();
      case MODE_SMEM16: return kernel_ptr<uint16_t, MODE_SMEM16>();
      default: return kernel_ptr<uint16_t, MODE_GLOBAL>();
    }
  }
  switch (mode) {
    case MODE_SMEM32: return kernel_ptr<uint8_t, MODE_SMEM32>();
    case MODE_SMEM16: return kernel_ptr<uint8_t, MODE_SMEM16>();
    default: return kernel_ptr<uint8_t, MODE_GLOBAL>();
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
                             const HistPlan& plan, uint32_t* err, cudaStream_t stream, const uint32_t* phi,
                             uint32_t M) {
  const void* fn = pick_kernel(key_bytes, mode_of(plan.regime));
  if (plan.smem_bytes > 48u * 1024u) {
    cudaError_t e = kernel_config(fn, (int)plan.threads, plan.smem_bytes, false, nullptr);
    if (e != cudaSuccess) return e;
  }
  uint32_t replicas = plan.replicas, wpc = plan.words_per_copy, crn = plan.crn;
  KeyMap map{phi, M};
  void* args[] = {const_cast<void**>(&keys), &n, &U, &H, &err, &replicas, &wpc, &crn, &map};
  return cudaLaunchKernel(fn, dim3(plan.blocks), dim3(plan.threads), args, plan.smem_bytes, stream);
}

// ---------------------------------------------------------------- autotuner

// Cost model (per CTA-resident SM, from the kernels above):
//   * shared-memory regimes pay a merge of words_per_copy * replicas words per
//     CTA at the end, i.e. blocks * U global adds in total; they win when that
//     is small next to n.
//   * the global regime pays one L2 atomic per key run (per distinct key of a
//     warp with the CRN on); with H resident in L2 it needs no merge at all.
constexpr uint32_t kGlobalHotBins = 8192;  // 32 KB: two 1024-thread CTAs per SM still fit

namespace {
dialsort_status_t plan_core(uint64_t n, uint32_t U, uint32_t key_bytes, uint32_t skew_hint,
                            const dialsort_hist_config_t& c, const DeviceInfo& dev, HistPlan* plan);
}

dialsort_status_t plan_histogram(uint64_t n, uint32_t U, uint32_t key_bytes, uint32_t skew_hint,
                                 const dialsort_hist_config_t* cfg, const DeviceInfo& dev, HistPlan* plan,
                                 bool use_table) {
  dialsort_hist_config_t c = cfg ? *cfg : dialsort_hist_config_t{};
  if (skew_hint > 3) return DIALSORT_ERR_INVALID_ARG;
  const bool all_auto = c.regime == 0 && c.crn == 0 && c.blocks == 0 && c.threads == 0 && c.replicas == 0 &&
                        c.cluster == 0;
  dialsort_hist_config_t t;
  uint32_t per_sm = 0;
  // (an entry with regime 0 says the cost model is right at that shape: the untuned path below)
  if (use_table && all_auto && tuned_choice(n, U, key_bytes, skew_hint, &t, &per_sm) && t.regime != 0) {
    // the measured entry; an entry that does not apply to this shape falls back to the cost model
    const uint32_t sms = dev.sms > 0 ? (uint32_t)dev.sms : 152u;
    if (per_sm) t.blocks = sms * per_sm;
    if (t.regime == DIALSORT_REGIME_SMEM32 || t.regime == DIALSORT_REGIME_SMEM16) {
      // never more CTAs than keep the end-of-kernel merge below about 1/8 of the keys
      const uint64_t rep = t.replicas ? t.replicas : 1;
      const uint64_t max_blocks = std::max<uint64_t>(1, n / (8ull * U * rep));
      if (t.blocks > max_blocks) t.blocks = (uint32_t)max_blocks;
    }
    HistPlan p;
    if (plan_core(n, U, key_bytes, skew_hint, t, dev, &p) == DIALSORT_OK) {
      p.tuned = true;
      *plan = p;
      return DIALSORT_OK;
    }
  }
  return plan_core(n, U, key_bytes, skew_hint, c, dev, plan);
}

namespace {
dialsort_status_t plan_core(uint64_t n, uint32_t U, uint32_t key_bytes, uint32_t skew_hint,
                            const dialsort_hist_config_t& c, const DeviceInfo& dev, HistPlan* plan) {
  HistPlan p;
  const size_t smem_cap = dev.smem_optin ? dev.smem_optin : 227u * 1024u;
  const uint32_t sms = dev.sms > 0 ? (uint32_t)dev.sms : 152u;

  if (c.threads != 0 && c.threads != 256 && c.threads != 512 && c.threads != 1024) return DIALSORT_ERR_INVALID_ARG;
  if (c.crn > 3) return DIALSORT_ERR_INVALID_ARG;

  uint32_t regime = c.regime;
  if (regime == DIALSORT_REGIME_CLUSTER) return DIALSORT_ERR_INVALID_ARG;  // not built in this library version
  if (regime > DIALSORT_REGIME_TWO_LEVEL) return DIALSORT_ERR_INVALID_ARG;
  if (regime == DIALSORT_REGIME_TWO_LEVEL) {  // resolved by the caller (needs workspace); fill the CRN choice
    p.regime = regime;
    p.crn = c.crn == 1 ? CRN_ON : c.crn == 2 ? CRN_OFF : CRN_ADAPTIVE;
    p.threads = 256;
    p.blocks = 0;
    *plan = p;
    return DIALSORT_OK;
  }
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
      regime = skew_hint == DIALSORT_SKEW_LOW ? DIALSORT_REGIME_GLOBAL : DIALSORT_REGIME_GLOBAL_CRN;
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
    p.crn = (regime == DIALSORT_REGIME_GLOBAL || skew_hint == DIALSORT_SKEW_LOW) ? CRN_OFF : CRN_ADAPTIVE;
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
    // the low bins in shared memory (hot keys), the rest in L2
    p.replicas = 1;
    p.words_per_copy = (uint32_t)std::min<uint64_t>(align_up(U, 4), kGlobalHotBins);
    p.smem_bytes = (size_t)p.words_per_copy * 4;
    uint64_t vec_per_thread = 16;  // aim for a handful of loop trips per thread
    uint64_t want = (n / (16 / key_bytes) + (uint64_t)p.threads * vec_per_thread - 1) / ((uint64_t)p.threads * vec_per_thread);
    uint64_t blocks = std::min<uint64_t>((uint64_t)sms * (2048u / p.threads), std::max<uint64_t>(1, want));
    p.blocks = c.blocks ? c.blocks : (uint32_t)blocks;
  }
  p.cluster = 1;
  *plan = p;
  return DIALSORT_OK;
}
}  // namespace

}  // namespace dialsort
