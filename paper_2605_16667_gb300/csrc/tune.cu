// The autotuner's inputs: a device probe of the keys' skew, and a table of
// measured launch choices per (n, U, key width, skew class).
//
// Skew probe.  How much the CRN pays, and how contended the counters get,
// depends on how often equal keys meet (Sec. "Conflict Resolution Network
// (CRN)", subsection "Performance consequence under skewed input").  One CTA samples 128 windows of
// 32 consecutive keys spread over the input and measures, with equality tests
// only:
//   adjacent  how many neighbours in a window are equal (sorted input and
//             runs of one key make most of them equal);
//   top       the largest multiplicity of one key in the sample, counted in a
//             shared-memory hash table whose probes compare keys for equality.
// The host turns these into a class: 3 runs, 2 skewed (a hot key), 1 low
// conflict.
//
// Tuning table.  Text lines "log2n log2U width skew regime crn replicas
// threads blocks_per_sm", written by the tuning script from launches timed on
// the device; the planner takes the entry nearest to (log2 n, log2 U) with the
// same width and skew class, and falls back to its cost model where no entry
// applies.  Loaded at first use from the file named by DIALSORT_TUNE_CACHE, or
// else from tune_table.txt next to the library; dialsort_tune_table_load
// replaces it (NULL: none, the cost model alone).
#include <dlfcn.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace dialsort {

namespace {

constexpr uint32_t kProbeThreads = 256;
constexpr uint32_t kProbeWindows = 128;
constexpr uint32_t kProbeWindow = 32;
constexpr uint32_t kProbeSlots = 8192;  // hash table slots (twice the largest sample)
constexpr uint32_t kEmpty = 0xffffffffu;

struct ProbeJob {
  const void* keys;
  uint64_t n;
  uint32_t U;
  uint32_t key_bytes;
};

// One CTA probes one key sequence: stats[0] sampled keys below U, [1] equal
// neighbour pairs, [2] neighbour pairs, [3] top multiplicity.  Windows: with
// n <= 4096 the keys themselves, 32 at a time (each key once); above, 128
// windows whose starts (n - 32) w / 127 lie at least 32 apart.
__device__ void probe_one(const ProbeJob job, uint32_t* stats, uint32_t* tkey, uint32_t* tcnt, uint32_t* red) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  for (uint32_t i = tid; i < kProbeSlots; i += kProbeThreads) {
    tkey[i] = kEmpty;
    tcnt[i] = 0;
  }
  if (tid < 4) red[tid] = 0;
  __syncthreads();
  const uint64_t n = job.n;
  const bool dense = n <= (uint64_t)kProbeWindows * kProbeWindow;
  const uint32_t windows = dense ? (uint32_t)((n + kProbeWindow - 1) / kProbeWindow) : kProbeWindows;
  for (uint32_t w = warp; w < windows; w += kProbeThreads / 32) {
    const uint64_t start = dense ? (uint64_t)w * kProbeWindow : (n - kProbeWindow) * w / (kProbeWindows - 1);
    const uint64_t i = start + lane;
    uint32_t k = kEmpty;
    if (i < n)
      k = job.key_bytes == 4 ? static_cast<const uint32_t*>(job.keys)[i]
                             : (uint32_t) static_cast<const uint16_t*>(job.keys)[i];
    const bool ok = i < n && k < job.U;
    // neighbours (lane - 1, lane), both sampled keys below U; equality only
    const uint32_t prev = __shfl_up_sync(0xffffffffu, k, 1);
    const bool prev_ok = __shfl_up_sync(0xffffffffu, ok ? 1u : 0u, 1) != 0u;
    const bool pair = lane > 0 && ok && prev_ok;
    const uint32_t eq = __ballot_sync(0xffffffffu, pair && prev == k);
    const uint32_t np = __ballot_sync(0xffffffffu, pair);
    const uint32_t ns = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) {
      atomicAdd(&red[0], (uint32_t)__popc(ns));
      atomicAdd(&red[1], (uint32_t)__popc(eq));
      atomicAdd(&red[2], (uint32_t)__popc(np));
    }
    if (ok) {  // count k: linear probing until k's slot or an empty one (at most 4096 keys, 8192 slots)
      uint32_t h = (k * 0x9E3779B1u) >> 19;
      for (uint32_t t = 0; t < kProbeSlots; ++t, h = (h + 1) & (kProbeSlots - 1)) {
        const uint32_t cur = atomicCAS(&tkey[h], kEmpty, k);
        if (cur == kEmpty || cur == k) {
          atomicAdd(&tcnt[h], 1u);
          break;
        }
      }
    }
  }
  __syncthreads();
  uint32_t top = 0;
  for (uint32_t i = tid; i < kProbeSlots; i += kProbeThreads) top = max(top, tcnt[i]);  // counts, not keys
  atomicMax(&red[3], top);
  __syncthreads();
  if (tid < 4) stats[tid] = red[tid];
}

// dynamic shared memory: the hash table's keys and counts (64 KB)
constexpr size_t kProbeSmem = 2 * kProbeSlots * sizeof(uint32_t);

__global__ void __launch_bounds__(kProbeThreads) probe_kernel(const ProbeJob job, uint32_t* stats) {
  extern __shared__ uint32_t table[];
  __shared__ uint32_t red[4];
  probe_one(job, stats, table, table + kProbeSlots, red);
}

__global__ void __launch_bounds__(kProbeThreads) probe_batch_kernel(const ProbeJob* jobs, uint32_t* stats) {
  extern __shared__ uint32_t table[];
  __shared__ uint32_t red[4];
  probe_one(jobs[blockIdx.x], stats + 4ull * blockIdx.x, table, table + kProbeSlots, red);
}

static __device__ uint32_t g_probe_stats[4];

struct TuneEntry {
  int lg_n, lg_u, width, skew;
  uint32_t regime, crn, replicas, threads, blocks_per_sm;
};

std::mutex g_tune_mu;
bool g_tune_loaded = false;
std::vector<TuneEntry> g_tune;

bool parse_table(const char* path, std::vector<TuneEntry>* out) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    TuneEntry e;
    if (std::sscanf(line, "%d %d %d %d %u %u %u %u %u", &e.lg_n, &e.lg_u, &e.width, &e.skew, &e.regime, &e.crn,
                    &e.replicas, &e.threads, &e.blocks_per_sm) == 9)
      out->push_back(e);
  }
  std::fclose(f);
  return true;
}

// The default table: tune_table.txt beside libdialsort.so.
std::string default_table_path() {
  Dl_info info;
  if (dladdr(reinterpret_cast<void*>(&parse_table), &info) == 0 || info.dli_fname == nullptr) return "";
  std::string p = info.dli_fname;
  const size_t slash = p.rfind('/');
  return (slash == std::string::npos ? std::string(".") : p.substr(0, slash)) + "/tune_table.txt";
}

void ensure_loaded() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* env = std::getenv("DIALSORT_TUNE_CACHE");
  if (env != nullptr) {
    if (*env) parse_table(env, &g_tune);
    return;  // set but empty: no table
  }
  const std::string p = default_table_path();
  if (!p.empty()) parse_table(p.c_str(), &g_tune);
}

int lg2(uint64_t x) {
  int r = 0;
  while (r < 63 && (1ull << (r + 1)) <= x) ++r;
  return r;
}

}  // namespace

bool tuned_choice(uint64_t n, uint32_t U, uint32_t key_bytes, uint32_t skew, dialsort_hist_config_t* cfg,
                  uint32_t* blocks_per_sm) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  ensure_loaded();
  const int ln = lg2(std::max<uint64_t>(n, 1)), lu = lg2(std::max<uint32_t>(U, 1));
  const TuneEntry* best = nullptr;
  int best_d = 1 << 30;
  for (const TuneEntry& e : g_tune) {
    if (e.width != (int)key_bytes || e.skew != (int)skew) continue;
    const int d = 2 * std::abs(e.lg_u - lu) + std::abs(e.lg_n - ln);  // the universe matters most
    if (d < best_d) {
      best_d = d;
      best = &e;
    }
  }
  if (!best || best_d > 6) return false;  // nothing measured near this shape
  *cfg = dialsort_hist_config_t{best->regime, best->crn, 0, best->threads, best->replicas, 0};
  *blocks_per_sm = best->blocks_per_sm;
  return true;
}

uint32_t skew_class_of(const uint32_t stats[4], uint32_t U) {
  const double samples = stats[0], adj = stats[1], pairs = stats[2], top = stats[3];
  if (samples < 64) return 0;
  if (pairs > 0 && adj >= 0.5 * pairs) return 3;  // runs: most neighbours equal
  const double uniform_top = std::max(4.0 * samples / std::max<double>(U, 1.0), samples / 64.0);
  if (top >= uniform_top) return 2;  // a hot key
  return 1;
}

}  // namespace dialsort

using namespace dialsort;

extern "C" {

dialsort_status_t dialsort_probe_skew(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U,
                                      dialsort_skew_t* out, void* stream) {
  if (out == nullptr || U == 0 || (key_bytes != 4 && key_bytes != 2) || (n > 0 && keys == nullptr))
    return DIALSORT_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(keys) % key_bytes) != 0) return DIALSORT_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (n == 0) return DIALSORT_OK;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  const void* kp;
  dialsort_status_t s = kernel_address(keys, *dev, &kp);
  if (s != DIALSORT_OK) return s;
  uint32_t* stats = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&stats), g_probe_stats) != cudaSuccess) {
    (void)cudaGetLastError();
    return DIALSORT_ERR_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (kernel_config(reinterpret_cast<const void*>(&probe_kernel), kProbeThreads, kProbeSmem, false, nullptr) !=
      cudaSuccess)
    return DIALSORT_ERR_CUDA;
  probe_kernel<<<1, kProbeThreads, kProbeSmem, st>>>(ProbeJob{kp, n, U, key_bytes}, stats);
  uint32_t h[4];
  if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(h, stats, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DIALSORT_ERR_CUDA;
  out->samples = h[0];
  out->equal_neighbours = h[1];
  out->neighbour_pairs = h[2];
  out->top_multiplicity = h[3];
  out->skew_class = skew_class_of(h, U);
  return DIALSORT_OK;
}

dialsort_status_t dialsort_probe_skew_batched(dialsort_instance_t* instances, uint32_t count, void* stream) {
  if (count == 0) return DIALSORT_OK;
  if (instances == nullptr) return DIALSORT_ERR_INVALID_ARG;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  std::vector<ProbeJob> jobs(count);
  for (uint32_t i = 0; i < count; ++i) {
    const dialsort_instance_t& in = instances[i];
    if (in.U == 0 || (in.key_bytes != 4 && in.key_bytes != 2) || (in.n > 0 && in.keys == nullptr) ||
        (reinterpret_cast<uintptr_t>(in.keys) % in.key_bytes) != 0)
      return DIALSORT_ERR_INVALID_ARG;
    const void* kp = nullptr;
    if (in.n > 0) {
      dialsort_status_t s = kernel_address(in.keys, *dev, &kp);
      if (s != DIALSORT_OK) return s;
    }
    jobs[i] = ProbeJob{kp, in.n, in.U, in.key_bytes};
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (kernel_config(reinterpret_cast<const void*>(&probe_batch_kernel), kProbeThreads, kProbeSmem, false,
                    nullptr) != cudaSuccess)
    return DIALSORT_ERR_CUDA;
  const size_t jb = align_up(sizeof(ProbeJob) * count, 256), sb = sizeof(uint32_t) * 4 * count;
  char* d = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&d), jb + sb, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return DIALSORT_ERR_CUDA;
  }
  std::vector<uint32_t> h(4ull * count);
  cudaError_t e = cudaMemcpyAsync(d, jobs.data(), sizeof(ProbeJob) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    probe_batch_kernel<<<count, kProbeThreads, kProbeSmem, st>>>(reinterpret_cast<const ProbeJob*>(d),
                                                        reinterpret_cast<uint32_t*>(d + jb));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d + jb, sb, cudaMemcpyDeviceToHost, st);
  const cudaError_t ef = cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  for (uint32_t i = 0; i < count; ++i)
    instances[i].skew = instances[i].n ? skew_class_of(&h[4ull * i], instances[i].U) : 0u;
  return DIALSORT_OK;
}

dialsort_status_t dialsort_tune_table_load(const char* path) {
  std::vector<TuneEntry> t;
  if (path != nullptr && !parse_table(path, &t)) return DIALSORT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.swap(t);
  g_tune_loaded = true;
  return DIALSORT_OK;
}

uint32_t dialsort_tune_table_size(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  ensure_loaded();
  return (uint32_t)g_tune.size();
}

}  // extern "C"
