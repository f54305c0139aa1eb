// extern "C" entry points of libdialsort.so (declared in include/dialsort.h):
// host-side argument checks, per-device state, and the launch sequences of the
// two steps of DialSort.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "internal.h"

namespace dialsort {

// The per-device error word.  Kernels receive its device address as an
// argument; host code never dereferences the symbol.
static __device__ uint32_t g_error_word;

namespace {

constexpr int kMaxDevices = 64;
DeviceInfo g_dev[kMaxDevices];
std::once_flag g_once[kMaxDevices];

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

const DeviceInfo* device_info() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::call_once(g_once[dev], [dev] {
    DeviceInfo d;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return;
    d.sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return;
    d.smem_optin = (size_t)v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) return;
    d.pageable = v != 0;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return;
    d.err = static_cast<uint32_t*>(p);
    d.device = dev;
    g_dev[dev] = d;
  });
  return g_dev[dev].device == dev ? &g_dev[dev] : nullptr;
}

namespace {
std::mutex g_cfg_mu;
std::map<std::tuple<int, const void*, int>, bool> g_cfg_done;                    // (device, kernel, carve-out)
std::map<std::tuple<int, const void*, int, size_t>, int> g_cfg_occupancy;       // (device, kernel, threads, smem)
}  // namespace

cudaError_t kernel_config(const void* fn, int threads, size_t dyn_smem, bool carveout_max, int* per_sm) {
  const DeviceInfo* dev = device_info();
  if (!dev) return cudaErrorNoDevice;
  std::lock_guard<std::mutex> lock(g_cfg_mu);
  const auto key = std::make_tuple(dev->device, fn, carveout_max ? 1 : 0);
  if (!g_cfg_done.count(key)) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    // the opt-in limit covers static and dynamic shared memory together
    const size_t room = dev->smem_optin > fa.sharedSizeBytes ? dev->smem_optin - fa.sharedSizeBytes : 0;
    if (room > 48u * 1024u) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room);
    if (e == cudaSuccess && carveout_max)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    g_cfg_done[key] = true;
  }
  if (per_sm) {
    const auto okey = std::make_tuple(dev->device, fn, threads, dyn_smem);
    auto it = g_cfg_occupancy.find(okey);
    if (it == g_cfg_occupancy.end()) {
      int v = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, threads, dyn_smem);
      if (e != cudaSuccess) return e;
      it = g_cfg_occupancy.emplace(okey, v).first;
    }
    *per_sm = it->second;
  }
  return cudaSuccess;
}

dialsort_status_t kernel_address(const void* p, const DeviceInfo& dev, const void** q, bool* in_host) {
  *q = p;
  if (in_host) *in_host = false;
  if (p == nullptr) return DIALSORT_OK;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();  // not a CUDA error of the stream: clear it
    return DIALSORT_ERR_INVALID_ARG;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
      return a.device == dev.device ? DIALSORT_OK : DIALSORT_ERR_INVALID_ARG;
    case cudaMemoryTypeManaged:
      return DIALSORT_OK;
    case cudaMemoryTypeHost:  // page-locked: the mapped address (equal to p under unified addressing)
      if (a.devicePointer == nullptr) return DIALSORT_ERR_INVALID_ARG;
      *q = a.devicePointer;
      if (in_host) *in_host = true;
      return DIALSORT_OK;
    default:  // pageable host memory
      if (in_host) *in_host = true;
      return dev.pageable ? DIALSORT_OK : DIALSORT_ERR_INVALID_ARG;
  }
}

}  // namespace dialsort

using namespace dialsort;

namespace {

dialsort_status_t check_keys(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U) {
  if (key_bytes != 4 && key_bytes != 2) return DIALSORT_ERR_INVALID_ARG;
  if (U == 0 || n >= (1ull << 32)) return DIALSORT_ERR_INVALID_ARG;
  if (key_bytes == 2 && U > 65536u) return DIALSORT_ERR_INVALID_ARG;
  if (n > 0 && (keys == nullptr || !aligned(keys, key_bytes))) return DIALSORT_ERR_INVALID_ARG;
  return DIALSORT_OK;
}

size_t hist_ws_bytes(uint64_t n, uint32_t U, uint32_t key_bytes) {
  if (key_bytes != 4 || n < (1u << 20)) return 0;
  if (hier_shape_fits(n, U, key_bytes)) return hier_layout(n, U).total;
  return two_level_layout(n, U).total;
}

dialsort_status_t histogram_impl(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H,
                                 const dialsort_hist_config_t* cfg, void* ws, size_t ws_bytes, cudaStream_t st,
                                 bool accumulate = false) {
  dialsort_status_t s = check_keys(keys, key_bytes, n, U);
  if (s != DIALSORT_OK) return s;
  if (H == nullptr || !aligned(H, 16)) return DIALSORT_ERR_INVALID_ARG;
  if (ws != nullptr && !aligned(ws, 256)) return DIALSORT_ERR_WORKSPACE;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  const void* kp;
  const void* hp;
  bool keys_in_host = false;
  if ((s = kernel_address(n ? keys : nullptr, *dev, &kp, &keys_in_host)) != DIALSORT_OK) return s;
  if ((s = kernel_address(H, *dev, &hp)) != DIALSORT_OK) return s;
  keys = kp;
  H = static_cast<uint32_t*>(const_cast<void*>(hp));
  HistPlan plan;
  const uint32_t skew = cfg ? cfg->skew : 0u;
  s = plan_histogram(n, U, key_bytes, skew, cfg, *dev, &plan);
  if (s != DIALSORT_OK) return s;
  // large universes: the two-level regime when it applies and the workspace holds its scratch: where
  // the tuning table names it, or (no table entry) for every shape where the cost model's L2 plan would
  // run.  A measured single-pass entry stands.
  const bool forced = plan.regime == DIALSORT_REGIME_TWO_LEVEL && !plan.tuned;
  const bool auto_large = (cfg == nullptr || cfg->regime == DIALSORT_REGIME_AUTO) &&
                          (plan.tuned ? plan.regime == DIALSORT_REGIME_TWO_LEVEL
                                      : (plan.regime == DIALSORT_REGIME_GLOBAL_CRN ||
                                         plan.regime == DIALSORT_REGIME_GLOBAL));
  // the two-level passes read device memory (the U > 2^21 form moves keys with bulk (TMA) copies)
  if ((forced || auto_large) && !keys_in_host && hier_fits(n, U, key_bytes, keys)) {
    const HierLayout T = hier_layout(n, U);
    if (ws != nullptr && ws_bytes >= T.total)
      return from_cuda(launch_hier(static_cast<const uint32_t*>(keys), n, U, H, ws, T, *dev, dev->err, st, accumulate));
    if (forced) return DIALSORT_ERR_WORKSPACE;
  } else if ((forced || auto_large) && !keys_in_host && two_level_fits(n, U, key_bytes, keys)) {
    const TwoLevelLayout T = two_level_layout(n, U);
    if (ws != nullptr && ws_bytes >= T.total)
      return from_cuda(launch_two_level(static_cast<const uint32_t*>(keys), n, U, H, ws, T, plan.crn, *dev,
                                        dev->err, st, accumulate));
    if (forced) return DIALSORT_ERR_WORKSPACE;
  } else if (forced) {
    return DIALSORT_ERR_INVALID_ARG;
  }
  // a tuned two-level entry without its workspace: the cost model's single-pass plan
  if (plan.regime == DIALSORT_REGIME_TWO_LEVEL &&
      (s = plan_histogram(n, U, key_bytes, skew, cfg, *dev, &plan, false)) != DIALSORT_OK)
    return s;
  if (plan.regime == DIALSORT_REGIME_TWO_LEVEL) return DIALSORT_ERR_INVALID_ARG;
  // Eq. (1) starts from H = 0: the Theta(U) initialisation (skipped when accumulating into H)
  cudaError_t e = accumulate ? cudaSuccess : cudaMemsetAsync(H, 0, (size_t)U * 4, st);
  if (e == cudaSuccess && n > 0) e = launch_histogram(keys, key_bytes, n, U, H, plan, dev->err, st);
  return from_cuda(e);
}

dialsort_status_t reconstruct_impl(const uint32_t* H, uint32_t U, void* out, uint32_t out_bytes, uint64_t n,
                                   void* ws, size_t ws_bytes, cudaStream_t st) {
  if (U == 0 || n >= (1ull << 32) || H == nullptr || !aligned(H, 16)) return DIALSORT_ERR_INVALID_ARG;
  if (out_bytes == 2 && U > 65536u) return DIALSORT_ERR_INVALID_ARG;
  if (n > 0 && (out == nullptr || !aligned(out, out_bytes))) return DIALSORT_ERR_INVALID_ARG;
  const ReconLayout L = recon_layout(U, n);
  if (ws == nullptr || !aligned(ws, 256) || ws_bytes < L.total) return DIALSORT_ERR_WORKSPACE;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  const void* hp;
  const void* op;
  dialsort_status_t s = kernel_address(H, *dev, &hp);
  if (s == DIALSORT_OK) s = kernel_address(n ? out : nullptr, *dev, &op);
  if (s != DIALSORT_OK) return s;
  H = static_cast<const uint32_t*>(hp);
  if (n) out = const_cast<void*>(op);
  return from_cuda(launch_projection(H, U, n, out, out_bytes, ws, L, *dev, dev->err, st));
}

size_t sort_h_bytes(uint32_t U) { return align_up((size_t)U * 4, 256); }

// sort workspace: H | reconstruction scratch | ingestion scratch
dialsort_status_t sort_impl(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, void* out, void* ws,
                            size_t ws_bytes, cudaStream_t st, const dialsort_hist_config_t* cfg = nullptr,
                            cudaEvent_t* marks = nullptr, bool* fused = nullptr) {
  if (fused) *fused = false;
  dialsort_status_t s = check_keys(keys, key_bytes, n, U);
  if (s != DIALSORT_OK) return s;
  if (n > 0 && (out == nullptr || !aligned(out, key_bytes))) return DIALSORT_ERR_INVALID_ARG;
  const size_t hb = sort_h_bytes(U), rb = recon_layout(U, n).total, ib = hist_ws_bytes(n, U, key_bytes);
  if (ws == nullptr || !aligned(ws, 256) || ws_bytes < hb + rb + ib) return DIALSORT_ERR_WORKSPACE;
  char* base = static_cast<char*>(ws);
  uint32_t* H = reinterpret_cast<uint32_t*>(base);
  const bool auto_cfg = cfg == nullptr || (cfg->regime == 0 && cfg->crn == 0 && cfg->blocks == 0 &&
                                            cfg->threads == 0 && cfg->replicas == 0 && cfg->cluster == 0);
  if (auto_cfg && small_sort_fits(n, U, key_bytes)) {
    // a small input: the whole sort in one launch
    const DeviceInfo* dev = device_info();
    if (!dev) return DIALSORT_ERR_CUDA;
    const void *kp, *op;
    if ((s = kernel_address(keys, *dev, &kp)) != DIALSORT_OK) return s;
    if ((s = kernel_address(out, *dev, &op)) != DIALSORT_OK) return s;
    return from_cuda(launch_small_sort(kp, key_bytes, n, U, H, const_cast<void*>(op), base + hb, recon_layout(U, n),
                                       *dev, dev->err, st));
  }
  if (key_bytes == 4 && (cfg == nullptr || cfg->regime == DIALSORT_REGIME_AUTO) && ib != 0) {
    // the two-level form, where the planner takes it: counting fused with the projection
    const DeviceInfo* dev = device_info();
    if (!dev) return DIALSORT_ERR_CUDA;
    const void *kp, *op;
    bool keys_in_host = false;
    if ((s = kernel_address(keys, *dev, &kp, &keys_in_host)) != DIALSORT_OK) return s;
    if ((s = kernel_address(out, *dev, &op)) != DIALSORT_OK) return s;
    HistPlan plan;
    if ((s = plan_histogram(n, U, key_bytes, cfg ? cfg->skew : 0u, cfg, *dev, &plan)) != DIALSORT_OK) return s;
    const bool two_level = plan.tuned ? plan.regime == DIALSORT_REGIME_TWO_LEVEL
                                      : (plan.regime == DIALSORT_REGIME_GLOBAL_CRN || plan.regime == DIALSORT_REGIME_GLOBAL);
    if (two_level && !keys_in_host && hier_fits(n, U, key_bytes, kp) && ib >= hier_layout(n, U).total) {
      if (fused) *fused = true;
      return from_cuda(launch_hier_sort(static_cast<const uint32_t*>(kp), n, U, H,
                                        static_cast<uint32_t*>(const_cast<void*>(op)), base + hb + rb,
                                        hier_layout(n, U), *dev, dev->err, st, marks));
    }
  }
  s = histogram_impl(keys, key_bytes, n, U, H, cfg, ib ? base + hb + rb : nullptr, ib, st);
  if (s != DIALSORT_OK) return s;
  return reconstruct_impl(H, U, out, key_bytes, n, base + hb, rb, st);
}

// Prop. "General Self-Indexing Principle": index = phi(key), counted by Eq. (1) over [0, U), then
// Eq. (2) emits inv(index) for every index in order.  Single-pass ingestion regimes only (the
// two-level path moves raw keys, not indices).
dialsort_status_t sort_mapped_impl(const void* keys, uint32_t key_bytes, uint64_t n, const uint32_t* phi,
                                   uint32_t M, const void* inv, uint32_t U, void* out, void* ws, size_t ws_bytes,
                                   cudaStream_t st) {
  if (key_bytes != 1 && key_bytes != 2 && key_bytes != 4) return DIALSORT_ERR_INVALID_ARG;
  if (U == 0 || n >= (1ull << 32)) return DIALSORT_ERR_INVALID_ARG;
  if (phi != nullptr && (M == 0 || (key_bytes < 4 && M > (1u << (8 * key_bytes))) || !aligned(phi, 4)))
    return DIALSORT_ERR_INVALID_ARG;
  if (inv != nullptr && !aligned(inv, key_bytes)) return DIALSORT_ERR_INVALID_ARG;
  if (n > 0 && (keys == nullptr || out == nullptr || !aligned(keys, key_bytes) || !aligned(out, key_bytes)))
    return DIALSORT_ERR_INVALID_ARG;
  const size_t hb = sort_h_bytes(U);
  const ReconLayout L = recon_layout(U, n);
  if (ws == nullptr || !aligned(ws, 256) || ws_bytes < hb + L.total) return DIALSORT_ERR_WORKSPACE;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  const void *kp, *op, *pp, *ip;
  dialsort_status_t s = kernel_address(n ? keys : nullptr, *dev, &kp);
  if (s == DIALSORT_OK) s = kernel_address(n ? out : nullptr, *dev, &op);
  if (s == DIALSORT_OK) s = kernel_address(phi, *dev, &pp);
  if (s == DIALSORT_OK) s = kernel_address(inv, *dev, &ip);
  if (s != DIALSORT_OK) return s;
  HistPlan plan;
  s = plan_histogram(n, U, key_bytes, 0, nullptr, *dev, &plan);
  if (s == DIALSORT_OK && plan.regime == DIALSORT_REGIME_TWO_LEVEL)  // single-pass regimes only here
    s = plan_histogram(n, U, key_bytes, 0, nullptr, *dev, &plan, false);
  if (s != DIALSORT_OK) return s;
  char* base = static_cast<char*>(ws);
  uint32_t* H = reinterpret_cast<uint32_t*>(base);
  cudaError_t e = cudaMemsetAsync(H, 0, (size_t)U * 4, st);
  if (e == cudaSuccess && n > 0)
    e = launch_histogram(kp, key_bytes, n, U, H, plan, dev->err, st, static_cast<const uint32_t*>(pp), M);
  if (e == cudaSuccess)
    e = launch_projection(H, U, n, const_cast<void*>(op), key_bytes, base + hb, L, *dev, dev->err, st, ip);
  return from_cuda(e);
}

// Chunked ingestion from host memory (the remark after Thm. "Parallel DialSort with pipelined CRN":
// Eq. (1) is a sum over keys, so H can absorb keys as they arrive).  Chunk i is copied into one of two
// device staging buffers on copy_stream while `st` accumulates chunk i - 1; staging buffer i & 1 is
// refilled only after the accumulation of chunk i - 2 has read it.  Workspace: staging[2] | ingestion
// scratch of one chunk | (sort) H | projection scratch.
struct ChunkedLayout {
  size_t stage, ingest, h, recon, total;
};

ChunkedLayout chunked_layout(uint64_t n, uint32_t U, uint32_t key_bytes, uint64_t chunk, bool sort) {
  ChunkedLayout L{};
  L.stage = align_up((size_t)std::min<uint64_t>(chunk, std::max<uint64_t>(n, 1)) * key_bytes, 256);
  L.ingest = hist_ws_bytes(std::min(chunk, n), U, key_bytes);
  L.h = sort ? sort_h_bytes(U) : 0;
  L.recon = sort ? recon_layout(U, n).total : 0;
  L.total = 2 * L.stage + L.ingest + L.h + L.recon;
  return L;
}

dialsort_status_t chunked_impl(const void* host_keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint64_t chunk,
                               uint32_t* H, void* out, void* ws, size_t ws_bytes, cudaStream_t st,
                               cudaStream_t cs, bool sort) {
  dialsort_status_t s = check_keys(host_keys, key_bytes, n, U);
  if (s != DIALSORT_OK) return s;
  if (chunk == 0 || cs == nullptr || cs == st) return DIALSORT_ERR_INVALID_ARG;
  if (sort && n > 0 && (out == nullptr || !aligned(out, key_bytes))) return DIALSORT_ERR_INVALID_ARG;
  const ChunkedLayout L = chunked_layout(n, U, key_bytes, chunk, sort);
  if (ws == nullptr || !aligned(ws, 256) || ws_bytes < L.total) return DIALSORT_ERR_WORKSPACE;
  char* base = static_cast<char*>(ws);
  char* stage[2] = {base, base + L.stage};
  void* ingest = L.ingest ? base + 2 * L.stage : nullptr;
  if (sort) H = reinterpret_cast<uint32_t*>(base + 2 * L.stage + L.ingest);
  if (H == nullptr || !aligned(H, 16)) return DIALSORT_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (sort) e = cudaMemsetAsync(H, 0, (size_t)U * 4, st);  // Eq. (1) starts from H = 0
  cudaEvent_t ev[5] = {};  // entry, copied[2], consumed[2]
  for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  // the copies start after the work already queued on `st` (earlier users of the workspace)
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[0], 0);
  const char* src = static_cast<const char*>(host_keys);
  const uint64_t chunks = (n + chunk - 1) / chunk;
  for (uint64_t i = 0; i < chunks && e == cudaSuccess && s == DIALSORT_OK; ++i) {
    const int slot = (int)(i & 1);
    const uint64_t len = std::min(chunk, n - i * chunk);
    if (i >= 2) e = cudaStreamWaitEvent(cs, ev[3 + slot], 0);  // chunk i - 2 has been ingested
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(stage[slot], src + i * chunk * key_bytes, len * key_bytes, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1 + slot], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[1 + slot], 0);
    if (e != cudaSuccess) break;
    s = histogram_impl(stage[slot], key_bytes, len, U, H, nullptr, ingest, L.ingest, st, true);
    if (s == DIALSORT_OK) e = cudaEventRecord(ev[3 + slot], st);
  }
  for (int i = 0; i < 5; ++i)
    if (ev[i]) (void)cudaEventDestroy(ev[i]);  // released once the recorded work has completed
  if (e != cudaSuccess) return from_cuda(e);
  if (s != DIALSORT_OK || !sort) return s;
  return reconstruct_impl(H, U, out, key_bytes, n, base + 2 * L.stage + L.ingest + L.h, L.recon, st);
}

}  // namespace

extern "C" {

size_t dialsort_chunked_workspace_size(uint64_t n, uint32_t U, uint32_t key_bytes, uint64_t chunk_keys, int sort) {
  if (chunk_keys == 0 || (key_bytes != 4 && key_bytes != 2)) return 0;
  return chunked_layout(n, U, key_bytes, chunk_keys, sort != 0).total;
}

dialsort_status_t dialsort_histogram_chunked(const void* host_keys, uint32_t key_bytes, uint64_t n, uint32_t U,
                                             uint64_t chunk_keys, uint32_t* H, void* ws, size_t ws_bytes,
                                             void* stream, void* copy_stream) {
  return chunked_impl(host_keys, key_bytes, n, U, chunk_keys, H, nullptr, ws, ws_bytes, as_stream(stream),
                      static_cast<cudaStream_t>(copy_stream), false);
}

dialsort_status_t dialsort_sort_chunked(const void* host_keys, uint32_t key_bytes, uint64_t n, uint32_t U,
                                        uint64_t chunk_keys, void* out, void* ws, size_t ws_bytes, void* stream,
                                        void* copy_stream) {
  return chunked_impl(host_keys, key_bytes, n, U, chunk_keys, nullptr, out, ws, ws_bytes, as_stream(stream),
                      static_cast<cudaStream_t>(copy_stream), true);
}

size_t dialsort_sort_mapped_workspace_size(uint64_t n, uint32_t U) { return sort_h_bytes(U) + recon_layout(U, n).total; }

dialsort_status_t dialsort_sort_mapped(const void* keys, uint32_t key_bytes, uint64_t n, const uint32_t* phi,
                                       uint32_t M, const void* phi_inv, uint32_t U, void* out, void* ws,
                                       size_t ws_bytes, void* stream) {
  return sort_mapped_impl(keys, key_bytes, n, phi, M, phi_inv, U, out, ws, ws_bytes, as_stream(stream));
}

size_t dialsort_selftest_workspace_size(void) {
  return std::max(offsets_selftest_bytes(), radix_selftest_bytes());
}

dialsort_status_t dialsort_selftest_wait_timeout(int which, void* ws, size_t ws_bytes, void* stream) {
  if (which != 0 && which != 1) return DIALSORT_ERR_INVALID_ARG;
  if (ws == nullptr || !aligned(ws, 256) || ws_bytes < dialsort_selftest_workspace_size())
    return DIALSORT_ERR_WORKSPACE;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  const cudaStream_t st = as_stream(stream);
  return from_cuda(which == 0 ? launch_offsets_selftest(ws, dev->err, st) : launch_radix_selftest(ws, dev->err, st));
}

int dialsort_pageable_host_access(void) {
  const DeviceInfo* dev = device_info();
  return dev ? (dev->pageable ? 1 : 0) : -1;
}

dialsort_status_t dialsort_histogram(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H, void* stream) {
  return histogram_impl(keys, 4, n, U, H, nullptr, nullptr, 0, as_stream(stream));
}

dialsort_status_t dialsort_histogram_u16(const uint16_t* keys, uint64_t n, uint32_t U, uint32_t* H, void* stream) {
  return histogram_impl(keys, 2, n, U, H, nullptr, nullptr, 0, as_stream(stream));
}

dialsort_status_t dialsort_histogram_ex(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H,
                                        const dialsort_hist_config_t* cfg, void* stream) {
  return histogram_impl(keys, key_bytes, n, U, H, cfg, nullptr, 0, as_stream(stream));
}

dialsort_status_t dialsort_histogram_accumulate(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U,
                                               uint32_t* H, void* ws, size_t ws_bytes, void* stream) {
  return histogram_impl(keys, key_bytes, n, U, H, nullptr, ws, ws_bytes, as_stream(stream), true);
}

size_t dialsort_histogram_workspace_size(uint64_t n, uint32_t U, uint32_t key_bytes) {
  return hist_ws_bytes(n, U, key_bytes);
}

dialsort_status_t dialsort_histogram_ws(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, uint32_t* H,
                                        const dialsort_hist_config_t* cfg, void* ws, size_t ws_bytes,
                                        void* stream) {
  return histogram_impl(keys, key_bytes, n, U, H, cfg, ws, ws_bytes, as_stream(stream));
}

dialsort_status_t dialsort_plan_histogram(uint64_t n, uint32_t U, uint32_t key_bytes, uint32_t skew_hint,
                                          dialsort_hist_config_t* cfg) {
  if (cfg == nullptr || U == 0 || (key_bytes != 4 && key_bytes != 2) || skew_hint > 3)
    return DIALSORT_ERR_INVALID_ARG;
  DeviceInfo fallback;  // planning works without a device (152 SMs, 227 KB)
  const DeviceInfo* dev = device_info();
  HistPlan p;
  dialsort_hist_config_t in = *cfg;
  dialsort_status_t s = plan_histogram(n, U, key_bytes, skew_hint, &in, dev ? *dev : fallback, &p);
  if (s != DIALSORT_OK) return s;
  const uint32_t crn_cfg = p.crn == 1 ? 1u : p.crn == 0 ? 2u : 3u;
  uint32_t regime = p.regime;
  // what dialsort_histogram_ws does with aligned keys and a large enough workspace
  if (in.regime == DIALSORT_REGIME_AUTO && !p.tuned &&
      (regime == DIALSORT_REGIME_GLOBAL_CRN || regime == DIALSORT_REGIME_GLOBAL) &&
      (hier_shape_fits(n, U, key_bytes) || two_level_shape_fits(n, U, key_bytes)))
    regime = DIALSORT_REGIME_TWO_LEVEL;
  *cfg = dialsort_hist_config_t{regime, crn_cfg, p.blocks, p.threads, p.replicas, p.cluster, skew_hint};
  return DIALSORT_OK;
}

size_t dialsort_reconstruct_workspace_size(uint32_t U, uint64_t n) { return recon_layout(U, n).total; }

dialsort_status_t dialsort_reconstruct(const uint32_t* H, uint32_t U, uint32_t* out, uint64_t n, void* ws,
                                       size_t ws_bytes, void* stream) {
  return reconstruct_impl(H, U, out, 4, n, ws, ws_bytes, as_stream(stream));
}

dialsort_status_t dialsort_reconstruct_u16(const uint32_t* H, uint32_t U, uint16_t* out, uint64_t n, void* ws,
                                           size_t ws_bytes, void* stream) {
  return reconstruct_impl(H, U, out, 2, n, ws, ws_bytes, as_stream(stream));
}

dialsort_status_t dialsort_offsets(const uint32_t* H, uint32_t U, uint64_t n, void* ws, size_t ws_bytes,
                                   void* stream) {
  if (U == 0 || n >= (1ull << 32) || H == nullptr || !aligned(H, 16)) return DIALSORT_ERR_INVALID_ARG;
  const ReconLayout L = recon_layout(U, n);
  if (ws == nullptr || !aligned(ws, 256) || ws_bytes < L.total) return DIALSORT_ERR_WORKSPACE;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  return from_cuda(launch_projection(H, U, n, nullptr, 4, ws, L, *dev, dev->err, as_stream(stream), nullptr, 1));
}

dialsort_status_t dialsort_read_chunk_offsets(const void* ws, uint32_t U, uint64_t n, uint64_t* chunk_offsets,
                                              void* stream) {
  if (ws == nullptr || chunk_offsets == nullptr || U == 0) return DIALSORT_ERR_INVALID_ARG;
  const ReconLayout L = recon_layout(U, n);
  const char* base = static_cast<const char*>(ws);
  return from_cuda(cudaMemcpyAsync(chunk_offsets, base + L.off_offsets, 8 * (L.num_chunks + 1),
                                   cudaMemcpyDeviceToDevice, as_stream(stream)));
}

size_t dialsort_sort_workspace_size(uint64_t n, uint32_t U) {
  return sort_h_bytes(U) + recon_layout(U, n).total + hist_ws_bytes(n, U, 4);
}

dialsort_status_t dialsort_sort(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* out, void* ws,
                                size_t ws_bytes, void* stream) {
  return sort_impl(keys, 4, n, U, out, ws, ws_bytes, as_stream(stream));
}

dialsort_status_t dialsort_sort_u16(const uint16_t* keys, uint64_t n, uint32_t U, uint16_t* out, void* ws,
                                    size_t ws_bytes, void* stream) {
  return sort_impl(keys, 2, n, U, out, ws, ws_bytes, as_stream(stream));
}

dialsort_status_t dialsort_sort_ex(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, void* out,
                                   const dialsort_hist_config_t* cfg, void* ws, size_t ws_bytes, void* stream) {
  return sort_impl(keys, key_bytes, n, U, out, ws, ws_bytes, as_stream(stream), cfg);
}

uint32_t* dialsort_sort_histogram(void* ws) { return static_cast<uint32_t*>(ws); }

dialsort_status_t dialsort_sort_stage_times(const void* keys, uint32_t key_bytes, uint64_t n, uint32_t U, void* out,
                                            void* ws, size_t ws_bytes, void* stream, float* ms, uint32_t* stages) {
  if (ms == nullptr || stages == nullptr) return DIALSORT_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  cudaEvent_t ev[5] = {};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  dialsort_status_t s = DIALSORT_ERR_CUDA;
  bool fused = false;
  if (e == cudaSuccess && (e = cudaEventRecord(ev[0], st)) == cudaSuccess) {
    s = sort_impl(keys, key_bytes, n, U, out, ws, ws_bytes, st, nullptr, ev + 1, &fused);
    if (s == DIALSORT_OK && (e = cudaEventRecord(ev[4], st)) == cudaSuccess) e = cudaEventSynchronize(ev[4]);
    if (s == DIALSORT_OK && e != cudaSuccess) s = DIALSORT_ERR_CUDA;
  }
  if (s == DIALSORT_OK) {
    if (fused) {  // pass 1 | split + schedule | counting fused with the projection | long runs
      *stages = 4;
      for (int i = 0; i < 4; ++i) cudaEventElapsedTime(ms + i, ev[i], ev[i + 1]);
    } else {
      *stages = 1;
      cudaEventElapsedTime(ms, ev[0], ev[4]);
    }
  }
  for (int i = 0; i < 5; ++i)
    if (ev[i]) (void)cudaEventDestroy(ev[i]);
  return s;
}

dialsort_status_t dialsort_stream_status(void* stream, int sync) {
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  cudaStream_t st = as_stream(stream);
  if (sync && cudaStreamSynchronize(st) != cudaSuccess) return DIALSORT_ERR_CUDA;
  uint32_t word = 0;
  // read and clear the word in stream order
  if (cudaMemcpyAsync(&word, dev->err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return DIALSORT_ERR_CUDA;
  if (cudaMemsetAsync(dev->err, 0, 4, st) != cudaSuccess) return DIALSORT_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DIALSORT_ERR_CUDA;
  if (word & ERRBIT_TIMEOUT) return DIALSORT_ERR_TIMEOUT;
  if (word & ERRBIT_OVERFLOW) return DIALSORT_ERR_OVERFLOW;
  if (word & ERRBIT_KEY_RANGE) return DIALSORT_ERR_KEY_RANGE;
  return DIALSORT_OK;
}

const char* dialsort_status_string(dialsort_status_t s) {
  switch (s) {
    case DIALSORT_OK: return "ok";
    case DIALSORT_ERR_INVALID_ARG: return "invalid argument";
    case DIALSORT_ERR_KEY_RANGE: return "a key was outside [0, U) and was not counted";
    case DIALSORT_ERR_CUDA: return "CUDA runtime error";
    case DIALSORT_ERR_BUDGET: return "request does not fit the HBM budget";
    case DIALSORT_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    case DIALSORT_ERR_BUSY: return "not finished yet";
    case DIALSORT_ERR_OVERFLOW: return "sum(H) exceeds the output capacity";
    case DIALSORT_ERR_WORKSPACE: return "workspace too small or misaligned";
  }
  return "unknown status";
}

int dialsort_device_sm_count(void) {
  const DeviceInfo* dev = device_info();
  return dev ? dev->sms : 0;
}

const char* dialsort_version(void) { return "dialsort-gb300 0.1.0 sm_103a"; }

}  // extern "C"
