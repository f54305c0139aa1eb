// Queries answered from the histogram itself (Sec. "Canonical ordered state"):
// H already holds the ordered multiset, so frequency(k) and presence(k) are one
// read of H[k] and range-count(a, b) is the sum of H over [a, b] -- no output
// array is reconstructed.
//
// frequency / presence: one thread per query, four queries in flight per
// thread (the reads of H are random gathers, bound by memory latency).
// range_count: one warp per query.  The warp reads H[a..b] with 16-byte loads
// over the 4-aligned middle of the range (scalar loads for the ragged ends)
// and reduces with redux.add, so a range of L bins costs about L/128 load
// steps of the warp.
#include "common.cuh"
#include "internal.h"

namespace dialsort {
namespace {

constexpr int kQueryThreads = 256;

__global__ void __launch_bounds__(kQueryThreads) point_query_kernel(const uint32_t* __restrict__ H, uint32_t U,
                                                                    const uint32_t* __restrict__ q, uint64_t m,
                                                                    uint32_t* __restrict__ freq,
                                                                    uint8_t* __restrict__ present) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += 4 * stride) {
    uint32_t k[4], f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t i = i0 + j * stride;
      k[j] = i < m ? __ldg(q + i) : 0xffffffffu;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) f[j] = k[j] < U ? __ldg(H + k[j]) : 0u;  // outside [0, U): no key counted
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t i = i0 + j * stride;
      if (i < m) {
        if (freq != nullptr) freq[i] = f[j];
        if (present != nullptr) present[i] = f[j] != 0u ? 1u : 0u;
      }
    }
  }
}

__global__ void __launch_bounds__(kQueryThreads) range_count_kernel(const uint32_t* __restrict__ H, uint32_t U,
                                                                    const uint32_t* __restrict__ a,
                                                                    const uint32_t* __restrict__ b, uint64_t m,
                                                                    uint32_t* __restrict__ count) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint4* H4 = reinterpret_cast<const uint4*>(H);  // H is 16-byte aligned
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
    const uint64_t lo = __ldg(a + i), hi = __ldg(b + i);
    uint32_t sum = 0;
    if (lo <= hi && lo < U) {
      const uint64_t end = (hi < U ? hi : U - 1u) + 1u;  // exclusive
      const uint64_t body = ((lo + 3u) & ~3ull) < end ? ((lo + 3u) & ~3ull) : end;
      const uint64_t body_end = body + ((end - body) & ~3ull);
      if (lo + lane < body) sum += __ldg(H + lo + lane);  // head: at most 3 bins
      uint64_t j = body / 4u + lane;
      const uint64_t j_end = body_end / 4u;
      for (; j + 96u < j_end; j += 128u) {  // four 16-byte loads in flight per lane
        const uint4 v0 = __ldg(H4 + j), v1 = __ldg(H4 + j + 32u), v2 = __ldg(H4 + j + 64u),
                    v3 = __ldg(H4 + j + 96u);
        sum += (v0.x + v0.y + v0.z + v0.w) + (v1.x + v1.y + v1.z + v1.w) + (v2.x + v2.y + v2.z + v2.w) +
               (v3.x + v3.y + v3.z + v3.w);
      }
      for (; j < j_end; j += 32u) {
        const uint4 v = __ldg(H4 + j);
        sum += v.x + v.y + v.z + v.w;
      }
      if (body_end + lane < end) sum += __ldg(H + body_end + lane);  // tail: at most 3 bins
    }
    sum = __reduce_add_sync(0xffffffffu, sum);  // exact: sum(H) < 2^32
    if (lane == 0) count[i] = sum;
  }
}

int query_grid(uint64_t threads_needed, const DeviceInfo& dev) {
  const uint64_t blocks = (threads_needed + kQueryThreads - 1) / kQueryThreads;
  const uint64_t cap = (uint64_t)dev.sms * 8u;  // 8 CTAs of 256 threads fill an SM
  return (int)(blocks < cap ? blocks : cap);
}

template <class T>
dialsort_status_t resolve(const T* p, const DeviceInfo& dev, T** q) {
  const void* r;
  const dialsort_status_t s = kernel_address(p, dev, &r);
  *q = static_cast<T*>(const_cast<void*>(r));
  return s;
}

dialsort_status_t point_query(const uint32_t* H, uint32_t U, const uint32_t* q, uint64_t m, uint32_t* freq,
                              uint8_t* present, void* stream) {
  if (U == 0 || H == nullptr || (reinterpret_cast<uintptr_t>(H) & 15u) != 0) return DIALSORT_ERR_INVALID_ARG;
  if (m == 0) return DIALSORT_OK;
  if (q == nullptr || (freq == nullptr && present == nullptr) || (reinterpret_cast<uintptr_t>(q) & 3u) != 0 ||
      (reinterpret_cast<uintptr_t>(freq) & 3u) != 0)
    return DIALSORT_ERR_INVALID_ARG;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  dialsort_status_t s;
  uint32_t *h, *qq, *f = nullptr;
  uint8_t* pr = nullptr;
  if ((s = resolve(H, *dev, &h)) != DIALSORT_OK || (s = resolve(q, *dev, &qq)) != DIALSORT_OK) return s;
  if (freq && (s = resolve(freq, *dev, &f)) != DIALSORT_OK) return s;
  if (present && (s = resolve(present, *dev, &pr)) != DIALSORT_OK) return s;
  point_query_kernel<<<query_grid((m + 3) / 4, *dev), kQueryThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      h, U, qq, m, f, pr);
  return cudaGetLastError() == cudaSuccess ? DIALSORT_OK : DIALSORT_ERR_CUDA;
}

}  // namespace
}  // namespace dialsort

using namespace dialsort;

extern "C" {

dialsort_status_t dialsort_frequency(const uint32_t* H, uint32_t U, const uint32_t* q, uint64_t m, uint32_t* freq,
                                     void* stream) {
  if (m > 0 && freq == nullptr) return DIALSORT_ERR_INVALID_ARG;
  return point_query(H, U, q, m, freq, nullptr, stream);
}

dialsort_status_t dialsort_presence(const uint32_t* H, uint32_t U, const uint32_t* q, uint64_t m, uint8_t* present,
                                    void* stream) {
  if (m > 0 && present == nullptr) return DIALSORT_ERR_INVALID_ARG;
  return point_query(H, U, q, m, nullptr, present, stream);
}

dialsort_status_t dialsort_range_count(const uint32_t* H, uint32_t U, const uint32_t* a, const uint32_t* b,
                                       uint64_t m, uint32_t* count, void* stream) {
  if (U == 0 || H == nullptr || (reinterpret_cast<uintptr_t>(H) & 15u) != 0) return DIALSORT_ERR_INVALID_ARG;
  if (m == 0) return DIALSORT_OK;
  if (a == nullptr || b == nullptr || count == nullptr) return DIALSORT_ERR_INVALID_ARG;
  if (((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(count)) & 3u) != 0)
    return DIALSORT_ERR_INVALID_ARG;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  dialsort_status_t s;
  uint32_t *h, *aa, *bb, *c;
  if ((s = resolve(H, *dev, &h)) != DIALSORT_OK || (s = resolve(a, *dev, &aa)) != DIALSORT_OK ||
      (s = resolve(b, *dev, &bb)) != DIALSORT_OK || (s = resolve(count, *dev, &c)) != DIALSORT_OK)
    return s;
  const uint64_t warps = m < (uint64_t)dev->sms * 64u ? m : (uint64_t)dev->sms * 64u;
  range_count_kernel<<<query_grid(warps * 32u, *dev), kQueryThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      h, U, aa, bb, m, c);
  return cudaGetLastError() == cudaSuccess ? DIALSORT_OK : DIALSORT_ERR_CUDA;
}

}  // extern "C"
