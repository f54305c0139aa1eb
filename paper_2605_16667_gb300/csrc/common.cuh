// Device helpers shared by the DialSort kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dialsort {

// Bits of the per-device error word (reported by dialsort_stream_status).
enum : uint32_t {
  ERRBIT_KEY_RANGE = 1u,  // a key >= U was seen and skipped
  ERRBIT_TIMEOUT = 2u,    // a bounded spin-wait gave up
  ERRBIT_OVERFLOW = 4u,   // sum(H) exceeded the output capacity
};

// Spin limit for every device-side wait: after this many polls (each an L2
// round trip plus a 64 ns back-off, about a second in all) the waiter records
// ERRBIT_TIMEOUT and stops waiting.
constexpr uint32_t kSpinLimit = 1u << 21;

__device__ __forceinline__ uint32_t lane_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%laneid;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

// 128-bit streaming load through the non-coherent path, not kept in L1.
__device__ __forceinline__ uint4 ld_stream_v4(const uint4* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// Fire-and-forget add into global memory (resolved in L2).
__device__ __forceinline__ void red_add_global(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void raise_error(uint32_t* err, uint32_t bit) { atomicOr(err, bit); }

}  // namespace dialsort
