// dialsort_reconstruct_noalloc: the ordered projection with its scratch in a
// fixed, library-owned device array instead of a caller-supplied workspace.
//
// Some callers cannot allocate device memory when they call us: a plugin that
// is handed only its input and output buffers by a host framework that owns
// all device memory, or a latency-critical loop that must never take an
// allocator's locks or risk an out-of-memory failure halfway through.  This
// entry point needs nothing from them but H and the output buffer.
//
// The scratch (look-back descriptors, chunk offsets, first chunk of each
// output tile) lives in g_noalloc_scratch below.  Host code may not use that
// symbol as an address: in host code it names a host-side stand-in, and a
// kernel handed it would fault or, where the GPU can reach host memory,
// silently use the wrong memory.  So, once per device and with that device
// current, the first call looks up the array's device address with
// cudaGetSymbolAddress, checks the result, and caches it; every launch gets
// that address.  The first call on a device should therefore come before any
// stream capture.
//
// Every call on a device shares the one array, which keeps the previous
// call's contents.  The parts that must start at zero (the tile ticket and the
// look-back descriptors) are cleared by each call, in stream order, before its
// kernels run; the rest is fully written before it is read.  Calls whose
// kernels overlap on the GPU (different streams, or another thread) race on
// the array and must be serialised by the caller.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace dialsort {
namespace {

constexpr size_t kNoallocScratchBytes = DIALSORT_NOALLOC_SCRATCH_BYTES;  // per device, held until exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDev = 64;
void* g_scratch_ptr[kMaxDev];
cudaError_t g_scratch_err[kMaxDev];
std::once_flag g_scratch_once[kMaxDev];

// Device address of this device's scratch array, looked up once per device.
cudaError_t scratch_address(int dev, void** ptr) {
  std::call_once(g_scratch_once[dev], [dev] {
    void* p = nullptr;
    g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    g_scratch_ptr[dev] = (g_scratch_err[dev] == cudaSuccess) ? p : nullptr;
  });
  *ptr = g_scratch_ptr[dev];
  return g_scratch_err[dev];
}

}  // namespace
}  // namespace dialsort

using namespace dialsort;

extern "C" dialsort_status_t dialsort_reconstruct_noalloc(const uint32_t* H, uint32_t U, uint32_t* out, uint64_t n,
                                                          void* stream) {
  if (U == 0 || n >= (1ull << 32) || H == nullptr || (reinterpret_cast<uintptr_t>(H) & 15u) != 0)
    return DIALSORT_ERR_INVALID_ARG;
  if (n > 0 && (out == nullptr || (reinterpret_cast<uintptr_t>(out) & 3u) != 0)) return DIALSORT_ERR_INVALID_ARG;
  const ReconLayout L = recon_layout(U, n);
  if (L.total > kNoallocScratchBytes) return DIALSORT_ERR_WORKSPACE;  // beyond the fixed scratch
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  void* scratch = nullptr;
  if (scratch_address(dev->device, &scratch) != cudaSuccess || scratch == nullptr) return DIALSORT_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_offsets(H, U, n, scratch, L, dev->err, st);  // clears ticket + descriptors first
  if (e == cudaSuccess) e = launch_expand(H, U, n, out, 4, scratch, L, st);
  return e == cudaSuccess ? DIALSORT_OK : DIALSORT_ERR_CUDA;
}
