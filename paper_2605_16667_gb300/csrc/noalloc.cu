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
// cudaGetSymbolAddress, checks the result, and caches it (a failed look-up is
// not cached: the next call retries); every launch gets that address.  The
// first call on a device should therefore come before any stream capture.
// H and out are checked like dialsort_reconstruct's: device memory of the
// current device, or host memory the device can reach.
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
void* g_scratch_ptr[kMaxDev];  // cached device addresses; only successful look-ups are kept
std::mutex g_scratch_mu;

// Device address of this device's scratch array.  A failed look-up (for
// example one made while a stream is being captured) is not cached: its
// error is cleared and the next call tries again.
cudaError_t scratch_address(int dev, void** ptr) {
  *ptr = nullptr;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();  // leave no sticky error behind for the caller's next CUDA call
      return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  return cudaSuccess;
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
  // H and out are classified exactly as dialsort_reconstruct classifies them: memory of another
  // device, or host memory this device cannot reach, is refused before any launch
  const void* hp;
  const void* op;
  dialsort_status_t s = kernel_address(H, *dev, &hp);
  if (s == DIALSORT_OK) s = kernel_address(n ? out : nullptr, *dev, &op);
  if (s != DIALSORT_OK) return s;
  void* scratch = nullptr;
  if (scratch_address(dev->device, &scratch) != cudaSuccess) return DIALSORT_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t* Hk = static_cast<const uint32_t*>(hp);
  void* outk = n ? const_cast<void*>(op) : static_cast<void*>(out);
  cudaError_t e = launch_offsets(Hk, U, n, scratch, L, dev->err, st);  // clears ticket + descriptors first
  if (e == cudaSuccess) e = launch_expand(Hk, U, n, outk, 4, scratch, L, st);
  return from_cuda(e);
}
